// Retained-profile export / import: the paper computes the KV caches offline,
// stores them, and at query time loads the precomputed caches of a model and
// compression ratio -- a profile -- for every query (Sec. 5, "Offline: KV Cache
// Creation" and "A Navigable Search Space").  A profile here is what operator
// evaluation reads: the rank-ordered retained K / V planes (used slots only),
// their E4M3 block scales, the per-tuple padded offsets and counts, and the
// pooled document states (the proxy's input).  Layout of the host blob:
//
//   ProfileHeader (128 bytes)
//   int64 offsets[T+1]   (document offsets: the table the profile belongs to)
//   int64 offp[T+1]      (padded retained offsets)
//   int32 nkeep[T]
//   Kr, Vr               [layers][hkv][Rp][hd] elements of the retained dtype
//   float scales         [layers][hkv][Rp/64][2]      (E4M3 profiles only)
//   float pooled         [T][d]
//
// Copies are one cudaMemcpy2DAsync per array (the device planes have a stride
// of the cache's capacity, the blob stores the used slots contiguously).
#include <cstring>
#include <string>

#include "kernels.h"

using namespace st;

namespace {

struct ProfileHeader {
  char magic[8];                       // "STKVPRF1"
  int32_t version, layers, hkv, hd, d, model_dtype, kv_dtype, T;
  int64_t R, Rp;
  double r;
  int64_t total_bytes;
  char pad[128 - 8 - 8 * 4 - 2 * 8 - 8 - 8];
};
static_assert(sizeof(ProfileHeader) == 128, "profile header");

int pfail(st_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

struct Sizes {
  size_t off, offp, nkeep, plane_row, planes, scales_row, scales, pooled, total;
};

Sizes sizes(const st_model_cfg& c, size_t esz_kv, int T, int64_t Rp, bool fp8) {
  Sizes z;
  const size_t LH = (size_t)c.layers * c.hkv;
  z.off = (size_t)(T + 1) * 8;
  z.offp = (size_t)(T + 1) * 8;
  z.nkeep = (size_t)T * 4;
  z.plane_row = (size_t)Rp * c.hd * esz_kv;
  z.planes = LH * z.plane_row;
  z.scales_row = fp8 ? (size_t)(Rp / 64) * 2 * sizeof(float) : 0;
  z.scales = LH * z.scales_row;
  z.pooled = (size_t)T * c.d * sizeof(float);
  z.total = sizeof(ProfileHeader) + z.off + z.offp + z.nkeep + 2 * z.planes + z.scales + z.pooled;
  return z;
}

size_t kv_esz(const st_ctx* ctx, int kv_dtype) { return kv_dtype == ST_E4M3 ? 1 : ctx->esz; }

}  // namespace

extern "C" int st_kv_profile_bytes(const st_kv* kv, size_t* bytes) {
  if (!kv || !bytes) return pfail(nullptr, ST_EINVAL, "st_kv_profile_bytes: bad argument");
  if (kv->r <= 0.0) return pfail(kv->ctx, ST_EINVAL, "st_kv_profile_bytes: no retained profile");
  *bytes = sizes(kv->ctx->cfg, kv_esz(kv->ctx, kv->kv_dtype), kv->T, kv->Rp, kv->kv_dtype == ST_E4M3).total;
  return ST_OK;
}

extern "C" int st_kv_export(st_ctx* ctx, const st_kv* kv, void* host, size_t bytes, void* stream) {
  ST_TRACE("st_kv_export");
  if (!ctx || !kv || kv->ctx != ctx || !host) return pfail(ctx, ST_EINVAL, "st_kv_export: bad argument");
  if (kv->r <= 0.0) return pfail(ctx, ST_EINVAL, "st_kv_export: no retained profile");
  const st_model_cfg& c = ctx->cfg;
  const bool fp8 = kv->kv_dtype == ST_E4M3;
  const size_t e = kv_esz(ctx, kv->kv_dtype);
  const Sizes z = sizes(c, e, kv->T, kv->Rp, fp8);
  if (bytes < z.total) return pfail(ctx, ST_EINVAL, "st_kv_export: buffer smaller than st_kv_profile_bytes");
  ProfileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "STKVPRF1", 8);
  h.version = 1;
  h.layers = c.layers;
  h.hkv = c.hkv;
  h.hd = c.hd;
  h.d = c.d;
  h.model_dtype = c.dtype;
  h.kv_dtype = kv->kv_dtype;
  h.T = kv->T;
  h.R = kv->R;
  h.Rp = kv->Rp;
  h.r = kv->r;
  h.total_bytes = (int64_t)z.total;
  char* p = (char*)host;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, kv->off_h.data(), z.off);
  p += z.off;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t LH = (size_t)c.layers * c.hkv;
  const size_t cap_row = (size_t)kv->Rp_cap * c.hd * e;
  auto ck = [&](cudaError_t err) { return err == cudaSuccess; };
  bool ok = ck(cudaMemcpyAsync(p, kv->offp, z.offp, cudaMemcpyDeviceToHost, s));
  p += z.offp;
  ok = ok && ck(cudaMemcpyAsync(p, kv->nkeep, z.nkeep, cudaMemcpyDeviceToHost, s));
  p += z.nkeep;
  if (z.plane_row) {
    ok = ok && ck(cudaMemcpy2DAsync(p, z.plane_row, kv->Kr, cap_row, z.plane_row, LH, cudaMemcpyDeviceToHost, s));
    p += z.planes;
    ok = ok && ck(cudaMemcpy2DAsync(p, z.plane_row, kv->Vr, cap_row, z.plane_row, LH, cudaMemcpyDeviceToHost, s));
    p += z.planes;
  }
  if (z.scales_row) {
    const size_t cap_srow = (size_t)(kv->Rp_cap / 64) * 2 * sizeof(float);
    ok = ok && ck(cudaMemcpy2DAsync(p, z.scales_row, kv->scales, cap_srow, z.scales_row, LH,
                                    cudaMemcpyDeviceToHost, s));
    p += z.scales;
  }
  ok = ok && ck(cudaMemcpyAsync(p, kv->pooled, z.pooled, cudaMemcpyDeviceToHost, s));
  ok = ok && ck(cudaStreamSynchronize(s));
  if (!ok) return pfail(ctx, ST_ECUDA, std::string("st_kv_export: ") + cudaGetErrorString(cudaGetLastError()));
  return ST_OK;
}

extern "C" int st_kv_import(st_ctx* ctx, st_kv* kv, const void* host, size_t bytes, void* stream) {
  ST_TRACE("st_kv_import");
  if (!ctx || !kv || kv->ctx != ctx || !host || bytes < sizeof(ProfileHeader))
    return pfail(ctx, ST_EINVAL, "st_kv_import: bad argument");
  if (kv->src) return pfail(ctx, ST_EINVAL, "st_kv_import: import into a cache of its own, not a profile alias");
  const st_model_cfg& c = ctx->cfg;
  ProfileHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "STKVPRF1", 8) != 0 || h.version != 1)
    return pfail(ctx, ST_EINVAL, "st_kv_import: not a profile blob");
  if (h.layers != c.layers || h.hkv != c.hkv || h.hd != c.hd || h.d != c.d || h.model_dtype != c.dtype)
    return pfail(ctx, ST_EINVAL, "st_kv_import: the profile belongs to another model shape or dtype");
  if (!(h.kv_dtype == c.dtype || (h.kv_dtype == ST_E4M3 && c.dtype == ST_BF16)) || !(h.r > 0.0 && h.r <= 1.0))
    return pfail(ctx, ST_EINVAL, "st_kv_import: bad retained dtype or r");
  if (h.T != kv->T || h.R != kv->R || h.Rp < 0 || h.Rp > kv->Rp_cap || h.Rp % 64)
    return pfail(ctx, ST_EINVAL, "st_kv_import: the profile belongs to another table");
  const bool fp8 = h.kv_dtype == ST_E4M3;
  const size_t e = kv_esz(ctx, h.kv_dtype);
  const Sizes z = sizes(c, e, h.T, h.Rp, fp8);
  if ((int64_t)z.total != h.total_bytes || bytes < z.total)
    return pfail(ctx, ST_EINVAL, "st_kv_import: truncated or inconsistent blob");
  const char* p = (const char*)host + sizeof(h);
  if (std::memcmp(p, kv->off_h.data(), z.off) != 0)
    return pfail(ctx, ST_EINVAL, "st_kv_import: document offsets differ from the cache's table");
  p += z.off;
  // padded offsets must be the prefix sums of pad64(nkeep) within capacity
  {
    const int64_t* offp = (const int64_t*)p;
    const int32_t* nk = (const int32_t*)(p + z.offp);
    if (offp[0] != 0 || offp[h.T] != h.Rp) return pfail(ctx, ST_EINVAL, "st_kv_import: corrupt padded offsets");
    for (int t = 0; t < h.T; ++t) {
      const int64_t L = kv->off_h[t + 1] - kv->off_h[t];
      if (nk[t] < (L > 0 ? 1 : 0) || nk[t] > L || offp[t + 1] - offp[t] != ((nk[t] + 63) & ~63))
        return pfail(ctx, ST_EINVAL, "st_kv_import: corrupt retained counts");
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t LH = (size_t)c.layers * c.hkv;
  const size_t cap_row = (size_t)kv->Rp_cap * c.hd * e;
  auto ck = [&](cudaError_t err) { return err == cudaSuccess; };
  bool ok = ck(cudaMemcpyAsync(kv->offp, p, z.offp, cudaMemcpyHostToDevice, s));
  p += z.offp;
  ok = ok && ck(cudaMemcpyAsync(kv->nkeep, p, z.nkeep, cudaMemcpyHostToDevice, s));
  p += z.nkeep;
  if (z.plane_row) {
    ok = ok && ck(cudaMemcpy2DAsync(kv->Kr, cap_row, p, z.plane_row, z.plane_row, LH, cudaMemcpyHostToDevice, s));
    p += z.planes;
    ok = ok && ck(cudaMemcpy2DAsync(kv->Vr, cap_row, p, z.plane_row, z.plane_row, LH, cudaMemcpyHostToDevice, s));
    p += z.planes;
  }
  if (z.scales_row) {
    const size_t cap_srow = (size_t)(kv->Rp_cap / 64) * 2 * sizeof(float);
    ok = ok && ck(cudaMemcpy2DAsync(kv->scales, cap_srow, p, z.scales_row, z.scales_row, LH,
                                    cudaMemcpyHostToDevice, s));
    p += z.scales;
  }
  ok = ok && ck(cudaMemcpyAsync(kv->pooled, p, z.pooled, cudaMemcpyHostToDevice, s));
  ok = ok && ck(cudaStreamSynchronize(s));
  if (!ok) return pfail(ctx, ST_ECUDA, std::string("st_kv_import: ") + cudaGetErrorString(cudaGetLastError()));
  kv->Rp = h.Rp;
  kv->r = h.r;
  kv->kv_dtype = h.kv_dtype;
  kv->built = false;   // the full cache no longer matches the profile: st_kv_retain needs a new build
  return ST_OK;
}
