// Operator evaluation that allocates no device memory.
//
// Some callers of this library cannot let it call cudaMalloc / cudaFree:
// a query executor that keeps several streams busy cannot afford the implicit
// device synchronisation cudaFree (and at times cudaMalloc) performs, and a
// process whose GPU memory is already claimed by another framework's caching
// allocator can see a fresh cudaMalloc fail although that allocator holds free
// blocks.  For them, st_op_eval_noalloc runs the same kernels as st_op_eval but
// takes its activations from one file-scope device array of fixed size instead
// of the context's workspace.
//
// The array lives in every GPU that loads the library, for the life of the
// process.  Host code cannot use its name as a device address; the address is
// resolved once per device with cudaGetSymbolAddress on the first call made
// with that device current.  All calls share the array and it keeps the last
// call's contents: nothing in it needs to start at zero (every buffer is fully
// written before it is read), and calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "kernels.h"

using namespace st;

namespace {

constexpr size_t kScratchBytes = ST_NOALLOC_SCRATCH_BYTES;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int na_fail(st_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

// Device address of g_scratch on the current device (resolved once per device).
int scratch_address(st_ctx* ctx, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(ctx, ST_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(ctx, ST_EUNSUPPORTED, "st_op_eval_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return na_fail(ctx, ST_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ST_OK;
}

// Aligned sub-buffers of the scratch array for `rows` prompt rows of `tuples` tuples.
struct Slices {
  float *x, *tmp;
  void *xn, *q, *kp, *vp, *o, *h;
  int32_t *pos, *tup, *len, *nk;
};

size_t carve(const st_ctx* ctx, int64_t rows, int64_t tuples, char* base, Slices* s) {
  const st_model_cfg& c = ctx->cfg;
  const size_t e = ctx->esz;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    char* p = base + off;
    off += bytes;
    return (void*)p;
  };
  s->x = (float*)take(rows * c.d * 4);
  s->xn = take(rows * c.d * e);
  s->q = take(rows * c.hq * c.hd * e);
  s->kp = take(rows * c.hkv * c.hd * e);
  s->vp = take(rows * c.hkv * c.hd * e);
  s->o = take(rows * c.hq * c.hd * e);
  s->h = take(rows * c.ffn * e);
  s->tmp = c.dtype == ST_F32 ? (float*)take(rows * 2 * c.ffn * 4) : nullptr;
  s->pos = (int32_t*)take(rows * 4);
  s->tup = (int32_t*)take(tuples * 4);
  s->len = (int32_t*)take(tuples * 4);
  s->nk = (int32_t*)take(tuples * 4);
  return off;
}

// Counts the launch; unlike the other entries it records no profiling events,
// so that this entry creates no CUDA resources at all.
struct Count {
  explicit Count(st_ctx* c) { c->launches++; }
};

int launched(st_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(ctx, ST_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return ST_OK;
}

int gemm(st_ctx* ctx, const void* A, const void* W, int M, int N, int K, EpiParams ep, float* tmp,
         void* h_out, cudaStream_t s) {
  ep.M = M;
  ep.N = N;
  if (ctx->cfg.dtype == ST_BF16) {
    Count L(ctx);
    int rc = gemm_tc((const bf16*)A, (const bf16*)W, M, N, K, ep, ctx->dstatus, s);
    if (rc != ST_OK) return na_fail(ctx, rc, "tcgen05 GEMM: unsupported shape or tensor-map encoding failed");
  } else if (ep.mode == EPI_SWIGLU) {
    EpiParams e2 = ep;
    e2.mode = EPI_STORE_F32;
    e2.out = tmp;
    e2.ld = N;
    {
      Count L(ctx);
      gemm_simt<float>((const float*)A, (const float*)W, M, N, K, e2, s);
    }
    Count L2(ctx);
    swiglu_from_f32(tmp, M, N / 2, (float*)h_out, s);
  } else {
    Count L(ctx);
    gemm_simt<float>((const float*)A, (const float*)W, M, N, K, ep, s);
  }
  return launched(ctx);
}

int norm(st_ctx* ctx, const float* x, int64_t rows, void* xn, cudaStream_t s) {
  const st_model_cfg& c = ctx->cfg;
  Count L(ctx);
  if (c.dtype == ST_BF16) rmsnorm_rows<bf16>(x, rows, c.d, c.eps, (bf16*)xn, nullptr, s);
  else rmsnorm_rows<float>(x, rows, c.d, c.eps, (float*)xn, nullptr, s);
  return launched(ctx);
}

#define NA_RC(x)                   \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != ST_OK) return rc_;  \
  } while (0)

}  // namespace

extern "C" int st_op_eval_noalloc(st_ctx* ctx, const st_kv* kv, const st_operator* op,
                                  const int32_t* tuple_ids_dev, int32_t n, float* logits_dev,
                                  int32_t* labels_dev, void* stream) {
  if (!ctx) return ST_EINVAL;
  if (!kv || !op || kv->ctx != ctx || n < 0) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: bad argument");
  if (n == 0) return ST_OK;
  if (!tuple_ids_dev || !logits_dev || !labels_dev) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: NULL buffer");
  if (kv->r <= 0.0) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: no retained profile (call st_kv_retain)");
  if (op->desc.r > kv->r) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: operator r exceeds the retained profile's r");
  const st_model_cfg& c = ctx->cfg;
  if (kv->max_len + op->desc.P > c.max_pos) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: document + prompt exceeds max_pos");
  const int P = op->desc.P;
  const int64_t M = (int64_t)n * P;
  Slices w;
  const size_t need = carve(ctx, M, n, nullptr, &w);
  if (need > kScratchBytes)
    return na_fail(ctx, ST_EINVAL,
                   "st_op_eval_noalloc: " + std::to_string(n) + " tuples x " + std::to_string(P) +
                       " prompt rows need " + std::to_string(need) + " bytes of scratch, more than the " +
                       std::to_string(kScratchBytes) + "-byte static scratch; pass fewer tuples per call");
  void* base = nullptr;
  NA_RC(scratch_address(ctx, &base));
  carve(ctx, M, n, (char*)base, &w);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int qd = c.hq * c.hd, kd = c.hkv * c.hd, nqkv = qd + 2 * kd;
  const size_t kr_e = kv->kv_dtype == ST_E4M3 ? 1 : ctx->esz;
  {
    Count L(ctx);
    eval_rowinfo(tuple_ids_dev, n, P, kv->off, op->desc.r, w.tup, w.len, w.nk, w.pos, s);
  }
  {
    Count L(ctx);
    embed_prompt(op->prompt, P, M, ctx->embed, c.dtype, c.d, w.x, s);
  }
  NA_RC(launched(ctx));
  for (int l = 0; l < c.layers; ++l) {
    const LayerW& LW = ctx->layers[l];
    NA_RC(norm(ctx, w.x, M, w.xn, s));
    EpiParams ep;
    ep.mode = EPI_QKV;
    ep.q = w.q;
    ep.kbase = w.kp;
    ep.vbase = w.vp;
    ep.kv_sg = c.hd;
    ep.kv_sr = kd;
    ep.pos = w.pos;
    ep.rope = ctx->rope;
    ep.hq = c.hq;
    ep.hkv = c.hkv;
    ep.hd = c.hd;
    ep.qkv_f16 = kv->kv_dtype == ST_E4M3 ? 1 : 0;
    NA_RC(gemm(ctx, w.xn, LW.wqkv, (int)M, nqkv, c.d, ep, w.tmp, nullptr, s));
    AttnParams a;
    a.mode = 1;
    a.q = w.q;
    a.o = w.o;
    a.hq = c.hq;
    a.hkv = c.hkv;
    a.hd = c.hd;
    a.scale = 1.0f / std::sqrt((float)c.hd);
    a.Kr = (const char*)kv->Kr + (size_t)l * c.hkv * kv->Rp_cap * c.hd * kr_e;
    a.Vr = (const char*)kv->Vr + (size_t)l * c.hkv * kv->Rp_cap * c.hd * kr_e;
    a.scales = kv->scales + (size_t)l * c.hkv * (kv->Rp_cap / 64) * 2;
    a.Rp_cap = kv->Rp_cap;
    a.offp = kv->offp;
    a.tup = w.tup;
    a.nk = w.nk;
    a.kp = w.kp;
    a.vp = w.vp;
    a.n = n;
    a.P = P;
    a.kv_dtype = kv->kv_dtype;
    {
      Count L(ctx);
      int rc = ST_OK;
      if (c.dtype == ST_F32) attn_simt<float, float>(a, s);
      else rc = attn_tc_eval(a, ctx->dstatus, s);
      if (rc != ST_OK) return na_fail(ctx, rc, "tcgen05 attention: unsupported shape or tensor-map encoding failed");
    }
    NA_RC(launched(ctx));
    EpiParams eo;
    eo.mode = EPI_RESID;
    eo.x = w.x;
    eo.ld = c.d;
    NA_RC(gemm(ctx, w.o, LW.wo, (int)M, c.d, qd, eo, w.tmp, nullptr, s));
    NA_RC(norm(ctx, w.x, M, w.xn, s));
    EpiParams eg;
    eg.mode = EPI_SWIGLU;
    eg.h = w.h;
    eg.ld = c.ffn;
    NA_RC(gemm(ctx, w.xn, LW.wgu, (int)M, 2 * c.ffn, c.d, eg, w.tmp, w.h, s));
    EpiParams ed;
    ed.mode = EPI_RESID;
    ed.x = w.x;
    ed.ld = c.d;
    NA_RC(gemm(ctx, w.h, LW.wd, (int)M, c.d, c.ffn, ed, w.tmp, nullptr, s));
  }
  {
    Count L(ctx);
    label_head(w.x, n, P, c.d, c.eps, ctx->w_lm, c.dtype, op->labels, op->desc.n_labels, op->bias,
               op->desc.kind, op->desc.theta_pos, op->desc.theta_neg, logits_dev, labels_dev, s);
  }
  return launched(ctx);
}
