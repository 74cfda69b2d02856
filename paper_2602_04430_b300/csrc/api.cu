// C ABI of libstretto: argument validation, memory, chunking and kernel
// sequencing of the three steps of Sec. 5 (offline cache creation, retention,
// online operator evaluation).  Every arithmetic step runs in a CUDA kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"

using namespace st;

namespace {

thread_local std::string g_err;   // errors raised before a context exists

int fail(const st_ctx* ctx, int code, const std::string& msg) {
  if (ctx) const_cast<st_ctx*>(ctx)->err = msg;
  else g_err = msg;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, ST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define CKLAUNCH()                                                                       \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, ST_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

int dev_alloc(st_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return ST_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, ST_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return ST_OK;
}

int grow(st_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return ST_OK;
  if (b.external)
    return fail(ctx, ST_ENOMEM, "the workspace given to st_set_workspace holds " + std::to_string(b.bytes) +
                                    " bytes, this call needs " + std::to_string(bytes));
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  int rc = dev_alloc(ctx, &b.p, bytes);
  if (rc == ST_OK) b.bytes = bytes;
  return rc;
}

// Carves aligned sub-buffers out of one workspace.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <typename T> T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = (T*)(base + off);
    off += n * sizeof(T);
    return p;
  }
};

int n_keep_host(int64_t L, double r) {
  volatile double rl = r * (double)L;   // rounded product, then the add (no fused multiply-add)
  double n = std::floor(rl + 0.5);
  if (n < 1) n = 1;
  if (n > (double)L) n = (double)L;
  return (int)n;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---- chunk plan of kv_build: whole tuples, at most `cap` rows per chunk
struct Chunk { int t0, t1; int64_t r0, rows; };

std::vector<Chunk> plan_chunks(const std::vector<int64_t>& off, int64_t cap) {
  std::vector<Chunk> out;
  int T = (int)off.size() - 1;
  int t = 0;
  while (t < T) {
    Chunk c{t, t, off[t], 0};
    while (c.t1 < T && (c.t1 == c.t0 || off[c.t1 + 1] - off[c.t0] <= cap)) c.t1++;
    c.rows = off[c.t1] - off[c.t0];
    out.push_back(c);
    t = c.t1;
  }
  return out;
}

struct BuildWs {
  float *x, *inv_rms, *mu, *s2, *tmp, *ssq;
  float *qm, *qM;   // full Expected Attention moments of the chunk's tuples (else null)
  void *xn, *q, *o, *h;
  int32_t *rowtup, *pos;
};

size_t build_ws_bytes(const st_ctx* ctx, int64_t rows, int64_t tuples, BuildWs* w, void* base) {
  const st_model_cfg& c = ctx->cfg;
  Carve cv(base ? base : (void*)0);
  const size_t e = ctx->esz;
  BuildWs ws;
  ws.x = cv.take<float>(rows * c.d);
  ws.inv_rms = cv.take<float>(rows);
  ws.mu = cv.take<float>(tuples * c.hkv * c.hd);
  ws.s2 = cv.take<float>(tuples * c.hkv * c.hd);
  ws.xn = cv.take<char>(rows * c.d * e);
  ws.q = cv.take<char>(rows * c.hq * c.hd * e);
  ws.o = cv.take<char>(rows * c.hq * c.hd * e);
  ws.h = cv.take<char>(rows * c.ffn * e);
  ws.tmp = c.dtype == ST_F32 ? cv.take<float>(rows * 2 * c.ffn) : nullptr;
  ws.ssq = cv.take<float>(rows * (c.d / 128));
  ws.rowtup = cv.take<int32_t>(rows);
  ws.pos = cv.take<int32_t>(rows);
  ws.qm = ws.qM = nullptr;
  if (ctx->score_mode == ST_SCORE_EA_FULL) {
    ws.qm = cv.take<float>(tuples * c.hkv * c.hd);
    ws.qM = cv.take<float>(tuples * c.hkv * c.hd * c.hd);
  }
  if (w) *w = ws;
  return cv.off + 256;
}

const int64_t kDefaultBuildRows = 1 << 20;
const int64_t kDefaultEvalRows = 1 << 18;

}  // namespace

// ------------------------------------------------------------------ profiling
namespace st {
static cudaEvent_t take_event(st_ctx* ctx) {
  if (!ctx->prof.pool.empty()) {
    cudaEvent_t e = ctx->prof.pool.back();
    ctx->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
thread_local bool tls_no_prof = false;

Launch::Launch(st_ctx* c, cudaStream_t st, int fam, double fl, double by)
    : ctx(c), s(st), family(fam), flops(fl), bytes(by), timed(c->prof.on && !tls_no_prof) {
  ctx->launches++;
  if (timed) {
    rec.family = fam;
    rec.flops = fl;
    rec.bytes = by;
    rec.a = take_event(ctx);
    rec.b = take_event(ctx);
    cudaEventRecord(rec.a, s);
  }
}
Launch::~Launch() {
  if (timed) {
    cudaEventRecord(rec.b, s);
    ctx->prof.pending.push_back(rec);
  }
}
}  // namespace st

// ------------------------------------------------------------------ internal step helpers
namespace st {

// One projection: dispatches to the tensor-core GEMM (bf16) or the CUDA-core GEMM (f32).
int project(st_ctx* ctx, const void* A, const void* W, int M, int N, int K, EpiParams ep,
            float* tmp, void* h_out, cudaStream_t s, bool f16_ops) {
  const st_model_cfg& c = ctx->cfg;
  ep.M = M;
  ep.N = N;
  ep.act_f16 = f16_ops ? 1 : 0;
  if (M <= 0) return ST_OK;
  const double flops = 2.0 * M * (double)N * K;
  const double bytes = ((double)M * K + (double)N * K) * ctx->esz;
  if (c.dtype == ST_BF16) {
    Launch L(ctx, s, ST_PROF_GEMM, flops, bytes);
    int rc = gemm_tc(A, W, M, N, K, ep, ctx->dstatus, s, f16_ops);
    if (rc != ST_OK) return fail(ctx, rc, "tcgen05 GEMM: unsupported shape or tensor-map encoding failed");
  } else if (ep.mode == EPI_SWIGLU) {
    EpiParams e2 = ep;
    e2.mode = EPI_STORE_F32;
    e2.out = tmp;
    e2.ld = N;
    {
      Launch L(ctx, s, ST_PROF_GEMM, flops, bytes);
      gemm_simt<float>((const float*)A, (const float*)W, M, N, K, e2, s);
    }
    Launch L2(ctx, s, ST_PROF_OTHER, 0, 0);
    swiglu_from_f32(tmp, M, N / 2, (float*)h_out, s);
  } else {
    Launch L(ctx, s, ST_PROF_GEMM, flops, bytes);
    gemm_simt<float>((const float*)A, (const float*)W, M, N, K, ep, s);
  }
  CKLAUNCH();
  return ST_OK;
}

int rmsnorm(st_ctx* ctx, const float* x, int64_t rows, void* xn, float* inv, cudaStream_t s) {
  const st_model_cfg& c = ctx->cfg;
  Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
  if (c.dtype == ST_BF16) rmsnorm_rows<__half>(x, rows, c.d, c.eps, (__half*)xn, inv, s);
  else rmsnorm_rows<float>(x, rows, c.d, c.eps, (float*)xn, inv, s);
  CKLAUNCH();
  return ST_OK;
}

int attention(st_ctx* ctx, const AttnParams& a, const int32_t* items, int n_items, cudaStream_t s) {
  const st_model_cfg& c = ctx->cfg;
  Launch L(ctx, s, ST_PROF_ATTN, 0, 0);
  int rc = ST_OK;
  if (c.dtype == ST_F32) {
    attn_simt<float, float>(a, s);
  } else if (a.mode == 0) {
    rc = attn_tc_prefill(a, items, n_items, ctx->dstatus, s);
  } else {
    rc = attn_tc_eval(a, ctx->dstatus, s);
  }
  if (rc != ST_OK) return fail(ctx, rc, "tcgen05 attention: unsupported shape or tensor-map encoding failed");
  CKLAUNCH();
  return ST_OK;
}

#define RC(x)                       \
  do {                              \
    int rc_ = (x);                  \
    if (rc_ != ST_OK) return rc_;   \
  } while (0)

void set_norm_in(EpiParams& ep, const float* ssq, const st_model_cfg& c) {
  ep.ssq_in = ssq;
  ep.ssq_parts = c.d / 128;
  ep.norm_d = c.d;
  ep.eps = c.eps;
}
void set_norm_out(EpiParams& ep, void* xb, float* ssq) {
  ep.xb = xb;
  ep.ssq_out = ssq;
}

}  // namespace st

// ================================================================== context
extern "C" const char* st_version(void) { return "stretto-b300 0.1 (sm_103a)"; }

extern "C" const char* st_last_error(const st_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_err.c_str();
}

extern "C" int st_create(const st_model_cfg* cfg, const void* const* weights, void* stream,
                         st_ctx** out) {
  ST_TRACE("st_create");
  st_ctx* ctx = nullptr;
  if (!cfg || !weights || !out) return fail(nullptr, ST_EINVAL, "st_create: NULL argument");
  *out = nullptr;
  const st_model_cfg& c = *cfg;
  if (c.layers < 1 || c.d < 128 || c.d % 128 || c.hq < 1 || c.hkv < 1 || c.hq % c.hkv ||
      c.ffn < 128 || c.ffn % 128 || c.vocab < 2 || c.max_pos < 2 || !(c.eps > 0) ||
      !(c.rope_theta > 0))
    return fail(nullptr, ST_EINVAL, "st_create: invalid model shape");
  if (c.dtype == ST_F32) {
    if (c.hd != 32 && c.hd != 64) return fail(nullptr, ST_EUNSUPPORTED, "f32 model: hd must be 32 or 64");
    if (((c.hq + 2 * c.hkv) * c.hd) % (4 * c.hd) || c.d % 128 || (c.hq * c.hd) % 16)
      return fail(nullptr, ST_EUNSUPPORTED, "f32 model: projection widths not tileable");
  } else if (c.dtype == ST_BF16) {
    if (c.hd != 64) return fail(nullptr, ST_EUNSUPPORTED, "bf16 model: hd must be 64");
    const int nq = (c.hq + 2 * c.hkv) * c.hd;
    if (!gemm_tc_supported(128, nq, c.d) || !gemm_tc_supported(128, c.d, c.hq * c.hd) ||
        !gemm_tc_supported(128, 2 * c.ffn, c.d) || !gemm_tc_supported(128, c.d, c.ffn))
      return fail(nullptr, ST_EUNSUPPORTED, "bf16 model: projection shapes not supported by the tcgen05 GEMM");
  } else {
    return fail(nullptr, ST_EINVAL, "st_create: dtype must be ST_F32 or ST_BF16");
  }
  ctx = new st_ctx();
  ctx->cfg = c;
  ctx->esz = c.dtype == ST_F32 ? 4 : 2;
  cudaGetDevice(&ctx->device);
  cudaStream_t s = S(stream);
  const size_t e = ctx->esz;
  const size_t d = c.d, qd = (size_t)c.hq * c.hd, kd = (size_t)c.hkv * c.hd, f = c.ffn;
  auto cleanup_fail = [&](int rc) { st_destroy(ctx); return rc; };
  auto copy = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
  };
  int rc;
  if ((rc = dev_alloc(ctx, &ctx->embed, c.vocab * d * e))) { g_err = ctx->err; return cleanup_fail(rc); }
  if ((rc = dev_alloc(ctx, &ctx->w_lm, c.vocab * d * e))) { g_err = ctx->err; return cleanup_fail(rc); }
  copy(ctx->embed, weights[0], c.vocab * d * e);
  copy(ctx->w_lm, weights[1 + 7 * c.layers], c.vocab * d * e);
  ctx->layers.resize(c.layers);
  for (int l = 0; l < c.layers; ++l) {
    LayerW& L = ctx->layers[l];
    const void* const* w = weights + 1 + 7 * l;
    if ((rc = dev_alloc(ctx, &L.wqkv, (qd + 2 * kd) * d * e)) ||
        (rc = dev_alloc(ctx, &L.wo, d * qd * e)) || (rc = dev_alloc(ctx, &L.wgu, 2 * f * d * e)) ||
        (rc = dev_alloc(ctx, &L.wd, d * f * e))) {
      g_err = ctx->err;
      return cleanup_fail(rc);
    }
    copy(L.wqkv, w[0], qd * d * e);
    copy((char*)L.wqkv + qd * d * e, w[1], kd * d * e);
    copy((char*)L.wqkv + (qd + kd) * d * e, w[2], kd * d * e);
    copy(L.wo, w[3], d * qd * e);
    // gate / up interleaved in blocks of 128 rows: [g0..g127, u0..u127, g128.., u128..]
    cudaMemcpy2DAsync(L.wgu, 256 * d * e, w[4], 128 * d * e, 128 * d * e, f / 128, cudaMemcpyDefault, s);
    cudaMemcpy2DAsync((char*)L.wgu + 128 * d * e, 256 * d * e, w[5], 128 * d * e, 128 * d * e,
                      f / 128, cudaMemcpyDefault, s);
    copy(L.wd, w[6], d * f * e);
  }
  // BF16 model: the projection and LM-head weights are held as IEEE half (every
  // bf16 value of a weight's magnitude converts exactly), the operand type of
  // the tcgen05 GEMMs, whose activation operands are half too (3 more mantissa
  // bits than bf16 where most of the rounding error arises).
  if (c.dtype == ST_BF16) {
    bf16_to_f16(ctx->w_lm, (size_t)c.vocab * d, s);
    for (auto& L : ctx->layers) {
      bf16_to_f16(L.wqkv, (qd + 2 * kd) * d, s);
      bf16_to_f16(L.wo, d * qd, s);
      bf16_to_f16(L.wgu, 2 * f * d, s);
      bf16_to_f16(L.wd, d * f, s);
    }
  }
  // RoPE table: cos / sin of pos * theta^(-2i/hd), computed in double on the host.
  const int half = c.hd / 2;
  std::vector<float2> tab((size_t)c.max_pos * half);
  for (int p = 0; p < c.max_pos; ++p)
    for (int i = 0; i < half; ++i) {
      double ang = (double)p * std::pow((double)c.rope_theta, -2.0 * i / c.hd);
      tab[(size_t)p * half + i] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  if ((rc = dev_alloc(ctx, (void**)&ctx->rope, tab.size() * sizeof(float2)))) {
    g_err = ctx->err;
    return cleanup_fail(rc);
  }
  copy(ctx->rope, tab.data(), tab.size() * sizeof(float2));
  // the same table position-fastest ([hd/2][max_pos]): the tcgen05 GEMM's
  // epilogue reads one frequency for 32 consecutive rows in one coalesced load
  {
    std::vector<float2> tt(tab.size());
    for (int p = 0; p < c.max_pos; ++p)
      for (int i = 0; i < half; ++i) tt[(size_t)i * c.max_pos + p] = tab[(size_t)p * half + i];
    if ((rc = dev_alloc(ctx, (void**)&ctx->rope_t, tt.size() * sizeof(float2)))) {
      g_err = ctx->err;
      return cleanup_fail(rc);
    }
    copy(ctx->rope_t, tt.data(), tt.size() * sizeof(float2));
  }
  if ((rc = dev_alloc(ctx, (void**)&ctx->dstatus, sizeof(int32_t)))) {
    g_err = ctx->err;
    return cleanup_fail(rc);
  }
  cudaMemsetAsync(ctx->dstatus, 0, sizeof(int32_t), s);
  cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    g_err = std::string("st_create: ") + cudaGetErrorString(err);
    return cleanup_fail(ST_ECUDA);
  }
  *out = ctx;
  return ST_OK;
}

extern "C" void st_destroy(st_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  cudaFree(ctx->embed);
  cudaFree(ctx->w_lm);
  for (auto& L : ctx->layers) {
    cudaFree(L.wqkv);
    cudaFree(L.wo);
    cudaFree(L.wgu);
    cudaFree(L.wd);
  }
  cudaFree(ctx->rope);
  cudaFree(ctx->rope_t);
  cudaFree(ctx->dstatus);
  if (!ctx->ws_build.external) cudaFree(ctx->ws_build.p);
  if (!ctx->ws_eval.external) cudaFree(ctx->ws_eval.p);
  cudaFree(ctx->ws_casc.p);
  cudaFree(ctx->ws_map.p);
  cudaFree(ctx->ws_score.p);
  cudaFree(ctx->ws_pcasc.p);
  cudaFree(ctx->rope_avg);
  for (auto& r : ctx->prof.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->prof.pool) cudaEventDestroy(e);
  delete ctx;
}

extern "C" int st_reserve(st_ctx* ctx, int64_t build_rows, int64_t eval_rows) {
  if (!ctx || build_rows < 0 || eval_rows < 0) return fail(ctx, ST_EINVAL, "st_reserve: bad argument");
  if (build_rows > 0) {
    ctx->build_rows_cap = build_rows;
    RC(grow(ctx, ctx->ws_build, build_ws_bytes(ctx, build_rows, build_rows, nullptr, nullptr)));
  }
  if (eval_rows > 0) {
    ctx->eval_rows_cap = eval_rows;
    RC(grow(ctx, ctx->ws_eval, eval_bufs(ctx, eval_rows, eval_rows, nullptr, nullptr)));
  }
  return ST_OK;
}

extern "C" size_t st_workspace_size(const st_ctx* ctx, int which, int64_t rows) {
  if (!ctx || rows <= 0) return 0;
  // a chunk of `rows` rows holds at most `rows` tuples (build) or pairs (eval)
  if (which == ST_WS_BUILD) return build_ws_bytes(ctx, rows, rows, nullptr, nullptr);
  if (which == ST_WS_EVAL) return eval_bufs(ctx, rows, rows, nullptr, nullptr);
  return 0;
}

extern "C" size_t st_workspace_held(const st_ctx* ctx, int which) {
  if (!ctx) return 0;
  auto own = [](const DevBuf& b) { return b.external ? (size_t)0 : b.bytes; };
  if (which == ST_WS_BUILD) return own(ctx->ws_build);
  if (which == ST_WS_EVAL) return own(ctx->ws_eval);
  if (which == ST_WS_ANY)
    return own(ctx->ws_build) + own(ctx->ws_eval) + own(ctx->ws_casc) + own(ctx->ws_map) + own(ctx->ws_score) +
           own(ctx->ws_pcasc);
  return 0;
}

extern "C" int st_set_workspace(st_ctx* ctx, int which, void* dev, size_t bytes) {
  if (!ctx || (which != ST_WS_BUILD && which != ST_WS_EVAL) || (dev == nullptr) != (bytes == 0) ||
      (reinterpret_cast<uintptr_t>(dev) & 255u))
    return fail(ctx, ST_EINVAL, "st_set_workspace: bad argument (which, a 256-byte aligned pointer and its size, "
                                "or NULL and 0)");
  DevBuf& b = which == ST_WS_BUILD ? ctx->ws_build : ctx->ws_eval;
  if (!b.external && b.p) cudaFree(b.p);   // the library's own buffer (waits for its users)
  b.p = dev;
  b.bytes = bytes;
  b.external = dev != nullptr;
  return ST_OK;
}

// ================================================================== KV caches
extern "C" int st_kv_alloc(st_ctx* ctx, const int64_t* offsets_host, int32_t T, st_kv** out) {
  if (!ctx || !offsets_host || !out || T < 1) return fail(ctx, ST_EINVAL, "st_kv_alloc: bad argument");
  *out = nullptr;
  const st_model_cfg& c = ctx->cfg;
  if (offsets_host[0] != 0) return fail(ctx, ST_EINVAL, "st_kv_alloc: offsets[0] must be 0");
  int64_t max_len = 0, rp = 0;
  for (int t = 0; t < T; ++t) {
    int64_t L = offsets_host[t + 1] - offsets_host[t];
    if (L < 1) return fail(ctx, ST_EINVAL, "st_kv_alloc: every document needs >= 1 token");
    if (L > c.max_pos - 1) return fail(ctx, ST_EINVAL, "st_kv_alloc: document longer than max_pos - 1");
    if (L > 16384) return fail(ctx, ST_EUNSUPPORTED, "st_kv_alloc: documents are limited to 16384 tokens");
    max_len = std::max(max_len, L);
    rp += (L + 63) & ~63LL;
  }
  st_kv* kv = new st_kv();
  kv->ctx = ctx;
  kv->T = T;
  kv->R = offsets_host[T];
  kv->Rp_cap = rp;
  kv->max_len = (int32_t)max_len;
  kv->off_h.assign(offsets_host, offsets_host + T + 1);
  const size_t e = ctx->esz, LH = (size_t)c.layers * c.hkv;
  int rc = ST_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == ST_OK) rc = dev_alloc(ctx, p, bytes);
  };
  A((void**)&kv->off, (T + 1) * sizeof(int64_t));
  A(&kv->K, LH * kv->R * c.hd * e);
  A(&kv->V, LH * kv->R * c.hd * e);
  A((void**)&kv->scores, LH * kv->R * sizeof(float));
  A((void**)&kv->pooled, (size_t)T * c.d * sizeof(float));
  A((void**)&kv->rank, LH * kv->R * sizeof(int32_t));
  A(&kv->Kr, LH * rp * c.hd * e);
  A(&kv->Vr, LH * rp * c.hd * e);
  A((void**)&kv->scales, LH * (rp / 64) * 2 * sizeof(float));
  A((void**)&kv->offp, (T + 1) * sizeof(int64_t));
  A((void**)&kv->nkeep, T * sizeof(int32_t));
  A((void**)&kv->status, sizeof(int32_t));
  if (rc != ST_OK) {
    st_kv_free(kv);
    return rc;
  }
  cudaMemcpy(kv->off, offsets_host, (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  cudaMemset(kv->status, 0, sizeof(int32_t));
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    st_kv_free(kv);
    return fail(ctx, ST_ECUDA, std::string("st_kv_alloc: ") + cudaGetErrorString(err));
  }
  // prefill work items for the tensor-core attention: (tuple, 32-position query block)
  const int qb = 128 / (c.hq / c.hkv);   // document positions per 128-row query block
  std::vector<int32_t> items;
  for (int t = 0; t < T; ++t) {
    int64_t L = offsets_host[t + 1] - offsets_host[t];
    for (int64_t j = 0; j < L; j += qb) {
      items.push_back(t);
      items.push_back((int32_t)j);
    }
  }
  kv->n_items = (int64_t)items.size() / 2;
  rc = dev_alloc(ctx, (void**)&kv->items, items.size() * sizeof(int32_t));
  if (rc != ST_OK) {
    st_kv_free(kv);
    return rc;
  }
  cudaMemcpy(kv->items, items.data(), items.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  // item ranges per tuple, for chunked builds
  kv->item_start.resize(T + 1);
  int64_t acc = 0;
  for (int t = 0; t < T; ++t) {
    kv->item_start[t] = acc;
    acc += (offsets_host[t + 1] - offsets_host[t] + qb - 1) / qb;
  }
  kv->item_start[T] = acc;
  // the retained cache starts zeroed: tiles that run past a tuple's padded segment
  // (into unused capacity) then read finite values, which the masks discard
  cudaMemset(kv->Kr, 0, LH * rp * c.hd * e);
  cudaMemset(kv->Vr, 0, LH * rp * c.hd * e);
  cudaMemset(kv->scales, 0, LH * (rp / 64) * 2 * sizeof(float));
  err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    st_kv_free(kv);
    return fail(ctx, ST_ECUDA, std::string("st_kv_alloc: ") + cudaGetErrorString(err));
  }
  *out = kv;
  return ST_OK;
}

extern "C" void st_kv_free(st_kv* kv) {
  if (!kv) return;
  cudaDeviceSynchronize();
  if (kv->src) {   // a profile: the full cache and offsets belong to its source
    void* own[] = {kv->rank, kv->Kr, kv->Vr, kv->scales, kv->offp, kv->nkeep, kv->status};
    for (void* p : own) cudaFree(p);
    delete kv;
    return;
  }
  void* ptrs[] = {kv->off, kv->K, kv->V, kv->scores, kv->pooled, kv->rank, kv->Kr, kv->Vr,
                  kv->scales, kv->offp, kv->nkeep, kv->status, kv->items, kv->tok, kv->iota,
                  kv->out_logits, kv->out_labels};
  for (void* p : ptrs) cudaFree(p);
  delete kv;
}

extern "C" int st_kv_profile_alloc(st_ctx* ctx, st_kv* src, double r_max, st_kv** out) {
  if (!ctx || !src || !out || src->ctx != ctx || src->src)
    return fail(ctx, ST_EINVAL, "st_kv_profile_alloc: bad argument (a cache of this context, not itself a profile)");
  if (!(r_max > 0.0 && r_max <= 1.0)) return fail(ctx, ST_EINVAL, "st_kv_profile_alloc: r_max must lie in (0, 1]");
  *out = nullptr;
  const st_model_cfg& c = ctx->cfg;
  int64_t rp = 0;
  for (int t = 0; t < src->T; ++t) rp += (n_keep_host(src->off_h[t + 1] - src->off_h[t], r_max) + 63) & ~63LL;
  st_kv* kv = new st_kv();
  kv->ctx = ctx;
  kv->src = src;
  kv->r_max = r_max;
  kv->T = src->T;
  kv->R = src->R;
  kv->Rp_cap = rp;
  kv->max_len = src->max_len;
  kv->off_h = src->off_h;
  kv->off = src->off;
  kv->K = src->K;
  kv->V = src->V;
  kv->scores = src->scores;
  kv->pooled = src->pooled;
  kv->items = src->items;
  kv->n_items = src->n_items;
  kv->item_start = src->item_start;
  const size_t e = ctx->esz, LH = (size_t)c.layers * c.hkv;
  int rc = ST_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == ST_OK) rc = dev_alloc(ctx, p, bytes);
  };
  A((void**)&kv->rank, LH * kv->R * sizeof(int32_t));
  A(&kv->Kr, LH * rp * c.hd * e);
  A(&kv->Vr, LH * rp * c.hd * e);
  A((void**)&kv->scales, LH * (rp / 64) * 2 * sizeof(float));
  A((void**)&kv->offp, (kv->T + 1) * sizeof(int64_t));
  A((void**)&kv->nkeep, kv->T * sizeof(int32_t));
  A((void**)&kv->status, sizeof(int32_t));
  if (rc != ST_OK) {
    st_kv_free(kv);
    return rc;
  }
  // zeroed like a cache's own retained buffers (tiles past a segment read finite values)
  cudaMemset(kv->Kr, 0, LH * rp * c.hd * e);
  cudaMemset(kv->Vr, 0, LH * rp * c.hd * e);
  cudaMemset(kv->scales, 0, LH * (rp / 64) * 2 * sizeof(float));
  cudaMemset(kv->status, 0, sizeof(int32_t));
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    st_kv_free(kv);
    return fail(ctx, ST_ECUDA, std::string("st_kv_profile_alloc: ") + cudaGetErrorString(err));
  }
  *out = kv;
  return ST_OK;
}

extern "C" int st_kv_build(st_ctx* ctx, st_kv* kv, const int32_t* tokens_dev, void* stream) {
  ST_TRACE("st_kv_build");
  if (!ctx || !kv || !tokens_dev || kv->ctx != ctx) return fail(ctx, ST_EINVAL, "st_kv_build: bad argument");
  if (kv->src) return fail(ctx, ST_EINVAL, "st_kv_build: a profile (st_kv_profile_alloc) is built through its source");
  const st_model_cfg& c = ctx->cfg;
  cudaStream_t s = S(stream);
  const bool ea_full = ctx->score_mode == ST_SCORE_EA_FULL;
  if (ea_full && !ea_full_supported(c.hd))
    return fail(ctx, ST_EUNSUPPORTED, "st_kv_build: full Expected Attention scores need hd 32 or 64");
  if (ea_full && (int64_t)kv->max_len + ctx->score_horizon > c.max_pos)
    return fail(ctx, ST_EINVAL, "st_kv_build: document length + scoring horizon exceeds max_pos");
  const int64_t cap = std::max<int64_t>(ctx->build_rows_cap > 0 ? ctx->build_rows_cap : kDefaultBuildRows,
                                        kv->max_len);
  std::vector<Chunk> chunks = plan_chunks(kv->off_h, cap);
  int64_t max_rows = 0, max_tup = 0;
  for (auto& ch : chunks) {
    max_rows = std::max(max_rows, ch.rows);
    max_tup = std::max<int64_t>(max_tup, ch.t1 - ch.t0);
  }
  RC(grow(ctx, ctx->ws_build, build_ws_bytes(ctx, max_rows, max_tup, nullptr, nullptr)));
  BuildWs w;
  build_ws_bytes(ctx, max_rows, max_tup, &w, ctx->ws_build.p);
  const size_t e = ctx->esz;
  const int qd = c.hq * c.hd, kd = c.hkv * c.hd, nqkv = qd + 2 * kd;
  for (const Chunk& ch : chunks) {
    const int M = (int)ch.rows;
    {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      build_rowinfo(kv->off, ch.t0, ch.t1, ch.r0, ch.rows, w.rowtup, w.pos, s);
    }
    // bf16 path: the gather writes layer 0's normalised rows too; afterwards every
    // residual epilogue leaves half(x) and the row's partial sums of squares, and
    // the next projection applies 1/rms in its epilogue.
    const bool fused = c.dtype == ST_BF16;
    {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      if (fused)
        embed_norm_rows(tokens_dev + ch.r0, ch.rows, (const bf16*)ctx->embed, c.d, c.vocab, c.eps, w.x,
                        (__half*)w.xn, ctx->dstatus, s);
      else
        embed_rows<float>(tokens_dev + ch.r0, ch.rows, (const float*)ctx->embed, c.d, c.vocab, w.x, ctx->dstatus, s);
    }
    CKLAUNCH();
    for (int l = 0; l < c.layers; ++l) {
      const LayerW& LW = ctx->layers[l];
      char* Kl = (char*)kv->K + (size_t)l * c.hkv * kv->R * c.hd * e;
      char* Vl = (char*)kv->V + (size_t)l * c.hkv * kv->R * c.hd * e;
      if (!fused) RC(rmsnorm(ctx, w.x, ch.rows, w.xn, nullptr, s));
      EpiParams ep;
      if (fused && l > 0) set_norm_in(ep, w.ssq, c);
      ep.mode = EPI_QKV;
      ep.q = w.q;
      ep.kbase = Kl + (size_t)ch.r0 * c.hd * e;
      ep.vbase = Vl + (size_t)ch.r0 * c.hd * e;
      ep.kv_sg = kv->R * c.hd;
      ep.kv_sr = c.hd;
      ep.pos = w.pos;
      ep.rope = ctx->rope;
      ep.rope_t = ctx->rope_t;
      ep.rope_np = c.max_pos;
      ep.hq = c.hq;
      ep.hkv = c.hkv;
      ep.hd = c.hd;
      RC(project(ctx, w.xn, LW.wqkv, M, nqkv, c.d, ep, w.tmp, nullptr, s));
      // causal attention of the document onto itself
      AttnParams a;
      a.mode = 0;
      a.q = w.q;
      a.o = w.o;
      a.hq = c.hq;
      a.hkv = c.hkv;
      a.hd = c.hd;
      a.scale = 1.0f / std::sqrt((float)c.hd);
      a.K = Kl;
      a.V = Vl;
      a.R = kv->R;
      a.off = kv->off;
      a.rowtup = w.rowtup;
      a.pos = w.pos;
      a.r0 = ch.r0;
      a.rows = ch.rows;
      const int64_t i0 = kv->item_start[ch.t0], i1 = kv->item_start[ch.t1];
      RC(attention(ctx, a, kv->items + 2 * i0, (int)(i1 - i0), s));
      // retention statistics and scores of this layer
      if (ea_full) {
        Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
        float* sl = kv->scores + (size_t)l * c.hkv * kv->R;
        if (c.dtype == ST_BF16)
          ea_full_scores<bf16>((const bf16*)w.q, (const bf16*)Kl, (const bf16*)Vl, kv->R, kv->off, ch.t0, ch.t1,
                               ch.r0, c.hq, c.hkv, c.hd, ctx->rope, ctx->rope_avg, w.qm, w.qM, sl, s);
        else
          ea_full_scores<float>((const float*)w.q, (const float*)Kl, (const float*)Vl, kv->R, kv->off, ch.t0,
                                ch.t1, ch.r0, c.hq, c.hkv, c.hd, ctx->rope, ctx->rope_avg, w.qm, w.qM, sl, s);
      } else {
        Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
        if (c.dtype == ST_BF16) {
          qstats<bf16>((const bf16*)w.q, kv->off, ch.t0, ch.t1, ch.r0, c.hq, c.hkv, c.hd, w.mu, w.s2, s);
        } else {
          qstats<float>((const float*)w.q, kv->off, ch.t0, ch.t1, ch.r0, c.hq, c.hkv, c.hd, w.mu, w.s2, s);
        }
      }
      if (!ea_full) {
        Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
        float* sl = kv->scores + (size_t)l * c.hkv * kv->R;
        if (c.dtype == ST_BF16)
          ea_scores<bf16>((const bf16*)Kl, (const bf16*)Vl, kv->R, c.hkv, c.hd, ch.r0, ch.rows,
                          w.rowtup, ch.t0, w.mu, w.s2, sl, s);
        else
          ea_scores<float>((const float*)Kl, (const float*)Vl, kv->R, c.hkv, c.hd, ch.r0, ch.rows,
                           w.rowtup, ch.t0, w.mu, w.s2, sl, s);
      }
      CKLAUNCH();
      EpiParams eo;
      eo.mode = EPI_RESID;
      eo.x = w.x;
      eo.ld = c.d;
      if (fused) set_norm_out(eo, w.xn, w.ssq);
      RC(project(ctx, w.o, LW.wo, M, c.d, qd, eo, w.tmp, nullptr, s));
      if (!fused) RC(rmsnorm(ctx, w.x, ch.rows, w.xn, nullptr, s));
      EpiParams eg;
      eg.mode = EPI_SWIGLU;
      eg.h = w.h;
      eg.ld = c.ffn;
      if (fused) set_norm_in(eg, w.ssq, c);
      RC(project(ctx, w.xn, LW.wgu, M, 2 * c.ffn, c.d, eg, w.tmp, w.h, s));
      EpiParams ed;
      ed.mode = EPI_RESID;
      ed.x = w.x;
      ed.ld = c.d;
      if (fused && l + 1 < c.layers) set_norm_out(ed, w.xn, w.ssq);
      if (fused && l + 1 == c.layers) ed.ssq_out = w.ssq;   // for the pooled state's 1/rms
      RC(project(ctx, w.h, LW.wd, M, c.d, c.ffn, ed, w.tmp, nullptr, s));
    }
    // pooled final-normed last-layer document state (bf16 path: 1/rms from the
    // last residual epilogue's partial sums of squares)
    if (!fused) RC(rmsnorm(ctx, w.x, ch.rows, nullptr, w.inv_rms, s));
    {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      pool_rows(w.x, fused ? nullptr : w.inv_rms, w.ssq, c.d / 128, c.eps, kv->off, ch.t0, ch.t1,
                ch.r0, c.d, kv->pooled, s);
    }
    CKLAUNCH();
  }
  kv->built = true;
  kv->r = 0.0;
  return ST_OK;
}

extern "C" int st_kv_retain(st_ctx* ctx, st_kv* kv, double r, int32_t kv_dtype, void* stream) {
  ST_TRACE("st_kv_retain");
  if (!ctx || !kv || kv->ctx != ctx) return fail(ctx, ST_EINVAL, "st_kv_retain: bad argument");
  if (!(r > 0.0 && r <= 1.0)) return fail(ctx, ST_EINVAL, "st_kv_retain: r must lie in (0, 1]");
  const st_model_cfg& c = ctx->cfg;
  if (!(kv_dtype == c.dtype || (kv_dtype == ST_E4M3 && c.dtype == ST_BF16)))
    return fail(ctx, ST_EINVAL, "st_kv_retain: kv_dtype must be the model dtype or ST_E4M3 (bf16 models)");
  if (!(kv->src ? kv->src->built : kv->built)) return fail(ctx, ST_EINVAL, "st_kv_retain: cache not built");
  if (r > kv->r_max)
    return fail(ctx, ST_EINVAL, "st_kv_retain: r exceeds the r_max this profile was allocated for");
  cudaStream_t s = S(stream);
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    nkeep_offp(kv->off, kv->T, r, kv->nkeep, kv->offp, s);
  }
  CKLAUNCH();
  int64_t rp = 0, kept = 0;
  for (int t = 0; t < kv->T; ++t) {
    int n = n_keep_host(kv->off_h[t + 1] - kv->off_h[t], r);
    kept += n;
    rp += (n + 63) & ~63;
  }
  RetainParams p;
  p.scores = kv->scores;
  p.K = kv->K;
  p.V = kv->V;
  p.rank = kv->rank;
  p.Kr = kv->Kr;
  p.Vr = kv->Vr;
  p.scales = kv->scales;
  p.off = kv->off;
  p.offp = kv->offp;
  p.nkeep = kv->nkeep;
  p.status = kv->status;
  p.T = kv->T;
  p.layers = c.layers;
  p.hkv = c.hkv;
  p.hd = c.hd;
  p.max_len = kv->max_len;
  p.R = kv->R;
  p.Rp_cap = kv->Rp_cap;
  p.in_dtype = c.dtype;
  p.out_dtype = kv_dtype;
  // algorithmic bytes: read scores + the kept K/V rows, write rank + retained K/V (+ scales)
  const double LH = (double)c.layers * c.hkv;
  const double out_e = kv_dtype == ST_E4M3 ? 1.0 : (double)ctx->esz;
  const double bytes = LH * (kv->R * 8.0 + kept * 2.0 * c.hd * ctx->esz + rp * 2.0 * c.hd * out_e);
  {
    Launch L(ctx, s, ST_PROF_RETAIN, 0, bytes);
    int rc = retain(p, s);
    if (rc != ST_OK) return fail(ctx, rc, "st_kv_retain: unsupported retained dtype for this head dim");
  }
  CKLAUNCH();
  kv->Rp = rp;
  kv->r = r;
  kv->kv_dtype = kv_dtype;
  return ST_OK;
}

extern "C" int st_kv_indices(st_ctx* ctx, const st_kv* kv, double r, int32_t* idx_dev, int64_t* off_dev,
                             void* stream) {
  ST_TRACE("st_kv_indices");
  if (!ctx || !kv || kv->ctx != ctx || !off_dev) return fail(ctx, ST_EINVAL, "st_kv_indices: bad argument");
  if (!(r > 0.0 && r <= 1.0)) return fail(ctx, ST_EINVAL, "st_kv_indices: r must lie in (0, 1]");
  if (!(kv->src ? kv->src->built : kv->built) || kv->r <= 0.0)
    return fail(ctx, ST_EINVAL, "st_kv_indices: no ranking (st_kv_retain after st_kv_build)");
  const st_model_cfg& c = ctx->cfg;
  std::vector<int64_t> o(kv->T + 1, 0);
  for (int t = 0; t < kv->T; ++t) o[t + 1] = o[t] + n_keep_host(kv->off_h[t + 1] - kv->off_h[t], r);
  cudaStream_t s = S(stream);
  // pageable source: the call returns once it has been staged
  if (cudaMemcpyAsync(off_dev, o.data(), o.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(ctx, ST_ECUDA, std::string("st_kv_indices: ") + cudaGetErrorString(cudaGetLastError()));
  if (idx_dev) {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    gather_indices(kv->rank, kv->off, off_dev, kv->T, c.layers * c.hkv, kv->R, o[kv->T], idx_dev, ctx->dstatus, s);
  }
  CKLAUNCH();
  return ST_OK;
}

extern "C" int st_kv_status(st_ctx* ctx, st_kv* kv, void* stream) {
  if (!ctx || !kv) return fail(ctx, ST_EINVAL, "st_kv_status: bad argument");
  int32_t h = 0;
  CK(cudaMemcpyAsync(&h, kv->status, sizeof(int32_t), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  CK(cudaMemsetAsync(kv->status, 0, sizeof(int32_t), S(stream)));
  if (h != ST_OK)
    return fail(ctx, h, h == ST_ECHECK ? "device status: an offset check of the checked build failed in retention"
                                       : "device status: NaN retention score");
  return ST_OK;
}

extern "C" int st_status(st_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, ST_EINVAL, "st_status: NULL context");
  int32_t h = 0;
  CK(cudaMemcpyAsync(&h, ctx->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int32_t), S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  if (h != ST_OK)
    return fail(ctx, h, h == ST_ETIMEOUT ? "device status: a bounded wait timed out"
                        : h == ST_ENAN   ? "device status: non-finite logits in a map operator step"
                        : h == ST_EINVAL ? "device status: a token id outside the vocabulary"
                        : h == ST_ERANGE ? "device status: a tuple id outside [0, T)"
                        : h == ST_ECHECK ? "device status: an index or offset check of the checked build failed"
                                         : "device status: error");
  return ST_OK;
}

extern "C" int st_kv_view(const st_kv* kv, int32_t which, void** ptr, size_t* bytes) {
  if (!kv || !ptr || !bytes) return fail(nullptr, ST_EINVAL, "st_kv_view: bad argument");
  const st_model_cfg& c = kv->ctx->cfg;
  const size_t e = kv->ctx->esz, LH = (size_t)c.layers * c.hkv;
  const size_t re = (kv->kv_dtype == ST_E4M3) ? 1 : e;
  switch (which) {
    case ST_VIEW_K: *ptr = kv->K; *bytes = LH * kv->R * c.hd * e; break;
    case ST_VIEW_V: *ptr = kv->V; *bytes = LH * kv->R * c.hd * e; break;
    case ST_VIEW_SCORES: *ptr = kv->scores; *bytes = LH * kv->R * 4; break;
    case ST_VIEW_POOLED: *ptr = kv->pooled; *bytes = (size_t)kv->T * c.d * 4; break;
    case ST_VIEW_RANK: *ptr = kv->rank; *bytes = LH * kv->R * 4; break;
    case ST_VIEW_KR: *ptr = kv->Kr; *bytes = LH * kv->Rp_cap * c.hd * re; break;
    case ST_VIEW_VR: *ptr = kv->Vr; *bytes = LH * kv->Rp_cap * c.hd * re; break;
    case ST_VIEW_SCALES: *ptr = kv->scales; *bytes = LH * (kv->Rp_cap / 64) * 8; break;
    case ST_VIEW_OFFP: *ptr = kv->offp; *bytes = (size_t)(kv->T + 1) * 8; break;
    case ST_VIEW_NKEEP: *ptr = kv->nkeep; *bytes = (size_t)kv->T * 4; break;
    default: return fail(kv->ctx, ST_EINVAL, "st_kv_view: unknown view");
  }
  return ST_OK;
}

extern "C" int st_kv_read(const st_kv* kv, int32_t which, void* dst_dev, size_t bytes,
                          void* stream) {
  if (!kv || !dst_dev) return fail(nullptr, ST_EINVAL, "st_kv_read: bad argument");
  void* p = nullptr;
  size_t n = 0;
  RC(st_kv_view(kv, which, &p, &n));
  const st_ctx* ctx = kv->ctx;
  CK(cudaMemcpyAsync(dst_dev, p, std::min(n, bytes), cudaMemcpyDeviceToDevice, S(stream)));
  return ST_OK;
}

extern "C" int st_kv_read_at(const st_kv* kv, int32_t which, size_t offset, void* dst_dev, size_t bytes,
                             void* stream) {
  if (!kv || !dst_dev) return fail(nullptr, ST_EINVAL, "st_kv_read_at: bad argument");
  void* p = nullptr;
  size_t n = 0;
  RC(st_kv_view(kv, which, &p, &n));
  if (offset > n || bytes > n - offset) return fail(kv->ctx, ST_EINVAL, "st_kv_read_at: range outside the view");
  const st_ctx* ctx = kv->ctx;
  CK(cudaMemcpyAsync(dst_dev, (const char*)p + offset, bytes, cudaMemcpyDeviceToDevice, S(stream)));
  return ST_OK;
}

extern "C" int st_gemm(st_ctx* ctx, const void* A_dev, const void* W_dev, int32_t M, int32_t N,
                       int32_t K, float* C_dev, void* stream) {
  ST_TRACE("st_gemm");
  if (!ctx || !A_dev || !W_dev || !C_dev || M < 0 || N <= 0 || K <= 0)
    return fail(ctx, ST_EINVAL, "st_gemm: bad argument");
  if (ctx->cfg.dtype == ST_BF16 && !gemm_tc_supported(M > 0 ? M : 1, N, K))
    return fail(ctx, ST_EUNSUPPORTED, "st_gemm: bf16 needs N % 256 == 0 and K % 64 == 0");
  if (ctx->cfg.dtype == ST_F32 && (N % 128 || K % 16))
    return fail(ctx, ST_EUNSUPPORTED, "st_gemm: f32 needs N % 128 == 0 and K % 16 == 0");
  EpiParams ep;
  ep.mode = EPI_STORE_F32;
  ep.out = C_dev;
  ep.ld = N;
  return project(ctx, A_dev, W_dev, M, N, K, ep, nullptr, nullptr, S(stream), false);
}

// ================================================================== operators
extern "C" int st_op_create(st_ctx* ctx, const st_op* op, st_operator** out) {
  if (!ctx || !op || !out || !op->prompt || !op->label_ids) return fail(ctx, ST_EINVAL, "st_op_create: bad argument");
  *out = nullptr;
  const st_model_cfg& c = ctx->cfg;
  if (op->P < 1 || op->P > 256) return fail(ctx, ST_EINVAL, "st_op_create: P must be in 1..256");
  if (op->kind == ST_OP_FILTER ? op->n_labels != 2 : (op->kind != ST_OP_CLASSIFY || op->n_labels < 2 || op->n_labels > 8))
    return fail(ctx, ST_EINVAL, "st_op_create: filters take 2 labels, classify 2..8");
  if (!(op->r > 0.0 && op->r <= 1.0)) return fail(ctx, ST_EINVAL, "st_op_create: r must lie in (0, 1]");
  for (int i = 0; i < op->P; ++i)
    if (op->prompt[i] < 0 || op->prompt[i] >= c.vocab) return fail(ctx, ST_EINVAL, "st_op_create: prompt id out of range");
  for (int i = 0; i < op->n_labels; ++i)
    if (op->label_ids[i] < 0 || op->label_ids[i] >= c.vocab) return fail(ctx, ST_EINVAL, "st_op_create: label id out of range");
  st_operator* o = new st_operator();
  o->desc = *op;
  o->desc.prompt = nullptr;
  o->desc.label_ids = nullptr;
  o->desc.bias = nullptr;
  int rc = ST_OK;
  if ((rc = dev_alloc(ctx, (void**)&o->prompt, op->P * 4)) ||
      (rc = dev_alloc(ctx, (void**)&o->labels, op->n_labels * 4)) ||
      (rc = dev_alloc(ctx, (void**)&o->bias, op->n_labels * 4))) {
    st_op_free(o);
    return rc;
  }
  std::vector<float> b(op->n_labels, 0.f);
  if (op->bias) b.assign(op->bias, op->bias + op->n_labels);
  cudaMemcpy(o->prompt, op->prompt, op->P * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(o->labels, op->label_ids, op->n_labels * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(o->bias, b.data(), op->n_labels * 4, cudaMemcpyHostToDevice);
  *out = o;
  return ST_OK;
}

extern "C" void st_op_free(st_operator* op) {
  if (!op) return;
  cudaFree(op->prompt);
  cudaFree(op->labels);
  cudaFree(op->bias);
  delete op;
}

namespace st {

size_t eval_bufs(const st_ctx* ctx, int64_t rows, int64_t pairs, char* base, EvalBufs* w) {
  const st_model_cfg& c = ctx->cfg;
  const size_t e = ctx->esz;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    char* p = base + off;
    off += bytes;
    return (void*)p;
  };
  // a pair's 128-row attention blocks: at most ceil(256 G / 128) (P <= 256)
  const int64_t max_blocks = (256LL * (c.hq / c.hkv) + 127) / 128;
  EvalBufs b;
  b.x = (float*)take(rows * c.d * 4);
  b.xn = take(rows * c.d * e);
  b.q = take(rows * c.hq * c.hd * e);
  b.kp = take(rows * c.hkv * c.hd * e);
  b.vp = take(rows * c.hkv * c.hd * e);
  b.o = take(rows * c.hq * c.hd * e);
  b.h = take(rows * c.ffn * e);
  b.tmp = c.dtype == ST_F32 ? (float*)take(rows * 2 * c.ffn * 4) : nullptr;
  b.ssq = (float*)take(rows * (c.d / 128) * 4);
  b.pos = (int32_t*)take(rows * 4);
  b.tok = (int32_t*)take(rows * 4);
  b.rowpair = (int32_t*)take(rows * 4);
  b.tup = (int32_t*)take(pairs * 4);
  b.len = (int32_t*)take(pairs * 4);
  b.nk = (int32_t*)take(pairs * 4);
  b.prow = (int32_t*)take(pairs * 4);
  b.pP = (int32_t*)take(pairs * 4);
  b.pop = (int32_t*)take(pairs * 4);
  b.pj = (int32_t*)take(pairs * 4);
  // (pieces: a split pair has up to 255 entries per row block, within SPLIT_SLOTS slots)
  const int64_t entries = pairs * max_blocks + (ctx->split_keys > 0 ? SPLIT_SLOTS : 0);
  b.order = (int32_t*)take(entries * WORK_INTS * 4);
  b.psplit = b.mlist = b.cnt = nullptr;
  b.part = nullptr;
  if (ctx->split_keys > 0 && c.dtype == ST_BF16) {
    b.psplit = (int32_t*)take(pairs * 4);
    b.mlist = (int32_t*)take((size_t)SPLIT_SLOTS * 16);
    b.cnt = (int32_t*)take(16);      // slots, merge entries, list entries
    b.part = (float*)take((size_t)SPLIT_SLOTS * c.hkv * 128 * SPLIT_STRIDE * 4);
  }
  if (w) *w = b;
  return off + 256;
}

int make_opset(st_ctx* ctx, const st_kv* kv, int n_ops, const st_operator* const* ops,
               const int32_t* const* tuple_ids, const int32_t* n, float* const* logits,
               int32_t* const* labels, OpSet* os, int64_t* rows_total, int* pairs_total) {
  if (!kv || kv->ctx != ctx || n_ops < 1 || n_ops > ST_MAX_OPS || !ops || !tuple_ids || !n ||
      !logits || !labels || !os)
    return fail(ctx, ST_EINVAL, "operator evaluation: bad argument (1 to 8 operators)");
  if (kv->r <= 0.0) return fail(ctx, ST_EINVAL, "operator evaluation: no retained profile (call st_kv_retain)");
  const st_model_cfg& c = ctx->cfg;
  *os = OpSet();
  os->n_ops = n_ops;
  os->T = kv->T;
  int64_t rows = 0;
  int64_t pairs = 0;
  for (int k = 0; k < n_ops; ++k) {
    const st_operator* op = ops[k];
    if (!op || n[k] < 0) return fail(ctx, ST_EINVAL, "operator evaluation: bad operator or count");
    if (n[k] > 0 && (!tuple_ids[k] || !logits[k] || !labels[k]))
      return fail(ctx, ST_EINVAL, "operator evaluation: NULL buffer");
    if (op->desc.r > kv->r) return fail(ctx, ST_EINVAL, "operator evaluation: operator r exceeds the retained profile's r");
    if (kv->max_len + op->desc.P > c.max_pos) return fail(ctx, ST_EINVAL, "operator evaluation: document + prompt exceeds max_pos");
    OpDev& o = os->op[k];
    o.tuple_ids = tuple_ids[k];
    o.prompt = op->prompt;
    o.labels = op->labels;
    o.bias = op->bias;
    o.logits = logits[k];
    o.out_labels = labels[k];
    o.row0 = rows;
    o.r = op->desc.r;
    o.n = n[k];
    o.P = op->desc.P;
    o.n_labels = op->desc.n_labels;
    o.kind = op->desc.kind;
    o.pair0 = (int)pairs;
    o.theta_pos = op->desc.theta_pos;
    o.theta_neg = op->desc.theta_neg;
    rows += (int64_t)n[k] * op->desc.P;
    pairs += n[k];
  }
  if (pairs > (1LL << 30)) return fail(ctx, ST_EINVAL, "operator evaluation: too many (operator, tuple) pairs");
  *rows_total = rows;
  *pairs_total = (int)pairs;
  return ST_OK;
}

int64_t opset_rows(const OpSet& os, int p0, int p1) {
  int64_t r = 0;
  for (int k = 0; k < os.n_ops; ++k) {
    const OpDev& o = os.op[k];
    const int a = std::max(p0, o.pair0), b = std::min(p1, o.pair0 + o.n);
    if (b > a) r += (int64_t)(b - a) * o.P;
  }
  return r;
}

int map_head(st_ctx* ctx, int np, int t, const EvalBufs& w, const MapCtx& mp, cudaStream_t s);

int eval_chunk(st_ctx* ctx, const st_kv* kv, const OpSet& os, int p0, int p1, int64_t row_base,
               int64_t M, const EvalBufs& w, cudaStream_t s, const MapCtx* mp, float* qscore) {
  const st_model_cfg& c = ctx->cfg;
  const int np = p1 - p0;
  if (np <= 0) return ST_OK;
  const int qd = c.hq * c.hd, kd = c.hkv * c.hd, nqkv = qd + 2 * kd;
  const size_t kr_e = kv->kv_dtype == ST_E4M3 ? 1 : ctx->esz;
  const bool fused = c.dtype == ST_BF16;
  const int G = c.hq / c.hkv;
  int n_entries = 0;   // attention work list entries: ceil(P G / 128) per pair
  for (int k = 0; k < os.n_ops; ++k) {
    const OpDev& o = os.op[k];
    const int a = std::max(p0, o.pair0), b = std::min(p1, o.pair0 + o.n);
    if (b > a) n_entries += (b - a) * ((o.P * G + 127) / 128);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    eval_pairs(os, p0, np, row_base, kv->off, w.tup, w.len, w.nk, w.prow, w.pP, w.pop, w.pj, ctx->dstatus, s);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    eval_rows(os, p0, row_base, M, kv->off, w.pos, w.tok, w.rowpair, ctx->dstatus, s);
  }
  if (c.dtype == ST_BF16) {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    eval_worklist(w.nk, w.pP, w.tup, w.prow, kv->offp, np, G, 0, ctx->longest_first != 0, w.order,
                  ctx->split_keys, w.psplit, w.mlist, w.cnt, s);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    if (c.dtype == ST_BF16) embed_rows<bf16>(w.tok, M, (const bf16*)ctx->embed, c.d, c.vocab, w.x, ctx->dstatus, s);
    else embed_rows<float>(w.tok, M, (const float*)ctx->embed, c.d, c.vocab, w.x, ctx->dstatus, s);
  }
  CKLAUNCH();
  for (int l = 0; l < c.layers; ++l) {
    const LayerW& LW = ctx->layers[l];
    if (!fused || l == 0) RC(rmsnorm(ctx, w.x, M, w.xn, nullptr, s));
    EpiParams ep;
    if (fused && l > 0) set_norm_in(ep, w.ssq, c);
    ep.mode = EPI_QKV;
    ep.q = w.q;
    ep.kbase = w.kp;
    ep.vbase = w.vp;
    ep.kv_sg = c.hd;
    ep.kv_sr = kd;
    ep.pos = w.pos;
    ep.rope = ctx->rope;
    ep.rope_t = ctx->rope_t;
    ep.rope_np = c.max_pos;
    ep.hq = c.hq;
    ep.hkv = c.hkv;
    ep.hd = c.hd;
    ep.qkv_f16 = kv->kv_dtype == ST_E4M3 ? 1 : 0;
    RC(project(ctx, w.xn, LW.wqkv, M, nqkv, c.d, ep, w.tmp, nullptr, s));
    if (mp) {
      // map operator: the prompt's keys and values of this layer into the decode cache
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      copy_prompt_kv(w.kp, (char*)mp->K + (size_t)l * mp->layer_elems * ctx->esz, np, os.op[0].P, mp->S, kd,
                     ctx->esz, s);
      CKLAUNCH();
      Launch L2(ctx, s, ST_PROF_OTHER, 0, 0);
      copy_prompt_kv(w.vp, (char*)mp->V + (size_t)l * mp->layer_elems * ctx->esz, np, os.op[0].P, mp->S, kd,
                     ctx->esz, s);
      CKLAUNCH();
    }
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
    a.prow = w.prow;
    a.pP = w.pP;
    a.rowpair = w.rowpair;
    a.work = w.order;
    a.n_work = n_entries;
    if (w.cnt) {
      // split-KV: the entry count is the work list kernel's (pieces add up to one
      // entry per partial-result slot)
      a.n_work = n_entries + SPLIT_SLOTS;
      a.nwork_dev = w.cnt + 2;
      a.part = w.part;
      a.split_keys = ctx->split_keys;
    }
    a.qrows = M;
    a.kp = w.kp;
    a.vp = w.vp;
    a.n = np;
    a.kv_dtype = kv->kv_dtype;
    a.nb = ctx->attn_nb;
    RC(attention(ctx, a, nullptr, 0, s));
    if (w.cnt) {
      // split-KV: the pieces' partial rows into the output rows
      Launch L(ctx, s, ST_PROF_ATTN, 0, 0);
      split_merge(w.mlist, w.cnt, w.part, w.prow, w.pP, G, c.hq, c.hkv, (__half*)w.o, s);
      CKLAUNCH();
    }
    if (qscore) {
      // query-specific scores: this layer's prompt attention mass on the document slots
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      const size_t kl = (size_t)l * c.hkv * kv->R * c.hd;
      float* sl = qscore + (size_t)l * c.hkv * kv->R;
      if (c.dtype == ST_BF16)
        query_mass<bf16>((const bf16*)w.q, (const bf16*)w.kp, (const bf16*)kv->K + kl, kv->R, kv->off, w.tup,
                         w.prow, os.op[0].P, np, c.hq, c.hkv, c.hd, a.scale, sl, s);
      else
        query_mass<float>((const float*)w.q, (const float*)w.kp, (const float*)kv->K + kl, kv->R, kv->off,
                          w.tup, w.prow, os.op[0].P, np, c.hq, c.hkv, c.hd, a.scale, sl, s);
      CKLAUNCH();
    }
    if (l + 1 < c.layers) {
      EpiParams eo;
      eo.mode = EPI_RESID;
      eo.x = w.x;
      eo.ld = c.d;
      if (fused) set_norm_out(eo, w.xn, w.ssq);
      RC(project(ctx, w.o, LW.wo, M, c.d, qd, eo, w.tmp, nullptr, s));
      if (!fused) {
        Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
        rmsnorm_rows<float>(w.x, M, c.d, c.eps, (float*)w.xn, nullptr, s);
        CKLAUNCH();
      }
      EpiParams eg;
      eg.mode = EPI_SWIGLU;
      eg.h = w.h;
      eg.ld = c.ffn;
      if (fused) set_norm_in(eg, w.ssq, c);
      RC(project(ctx, w.xn, LW.wgu, M, 2 * c.ffn, c.d, eg, w.tmp, w.h, s));
      EpiParams ed;
      ed.mode = EPI_RESID;
      ed.x = w.x;
      ed.ld = c.d;
      if (fused) set_norm_out(ed, w.xn, w.ssq);
      RC(project(ctx, w.h, LW.wd, M, c.d, c.ffn, ed, w.tmp, nullptr, s));
      continue;
    }
    // Last layer: only each pair's last prompt row feeds the label head, so the
    // output projection, the FFN and their norms run on those rows only, one
    // operator segment at a time (its rows are P apart): read in place through
    // a row stride, residual rows i*P + P-1 of the segment, compact norm / FFN
    // buffers at the segment's first pair.
    for (int k = 0; k < os.n_ops; ++k) {
      const OpDev& od = os.op[k];
      const int a0 = std::max(p0, od.pair0), b0 = std::min(p1, od.pair0 + od.n);
      if (b0 <= a0) continue;
      const int P = od.P, Mr = b0 - a0, ia = a0 - p0;            // pairs, first chunk pair
      const int64_t ra = od.row0 + (int64_t)(a0 - od.pair0) * P - row_base;   // first row
      EpiParams eo;
      eo.mode = EPI_RESID;
      eo.x = w.x;
      eo.ld = c.d;
      eo.a_ld = (int64_t)P * qd;
      eo.row_mul = P;
      eo.row_add = (int)(ra + P - 1);
      if (fused) set_norm_out(eo, (char*)w.xn + (size_t)ia * c.d * ctx->esz, w.ssq + (size_t)ia * (c.d / 128));
      const void* o_in = (const char*)w.o + (size_t)(ra + P - 1) * qd * ctx->esz;
      RC(project(ctx, o_in, LW.wo, Mr, c.d, qd, eo, w.tmp, nullptr, s));
      void* xn_k = (char*)w.xn + (size_t)ia * c.d * ctx->esz;
      if (!fused) {
        Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
        rmsnorm_rows<float>(w.x + (size_t)(ra + P - 1) * c.d, Mr, c.d, c.eps, (float*)xn_k, nullptr, s,
                            (int64_t)P * c.d);
        CKLAUNCH();
      }
      void* h_k = (char*)w.h + (size_t)ia * c.ffn * ctx->esz;
      EpiParams eg;
      eg.mode = EPI_SWIGLU;
      eg.h = h_k;
      eg.ld = c.ffn;
      if (fused) set_norm_in(eg, w.ssq + (size_t)ia * (c.d / 128), c);
      RC(project(ctx, xn_k, LW.wgu, Mr, 2 * c.ffn, c.d, eg, w.tmp, h_k, s));
      EpiParams ed;
      ed.mode = EPI_RESID;
      ed.x = w.x;
      ed.ld = c.d;
      ed.row_mul = P;
      ed.row_add = (int)(ra + P - 1);
      RC(project(ctx, h_k, LW.wd, Mr, c.d, c.ffn, ed, w.tmp, nullptr, s));
    }
  }
  if (mp) {
    // map operator: the first greedy token from the last prompt row's logits
    // over the whole vocabulary (one operator: pair i's last row is i*P + P-1)
    const int P = os.op[0].P;
    {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      if (c.dtype == ST_BF16)
        rmsnorm_rows<__half>(w.x + (size_t)(P - 1) * c.d, np, c.d, c.eps, (__half*)mp->xn, nullptr, s,
                             (int64_t)P * c.d);
      else
        rmsnorm_rows<float>(w.x + (size_t)(P - 1) * c.d, np, c.d, c.eps, (float*)mp->xn, nullptr, s, (int64_t)P * c.d);
      CKLAUNCH();
    }
    RC(map_head(ctx, np, 0, w, *mp, s));
    return ST_OK;
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    label_head(w.x, os, np, w.prow, w.pP, w.pop, w.pj, c.d, c.eps, ctx->w_lm, c.dtype, M, ctx->dstatus, s);
  }
  CKLAUNCH();
  return ST_OK;
}

// Greedy token t of every pair: logits of the final-normed rows mp.xn over the
// whole vocabulary (one GEMM against the LM head) and their argmax.
int map_head(st_ctx* ctx, int np, int t, const EvalBufs& w, const MapCtx& mp, cudaStream_t s) {
  const st_model_cfg& c = ctx->cfg;
  EpiParams el;
  el.mode = EPI_STORE_F32;
  el.out = mp.logits;
  el.ld = c.vocab;
  RC(project(ctx, mp.xn, ctx->w_lm, np, c.vocab, c.d, el, w.tmp, nullptr, s));
  Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
  argmax_rows(mp.logits, np, c.vocab, t, mp.n_gen, mp.tokens, mp.logits_out, ctx->dstatus, s);
  CKLAUNCH();
  return ST_OK;
}

// Decode step t >= 1 of the map operator: one row per pair (the token of step
// t - 1 at position L + P + t - 1) through every layer, its keys and values
// appended to the decode cache, attending to the retained slots and to the
// pair's P + t prompt / generated keys; then the greedy token t.
int decode_step(st_ctx* ctx, const st_kv* kv, int P, int np, int t, const EvalBufs& w, const MapCtx& mp,
                cudaStream_t s) {
  const st_model_cfg& c = ctx->cfg;
  const int qd = c.hq * c.hd, kd = c.hkv * c.hd, nqkv = qd + 2 * kd;
  const size_t kr_e = kv->kv_dtype == ST_E4M3 ? 1 : ctx->esz;
  const bool fused = c.dtype == ST_BF16;
  const int M = np;
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    decode_plan(np, mp.S, P, t, mp.n_gen, w.len, mp.tokens, w.prow, w.pP, mp.pq0, w.rowpair, w.pos, w.tok, s);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    if (c.dtype == ST_BF16) embed_rows<bf16>(w.tok, M, (const bf16*)ctx->embed, c.d, c.vocab, w.x, ctx->dstatus, s);
    else embed_rows<float>(w.tok, M, (const float*)ctx->embed, c.d, c.vocab, w.x, ctx->dstatus, s);
  }
  CKLAUNCH();
  for (int l = 0; l < c.layers; ++l) {
    const LayerW& LW = ctx->layers[l];
    char* Kl = (char*)mp.K + (size_t)l * mp.layer_elems * ctx->esz;
    char* Vl = (char*)mp.V + (size_t)l * mp.layer_elems * ctx->esz;
    if (!fused || l == 0) RC(rmsnorm(ctx, w.x, M, w.xn, nullptr, s));
    EpiParams ep;
    if (fused && l > 0) set_norm_in(ep, w.ssq, c);
    ep.mode = EPI_QKV;
    ep.q = w.q;
    ep.kbase = Kl + (size_t)(P + t - 1) * kd * ctx->esz;
    ep.vbase = Vl + (size_t)(P + t - 1) * kd * ctx->esz;
    ep.kv_sg = c.hd;
    ep.kv_sr = (int64_t)mp.S * kd;
    ep.pos = w.pos;
    ep.rope = ctx->rope;
    ep.rope_t = ctx->rope_t;
    ep.rope_np = c.max_pos;
    ep.hq = c.hq;
    ep.hkv = c.hkv;
    ep.hd = c.hd;
    ep.qkv_f16 = kv->kv_dtype == ST_E4M3 ? 1 : 0;
    RC(project(ctx, w.xn, LW.wqkv, M, nqkv, c.d, ep, w.tmp, nullptr, s));
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
    a.prow = w.prow;
    a.pP = w.pP;
    a.rowpair = w.rowpair;
    a.work = mp.work;
    a.n_work = np;
    a.qrows = np;
    a.kvrows = (int64_t)np * mp.S;
    a.nq = 1;
    a.pq0 = mp.pq0;
    a.kp = Kl;
    a.vp = Vl;
    a.n = np;
    a.kv_dtype = kv->kv_dtype;
    a.nb = ctx->attn_nb;
    RC(attention(ctx, a, nullptr, 0, s));
    EpiParams eo;
    eo.mode = EPI_RESID;
    eo.x = w.x;
    eo.ld = c.d;
    if (fused) set_norm_out(eo, w.xn, w.ssq);
    RC(project(ctx, w.o, LW.wo, M, c.d, qd, eo, w.tmp, nullptr, s));
    if (!fused) {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      rmsnorm_rows<float>(w.x, M, c.d, c.eps, (float*)w.xn, nullptr, s);
      CKLAUNCH();
    }
    EpiParams eg;
    eg.mode = EPI_SWIGLU;
    eg.h = w.h;
    eg.ld = c.ffn;
    if (fused) set_norm_in(eg, w.ssq, c);
    RC(project(ctx, w.xn, LW.wgu, M, 2 * c.ffn, c.d, eg, w.tmp, w.h, s));
    EpiParams ed;
    ed.mode = EPI_RESID;
    ed.x = w.x;
    ed.ld = c.d;
    if (fused && l + 1 < c.layers) set_norm_out(ed, w.xn, w.ssq);
    RC(project(ctx, w.h, LW.wd, M, c.d, c.ffn, ed, w.tmp, nullptr, s));
  }
  RC(rmsnorm(ctx, w.x, M, mp.xn, nullptr, s));
  return map_head(ctx, np, t, w, mp, s);
}

// Chunks the pairs (operator-major) into batches of at most `cap` prompt rows
// and runs each through eval_chunk.
int run_opset(st_ctx* ctx, const st_kv* kv, const OpSet& os, int pairs, cudaStream_t s, DevBuf* ws,
              float* qscore) {
  const st_model_cfg& c = ctx->cfg;
  int maxP = 1;
  for (int k = 0; k < os.n_ops; ++k) maxP = std::max(maxP, os.op[k].P);
  const int64_t cap = std::max<int64_t>(ctx->eval_rows_cap > 0 ? ctx->eval_rows_cap : kDefaultEvalRows, maxP);
  // chunk boundaries
  std::vector<int> cuts{0};
  int64_t acc = 0;
  for (int k = 0; k < os.n_ops; ++k)
    for (int j = 0; j < os.op[k].n; ++j) {
      if (acc + os.op[k].P > cap) {
        cuts.push_back(os.op[k].pair0 + j);
        acc = 0;
      }
      acc += os.op[k].P;
    }
  cuts.push_back(pairs);
  int64_t max_rows = 0;
  int max_pairs = 0;
  for (size_t q = 0; q + 1 < cuts.size(); ++q) {
    max_rows = std::max(max_rows, opset_rows(os, cuts[q], cuts[q + 1]));
    max_pairs = std::max(max_pairs, cuts[q + 1] - cuts[q]);
  }
  DevBuf& buf = ws ? *ws : ctx->ws_eval;
  RC(grow(ctx, buf, eval_bufs(ctx, max_rows, max_pairs, nullptr, nullptr)));
  EvalBufs w;
  eval_bufs(ctx, max_rows, max_pairs, (char*)buf.p, &w);
  int64_t row_base = 0;
  for (size_t q = 0; q + 1 < cuts.size(); ++q) {
    const int64_t M = opset_rows(os, cuts[q], cuts[q + 1]);
    if (M == 0) continue;
    RC(eval_chunk(ctx, kv, os, cuts[q], cuts[q + 1], row_base, M, w, s, nullptr, qscore));
    row_base += M;
  }
  (void)c;
  return ST_OK;
}

}  // namespace st

extern "C" int st_op_eval(st_ctx* ctx, const st_kv* kv, const st_operator* op,
                          const int32_t* tuple_ids_dev, int32_t n, float* logits_dev,
                          int32_t* labels_dev, void* stream) {
  ST_TRACE("st_op_eval");
  if (!ctx || !kv || !op || kv->ctx != ctx || n < 0) return fail(ctx, ST_EINVAL, "st_op_eval: bad argument");
  if (n == 0) return ST_OK;
  if (!tuple_ids_dev || !logits_dev || !labels_dev) return fail(ctx, ST_EINVAL, "st_op_eval: NULL buffer");
  OpSet os;
  int64_t rows = 0;
  int pairs = 0;
  RC(make_opset(ctx, kv, 1, &op, &tuple_ids_dev, &n, &logits_dev, &labels_dev, &os, &rows, &pairs));
  return run_opset(ctx, kv, os, pairs, S(stream), nullptr);
}

extern "C" int st_op_eval_multi(st_ctx* ctx, const st_kv* kv, int32_t n_ops,
                                const st_operator* const* ops, const int32_t* const* tuple_ids_dev,
                                const int32_t* n, float* const* logits_dev, int32_t* const* labels_dev,
                                void* stream) {
  ST_TRACE("st_op_eval_multi");
  if (!ctx) return fail(nullptr, ST_EINVAL, "st_op_eval_multi: NULL context");
  OpSet os;
  int64_t rows = 0;
  int pairs = 0;
  RC(make_opset(ctx, kv, n_ops, ops, tuple_ids_dev, n, logits_dev, labels_dev, &os, &rows, &pairs));
  if (pairs == 0) return ST_OK;
  return run_opset(ctx, kv, os, pairs, S(stream), nullptr);
}

extern "C" int st_map_eval(st_ctx* ctx, const st_kv* kv, const st_operator* op,
                           const int32_t* tuple_ids_dev, int32_t n, int32_t n_gen, int32_t* tokens_dev,
                           float* logits_dev, void* stream) {
  ST_TRACE("st_map_eval");
  if (!ctx || !kv || !op || kv->ctx != ctx || n < 0) return fail(ctx, ST_EINVAL, "st_map_eval: bad argument");
  if (n_gen < 1 || n_gen > 256) return fail(ctx, ST_EINVAL, "st_map_eval: n_gen must lie in 1..256");
  if (n == 0) return ST_OK;
  if (!tuple_ids_dev || !tokens_dev) return fail(ctx, ST_EINVAL, "st_map_eval: NULL buffer");
  const st_model_cfg& c = ctx->cfg;
  const int P = op->desc.P;
  if (kv->max_len + P + n_gen > c.max_pos)
    return fail(ctx, ST_EINVAL, "st_map_eval: document + prompt + generated tokens exceed max_pos");
  if ((c.dtype == ST_BF16 && c.vocab % 256) || (c.dtype == ST_F32 && c.vocab % 128))
    return fail(ctx, ST_EUNSUPPORTED, "st_map_eval: the vocabulary must be a multiple of 256 (bf16) / 128 (f32)");
  OpSet os;
  int64_t rows = 0;
  int pairs = 0;
  float* dummy_l = reinterpret_cast<float*>(tokens_dev);   // no label head in the map operator
  RC(make_opset(ctx, kv, 1, &op, &tuple_ids_dev, &n, &dummy_l, &tokens_dev, &os, &rows, &pairs));
  cudaStream_t s = S(stream);
  const int64_t cap = std::max<int64_t>(ctx->eval_rows_cap > 0 ? ctx->eval_rows_cap : kDefaultEvalRows, P);
  const int per = (int)std::max<int64_t>(1, std::min<int64_t>(n, cap / P));
  const int kd = c.hkv * c.hd, G = c.hq / c.hkv, S = P + n_gen;
  RC(grow(ctx, ctx->ws_eval, eval_bufs(ctx, (int64_t)per * P, per, nullptr, nullptr)));
  EvalBufs w;
  eval_bufs(ctx, (int64_t)per * P, per, (char*)ctx->ws_eval.p, &w);
  // decode cache, per-pair arrays, logits and final-normed rows of one chunk
  const int64_t layer_elems = (int64_t)per * S * kd;
  auto layout = [&](char* base, MapCtx* m) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
      off = (off + 255) & ~(size_t)255;
      char* p = base + off;
      off += bytes;
      return (void*)p;
    };
    m->K = take((size_t)c.layers * layer_elems * ctx->esz);
    m->V = take((size_t)c.layers * layer_elems * ctx->esz);
    m->pq0 = (int32_t*)take((size_t)per * 4);
    m->work = (int32_t*)take((size_t)per * WORK_INTS * 4);
    m->logits = (float*)take((size_t)per * c.vocab * 4);
    m->xn = take((size_t)per * c.d * ctx->esz);
    return off + 256;
  };
  MapCtx mp;
  RC(grow(ctx, ctx->ws_map, layout(nullptr, &mp)));
  layout((char*)ctx->ws_map.p, &mp);
  mp.n_gen = n_gen;
  mp.S = S;
  mp.layer_elems = layer_elems;
  for (int i0 = 0; i0 < n; i0 += per) {
    const int nc = std::min(per, n - i0);
    mp.tokens = tokens_dev + (size_t)i0 * n_gen;
    mp.logits_out = logits_dev ? logits_dev + (size_t)i0 * n_gen * c.vocab : nullptr;
    RC(eval_chunk(ctx, kv, os, i0, i0 + nc, (int64_t)i0 * P, (int64_t)nc * P, w, s, &mp));
    if (c.dtype == ST_BF16) {
      Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
      eval_worklist(w.nk, w.pP, w.tup, w.prow, kv->offp, nc, G, 1, ctx->longest_first != 0, mp.work, 0, nullptr,
                    nullptr, nullptr, s);
    }
    for (int t = 1; t < n_gen; ++t) RC(decode_step(ctx, kv, P, nc, t, w, mp, s));
  }
  return ST_OK;
}

extern "C" int st_set_gemm_pairs(int32_t on) {
  set_gemm_pairs(on != 0);
  return ST_OK;
}

extern "C" int st_set_scoring(st_ctx* ctx, int32_t mode, int32_t horizon) {
  ST_TRACE("st_set_scoring");
  if (!ctx) return fail(nullptr, ST_EINVAL, "st_set_scoring: NULL context");
  const st_model_cfg& c = ctx->cfg;
  if (mode == ST_SCORE_EA_LITE) {
    ctx->score_mode = mode;
    return ST_OK;
  }
  if (mode != ST_SCORE_EA_FULL || horizon < 1 || horizon > 4096 || horizon >= c.max_pos)
    return fail(ctx, ST_EINVAL, "st_set_scoring: mode or horizon out of range");
  // averaged rotation of every document length L <= max_pos - F, in double:
  // (1/F) sum over p = L .. L+F-1 of (cos, sin)(p theta^(-2i/hd))
  const int half = c.hd / 2;
  std::vector<float2> tab((size_t)c.max_pos * half, make_float2(0.f, 0.f));
  for (int i = 0; i < half; ++i) {
    const double w = std::pow((double)c.rope_theta, -2.0 * i / c.hd);
    for (int L = 0; L + horizon <= c.max_pos; ++L) {
      double cs = 0.0, sn = 0.0;
      for (int p = L; p < L + horizon; ++p) {
        cs += std::cos((double)p * w);
        sn += std::sin((double)p * w);
      }
      tab[(size_t)L * half + i] = make_float2((float)(cs / horizon), (float)(sn / horizon));
    }
  }
  if (!ctx->rope_avg) RC(dev_alloc(ctx, (void**)&ctx->rope_avg, tab.size() * sizeof(float2)));
  CK(cudaMemcpy(ctx->rope_avg, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice));
  ctx->score_mode = mode;
  ctx->score_horizon = horizon;
  return ST_OK;
}

extern "C" int st_kv_score_query(st_ctx* ctx, st_kv* kv, const st_operator* op, void* stream) {
  ST_TRACE("st_kv_score_query");
  if (!ctx || !kv || !op || kv->ctx != ctx) return fail(ctx, ST_EINVAL, "st_kv_score_query: bad argument");
  if (kv->src) return fail(ctx, ST_EINVAL, "st_kv_score_query: scores belong to the source cache, not to a profile");
  const st_model_cfg& c = ctx->cfg;
  if (!kv->built || kv->r != 1.0 || kv->kv_dtype != c.dtype)
    return fail(ctx, ST_EINVAL, "st_kv_score_query: the cache needs a retained profile at r = 1 in the model dtype");
  if (!ea_full_supported(c.hd)) return fail(ctx, ST_EUNSUPPORTED, "st_kv_score_query: hd must be 32 or 64");
  const int T = kv->T, nl = op->desc.n_labels;
  if (T == 0) return ST_OK;
  const size_t need = (size_t)T * 4 + 256 + (size_t)T * nl * 4 + 256 + (size_t)T * 4 + 256;
  RC(grow(ctx, ctx->ws_score, need));
  Carve cv(ctx->ws_score.p);
  int32_t* ids = cv.take<int32_t>(T);
  float* logits = cv.take<float>((int64_t)T * nl);
  int32_t* labels = cv.take<int32_t>(T);
  cudaStream_t s = S(stream);
  std::vector<int32_t> h(T);
  for (int t = 0; t < T; ++t) h[t] = t;
  CK(cudaMemcpyAsync(ids, h.data(), (size_t)T * 4, cudaMemcpyHostToDevice, s));
  OpSet os;
  int64_t rows = 0;
  int pairs = 0, n = T;
  const int32_t* idp = ids;
  RC(make_opset(ctx, kv, 1, &op, &idp, &n, &logits, &labels, &os, &rows, &pairs));
  os.op[0].r = 1.0;   // the prompt attends to every document slot, whatever the operator's own r
  RC(run_opset(ctx, kv, os, pairs, s, nullptr, kv->scores));
  CK(cudaStreamSynchronize(s));   // the host id buffer
  return ST_OK;
}

extern "C" int st_run_host(st_ctx* ctx, st_kv* kv, const st_operator* op, int32_t kv_dtype,
                           const int32_t* tokens_host, float* logits_host, int32_t* labels_host,
                           void* stream) {
  ST_TRACE("st_run_host");
  if (!ctx || !kv || !op || !tokens_host || !logits_host || !labels_host)
    return fail(ctx, ST_EINVAL, "st_run_host: bad argument");
  cudaStream_t s = S(stream);
  const int T = kv->T, nl = op->desc.n_labels;
  if (!kv->tok) {
    RC(dev_alloc(ctx, (void**)&kv->tok, (size_t)kv->R * 4));
    RC(dev_alloc(ctx, (void**)&kv->iota, (size_t)T * 4));
    std::vector<int32_t> ids(T);
    for (int t = 0; t < T; ++t) ids[t] = t;
    CK(cudaMemcpy(kv->iota, ids.data(), (size_t)T * 4, cudaMemcpyHostToDevice));
    RC(dev_alloc(ctx, (void**)&kv->out_logits, (size_t)T * 8 * 4));
    RC(dev_alloc(ctx, (void**)&kv->out_labels, (size_t)T * 4));
  }
  CK(cudaMemcpyAsync(kv->tok, tokens_host, (size_t)kv->R * 4, cudaMemcpyHostToDevice, s));
  RC(st_kv_build(ctx, kv, kv->tok, stream));
  RC(st_kv_retain(ctx, kv, op->desc.r, kv_dtype, stream));
  RC(st_op_eval(ctx, kv, op, kv->iota, T, kv->out_logits, kv->out_labels, stream));
  CK(cudaMemcpyAsync(logits_host, kv->out_logits, (size_t)T * nl * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(labels_host, kv->out_labels, (size_t)T * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return ST_OK;
}

// ================================================================== profiling
extern "C" int st_prof_enable(st_ctx* ctx, int32_t on) {
  if (!ctx) return fail(nullptr, ST_EINVAL, "st_prof_enable: NULL context");
  ctx->prof.on = on != 0;
  return ST_OK;
}

extern "C" int st_prof_read(st_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(ctx, ST_EINVAL, "st_prof_read: bad argument");
  for (auto& r : ctx->prof.pending) {
    CK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    double* a = ctx->prof.acc[r.family];
    a[0] += 1;
    a[1] += ms;
    a[2] += r.flops;
    a[3] += r.bytes;
    ctx->prof.pool.push_back(r.a);
    ctx->prof.pool.push_back(r.b);
  }
  ctx->prof.pending.clear();
  std::memcpy(out, ctx->prof.acc, sizeof(ctx->prof.acc));
  return ST_OK;
}

extern "C" int st_prof_reset(st_ctx* ctx) {
  if (!ctx) return fail(nullptr, ST_EINVAL, "st_prof_reset: NULL context");
  double tmp[ST_PROF_N * 4];
  st_prof_read(ctx, tmp);
  std::memset(ctx->prof.acc, 0, sizeof(ctx->prof.acc));
  ctx->launches = 0;
  return ST_OK;
}

extern "C" int64_t st_launch_count(const st_ctx* ctx) { return ctx ? ctx->launches : 0; }
