// Internal launchers of libstretto (host-callable; all enqueue on `s`).
#pragma once

#include "common.cuh"

namespace st {

enum EpiMode { EPI_QKV = 0, EPI_RESID = 1, EPI_SWIGLU = 2, EPI_STORE_F32 = 3 };

// Epilogue of a projection GEMM C[M][N] = A[M][K] . W[N][K]^T.
struct EpiParams {
  int mode = EPI_STORE_F32;
  int M = 0, N = 0;
  int64_t a_ld = 0;               // row stride of A in elements (0: K)
  int qkv_f16 = 0;                // EPI_QKV: store q / k / v as IEEE half instead of the act type
  // Fused RMSNorm (tensor-core path).  EPI_RESID also writes xb[row * N + col] =
  // bf16(new stream value) and ssq_out[row * (N/128) + col/128] = the sum of the
  // squares of its 128-column slice.  EPI_QKV / EPI_SWIGLU multiply every
  // accumulator of row r by 1 / sqrt(sum_k ssq_in[r * ssq_parts + k] / norm_d + eps),
  // i.e. they project bf16(x) and apply the norm afterwards: (x / rms) W = (x W) / rms.
  void* xb = nullptr;
  float* ssq_out = nullptr;
  const float* ssq_in = nullptr;
  int ssq_parts = 0, norm_d = 0;
  float eps = 0.f;
  int64_t row_mul = 1, row_add = 0;   // EPI_RESID writes stream row (row*row_mul + row_add)
  // EPI_QKV: columns [0, hq*hd) are queries, then hkv*hd keys, then hkv*hd values.
  void* q = nullptr;              // act [M][hq*hd]
  void* kbase = nullptr;          // key of (row, kv head g, dim c) at kbase + g*kv_sg + row*kv_sr + c
  void* vbase = nullptr;
  int64_t kv_sg = 0, kv_sr = 0;
  const int32_t* pos = nullptr;   // [M] RoPE position of each row
  const float2* rope = nullptr;   // [max_pos][hd/2] (cos, sin)
  const float2* rope_t = nullptr; // the same, [hd/2][rope_np] (tcgen05 GEMM)
  int rope_np = 0;
  int hq = 0, hkv = 0, hd = 0;
  // EPI_RESID: x[row*ld + col] += acc (float32 residual stream)
  float* x = nullptr;
  // EPI_SWIGLU: h[row*ld + f] = silu(gate) * up; W rows interleaved in blocks of 128
  void* h = nullptr;
  // EPI_STORE_F32: out[row*ld + col] = acc
  float* out = nullptr;
  int64_t ld = 0;
};

// Launch record helper (profiling + launch count).
struct Launch {
  st_ctx* ctx;
  cudaStream_t s;
  int family;
  double flops, bytes;
  ProfRec rec;
  Launch(st_ctx* c, cudaStream_t st, int fam, double fl, double by);
  ~Launch();
};

// ---- misc kernels (kernels_misc.cu) ----
template <typename act_t>
void embed_rows(const int32_t* tok, int64_t rows, const act_t* E, int d, float* x, cudaStream_t s);
void embed_prompt(const int32_t* prompt, int P, int64_t rows, const void* E, int dtype, int d,
                  float* x, cudaStream_t s);
template <typename act_t>
void rmsnorm_rows(const float* x, int64_t rows, int d, float eps, act_t* xn, float* inv_rms,
                  cudaStream_t s, int64_t x_ld = 0);
void build_rowinfo(const int64_t* off, int t0, int t1, int64_t r0, int64_t rows, int32_t* rowtup,
                   int32_t* pos, cudaStream_t s);
void eval_rowinfo(const int32_t* tuple_ids, int n, int P, const int64_t* off, double r,
                  int32_t* tup, int32_t* len, int32_t* nk, int32_t* pos, cudaStream_t s);
void eval_order(const int32_t* nk, int n, int32_t* order, cudaStream_t s);
template <typename act_t>
void qstats(const act_t* q, const int64_t* off, int t0, int t1, int64_t r0, int hq, int hkv,
            int hd, float* mu, float* s2, cudaStream_t s);
template <typename act_t>
void ea_scores(const act_t* K, const act_t* V, int64_t R, int hkv, int hd, int64_t r0,
               int64_t rows, const int32_t* rowtup, int t0, const float* mu, const float* s2,
               float* scores, cudaStream_t s);
// pooled[t] = mean of x[m] / rms(x[m]) over tuple t's rows; 1/rms from inv_rms or,
// when inv_rms is nullptr, from the partial sums of squares ssq[m][parts]
void pool_rows(const float* x, const float* inv_rms, const float* ssq, int parts, float eps,
               const int64_t* off, int t0, int t1, int64_t r0, int d, float* pooled, cudaStream_t s);
void label_head(const float* x, int n, int P, int d, float eps, const void* w_lm, int dtype,
                const int32_t* labels, int n_labels, const float* bias, int kind,
                float theta_pos, float theta_neg, float* logits, int32_t* out_labels,
                cudaStream_t s);
void swiglu_from_f32(const float* t, int64_t rows, int ffn, float* h, cudaStream_t s);
void nkeep_offp(const int64_t* off, int T, double r, int32_t* nkeep, int64_t* offp,
                cudaStream_t s);

// ---- GEMMs ----
template <typename act_t>
void gemm_simt(const act_t* A, const act_t* W, int M, int N, int K, const EpiParams& ep,
               cudaStream_t s);
bool gemm_tc_supported(int M, int N, int K);
int gemm_tc(const bf16* A, const bf16* W, int M, int N, int K, const EpiParams& ep, int* status,
            cudaStream_t s);

// ---- attention ----
struct AttnParams {
  // queries: q[(qrow)*hq*hd + h*hd + c]
  const void* q = nullptr;
  void* o = nullptr;              // o[(qrow)*hq*hd + h*hd + c]
  int hq = 0, hkv = 0, hd = 0;
  float scale = 0.f;
  // prefill: keys of tuple t, kv head g at K + g*k_sg + (off[t]-... ) handled by mode
  int mode = 0;                   // 0 = prefill (causal over the document), 1 = operator eval
  // prefill
  const void* K = nullptr;        // layer base of the full cache [hkv][R][hd]
  const void* V = nullptr;
  int64_t R = 0;
  const int64_t* off = nullptr;
  const int32_t* rowtup = nullptr;
  const int32_t* pos = nullptr;
  int64_t r0 = 0;
  int64_t rows = 0;
  // eval
  const void* Kr = nullptr;       // layer base of the retained cache [hkv][Rp_cap][hd]
  const void* Vr = nullptr;
  const float* scales = nullptr;  // layer base of [hkv][Rp_cap/64][2] (E4M3 only)
  int64_t Rp_cap = 0;
  const int64_t* offp = nullptr;
  const int32_t* tup = nullptr;   // [n] tuple of each evaluated item
  const int32_t* nk = nullptr;    // [n] retained slots read per item
  const int32_t* order = nullptr; // [n] item positions, longest first (nullptr: as given)
  const void* kp = nullptr;       // prompt keys kp[(i*P + p)*hkv*hd + g*hd + c]
  const void* vp = nullptr;
  int n = 0, P = 0;
  int kv_dtype = ST_F32;
};
template <typename act_t, typename kv_t>
void attn_simt(const AttnParams& a, cudaStream_t s);
void attn_mma_eval(const AttnParams& a, cudaStream_t s);
bool attn_tc_supported(int hq, int hkv, int hd);
int attn_tc_eval(const AttnParams& a, int* status, cudaStream_t s);
int attn_tc_prefill(const AttnParams& a, const int32_t* items, int n_items, int* status,
                    cudaStream_t s);
void attn_mma_prefill(const AttnParams& a, const int32_t* items, int n_items, cudaStream_t s);

// ---- operator evaluation sequence (api.cu), shared by st_op_eval and st_op_eval_noalloc ----
struct EvalBufs {
  float *x, *tmp, *ssq;
  void *xn, *q, *kp, *vp, *o, *h;
  int32_t *pos, *tup, *len, *nk, *order;
};
// Lays the buffers for `rows` prompt rows of `tuples` tuples out from `base`
// (nullptr: layout only); returns the bytes needed.
size_t eval_bufs(const st_ctx* ctx, int64_t rows, int64_t tuples, char* base, EvalBufs* w);
// One batch of nc tuples through every layer and the label head.
int eval_chunk(st_ctx* ctx, const st_kv* kv, const st_operator* op, const int32_t* tuple_ids,
               int nc, const EvalBufs& w, float* logits, int32_t* labels, cudaStream_t s);

// ---- retention (retain.cu) ----
struct RetainParams {
  const float* scores;            // [layers][hkv][R]
  const void* K;                  // [layers][hkv][R][hd]
  const void* V;
  int32_t* rank;                  // [layers][hkv][R]
  void* Kr;                       // [layers][hkv][Rp_cap][hd]
  void* Vr;
  float* scales;                  // [layers][hkv][Rp_cap/64][2]
  const int64_t* off;
  const int64_t* offp;
  const int32_t* nkeep;
  int32_t* status;
  int T, layers, hkv, hd, max_len;
  int64_t R, Rp_cap;
  int in_dtype, out_dtype;
};
int retain(const RetainParams& p, cudaStream_t s);

}  // namespace st
