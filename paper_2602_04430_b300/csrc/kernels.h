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
  int act_f16 = 0;                // EPI_RESID xb and EPI_SWIGLU h as IEEE half (the next GEMM's operand type)
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
  bool timed;          // profiling events recorded for this launch
  ProfRec rec;
  Launch(st_ctx* c, cudaStream_t st, int fam, double fl, double by);
  ~Launch();
};
// Set by an entry that must create no CUDA resources (st_op_eval_noalloc) for
// the duration of its call, on its own host thread only: Launch records no
// profiling events while it is set.  Thread-local, so another thread's calls
// on the same context keep their profiling.
extern thread_local bool tls_no_prof;

// ---- batched operator evaluation: the operators of one call as the kernels see
// them (passed by value in kernel parameters, so a captured graph replays them)
constexpr int ST_MAX_OPS = 8;
struct OpDev {
  const int32_t* tuple_ids = nullptr;   // [n] device: the tuples this operator evaluates
  const int32_t* prompt = nullptr;      // [P] device
  const int32_t* labels = nullptr;      // [n_labels] device: label token ids
  const float* bias = nullptr;          // [n_labels] device (classify)
  float* logits = nullptr;              // [n][n_labels] device output
  int32_t* out_labels = nullptr;        // [n] device output
  int64_t row0 = 0;                     // first prompt row of this operator in the call
  double r = 1.0;
  int n = 0, P = 0, n_labels = 0, kind = 0, pair0 = 0;   // pair0: first (operator, tuple) pair
  float theta_pos = 0.f, theta_neg = 0.f;
};
struct OpSet {
  int n_ops = 0;
  int T = 0;                            // tuples of the cache: valid ids are [0, T)
  OpDev op[ST_MAX_OPS];
};

// ---- misc kernels (kernels_misc.cu) ----
template <typename act_t>
void embed_rows(const int32_t* tok, int64_t rows, const act_t* E, int d, int vocab, float* x, int* status,
                cudaStream_t s);
// BF16 model: the gather fused with the first layer's RMSNorm (xn in half).
// st_kv_indices: the first n_t entries of every rank-ordered segment, compacted
// at out_off (int64 [T+1]) into idx [layers * hkv][out_off[T]].
void gather_indices(const int32_t* rank, const int64_t* doc_off, const int64_t* out_off, int T, int LH,
                    int64_t R, int64_t Rn, int32_t* idx, int* status, cudaStream_t s);
void embed_norm_rows(const int32_t* tok, int64_t rows, const bf16* E, int d, int vocab, float eps, float* x,
                     __half* xn, int* status, cudaStream_t s);
template <typename act_t>
void rmsnorm_rows(const float* x, int64_t rows, int d, float eps, act_t* xn, float* inv_rms,
                  cudaStream_t s, int64_t x_ld = 0);
void build_rowinfo(const int64_t* off, int t0, int t1, int64_t r0, int64_t rows, int32_t* rowtup,
                   int32_t* pos, cudaStream_t s);
// Plan of pairs [p0, p0 + np) of an operator set whose rows start at row_base:
// per pair (eval_pairs) its tuple, document length, retained count, prompt row
// (relative to row_base), prompt length, operator and index within the
// operator; per row (eval_rows) its RoPE position, prompt token and pair.
// A tuple id outside [0, os.T) is replaced by 0 and ST_ERANGE is recorded in
// *status (first error wins).
void eval_pairs(const OpSet& os, int p0, int np, int64_t row_base, const int64_t* off, int32_t* tup,
                int32_t* len, int32_t* nk, int32_t* prow, int32_t* pP, int32_t* pop, int32_t* pj,
                int* status, cudaStream_t s);
void eval_rows(const OpSet& os, int p0, int64_t row_base, int64_t rows, const int64_t* off,
               int32_t* pos, int32_t* tok, int32_t* rowpair, int* status, cudaStream_t s);
// Attention work list: (pair, 128-row block) entries, longest retained
// documents first; G = query heads per kv head.
// nq: query positions per pair (0: its prompt length).
// Each entry is a fully decoded item record of WORK_INTS int32 (32 bytes, one
// pair of 16-byte loads in the attention kernel): pair, row block | piece << 8
// | pieces << 16, prompt length, retained slots, first prompt row, the piece's
// partial-result slot (-1: not split), and the tuple's padded retained offset
// offp[tup] as an int64 in two words.  split_keys > 0 (with nq = 0): a pair
// whose retained slots exceed it is cut into pieces of split_keys slots (at
// most 255), while SPLIT_SLOTS partial-result slots last; cnt[0] counts the
// slots taken, cnt[1] the merge list's entries (pair, row block, first slot,
// pieces), cnt[2] the list's entries; psplit[pair] is the pair's first slot or -1.
constexpr int WORK_INTS = 8;
void eval_worklist(const int32_t* nk, const int32_t* pP, const int32_t* tup, const int32_t* prow,
                   const int64_t* offp, int np, int G, int nq, bool longest_first, int32_t* list,
                   int split_keys, int32_t* psplit, int32_t* mlist, int32_t* cnt, cudaStream_t s);
// Split-KV merge: for every (split pair, row block) of the merge list and kv
// head, the output rows from the pieces' partial results (f16, O's layout).
void split_merge(const int32_t* mlist, const int32_t* cnt, const float* part, const int32_t* prow,
                 const int32_t* pP, int G, int hq, int hkv, __half* o, cudaStream_t s);
template <typename act_t>
void qstats(const act_t* q, const int64_t* off, int t0, int t1, int64_t r0, int hq, int hkv,
            int hd, float* mu, float* s2, cudaStream_t s);
template <typename act_t>
void ea_scores(const act_t* K, const act_t* V, int64_t R, int hkv, int hd, int64_t r0,
               int64_t rows, const int32_t* rowtup, int t0, const float* mu, const float* s2,
               float* scores, cudaStream_t s);
// Scoring ablation (scoring.cu).  Full Expected Attention scores of the chunk's
// tuples [t0, t1) at one layer (hd 32 or 64): query moments into m_ws
// [tuples][hkv][hd] and M_ws [tuples][hkv][hd][hd], then every slot's score.
bool ea_full_supported(int hd);
template <typename act_t>
void ea_full_scores(const act_t* q, const act_t* K, const act_t* V, int64_t R, const int64_t* off, int t0,
                    int t1, int64_t r0, int hq, int hkv, int hd, const float2* rope, const float2* ravg,
                    float* m_ws, float* M_ws, float* scores, cudaStream_t s);
// Query-specific scores of one layer: for each of the np pairs (tuple tup[i],
// prompt rows prow[i] .. + P of q / kp), the attention probability its prompt
// queries put on every document slot, written to scores[g][off[t] + j].
template <typename act_t>
void query_mass(const act_t* q, const act_t* kp, const act_t* K, int64_t R, const int64_t* off,
                const int32_t* tup, const int32_t* prow, int P, int np, int hq, int hkv, int hd, float scale,
                float* scores, cudaStream_t s);
// pooled[t] = mean of x[m] / rms(x[m]) over tuple t's rows; 1/rms from inv_rms or,
// when inv_rms is nullptr, from the partial sums of squares ssq[m][parts]
void pool_rows(const float* x, const float* inv_rms, const float* ssq, int parts, float eps,
               const int64_t* off, int t0, int t1, int64_t r0, int d, float* pooled, cudaStream_t s);
// Map operator (greedy decode): prompt K/V of one layer into the decode cache
// [pair][S][kd]; the plan of decode step t; the greedy token of each row.
void copy_prompt_kv(const void* src, void* dst, int n, int P, int S, int kd, size_t esz, cudaStream_t s);
void decode_plan(int n, int S, int P, int t, int n_gen, const int32_t* len, const int32_t* tokens,
                 int32_t* prow, int32_t* pP, int32_t* pq0, int32_t* rowpair, int32_t* pos, int32_t* tok,
                 cudaStream_t s);
void argmax_rows(const float* logits, int n, int V, int t, int n_gen, int32_t* tokens, float* logits_out,
                 int* status, cudaStream_t s);
// In-place conversion of n bfloat16 values to IEEE half (round to nearest).
void bf16_to_f16(void* p, size_t n, cudaStream_t s);
// Final RMSNorm of each pair's last prompt row, its operator's label logits and decision.
void label_head(const float* x, const OpSet& os, int np, const int32_t* prow, const int32_t* pP,
                const int32_t* pop, const int32_t* pj, int d, float eps, const void* w_lm, int dtype,
                int64_t rows, int* status, cudaStream_t s);
void swiglu_from_f32(const float* t, int64_t rows, int ffn, float* h, cudaStream_t s);
void nkeep_offp(const int64_t* off, int T, double r, int32_t* nkeep, int64_t* offp,
                cudaStream_t s);

// ---- GEMMs ----
template <typename act_t>
void gemm_simt(const act_t* A, const act_t* W, int M, int N, int K, const EpiParams& ep,
               cudaStream_t s);
bool gemm_tc_supported(int M, int N, int K);
// Process-wide choice of the tcgen05 GEMM for M > 128: CTA pairs (2-SM MMA,
// the default) or single CTAs.
void set_gemm_pairs(bool on);
// f16: A and W are IEEE half (the model path, whose BF16 weights are held
// exactly as f16); otherwise bfloat16 (st_gemm).
int gemm_tc(const void* A, const void* W, int M, int N, int K, const EpiParams& ep, int* status,
            cudaStream_t s, bool f16);

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
  const int32_t* prow = nullptr;  // [n] first prompt row of each pair
  const int32_t* pP = nullptr;    // [n] prompt length of each pair
  const int32_t* rowpair = nullptr; // [qrows] pair of each prompt row (CUDA-core path)
  const int32_t* work = nullptr;  // tensor-core path: (pair, 128-row block) entries
  float* part = nullptr;          // split-KV partial results [slot][hkv][128 rows][SPLIT_STRIDE]
  const int32_t* nwork_dev = nullptr;  // split-KV: the list's entry count on the device (n_work: a bound)
  int split_keys = 0;             // split-KV piece length (0: no item is split)
  int n_work = 0;                 // entries in work
  int64_t qrows = 0;              // prompt rows of the call
  int nb = 0;                     // BF16-KV attention layout: 0 / 1 = two CTAs per SM, 2 = one
  // Decode steps: a pair's queries are its last nq prompt positions (0 = all
  // pP), their Q rows start at pq0[i] (nullptr: prow[i]); the prompt K/V
  // tensors have kvrows rows (0: qrows).
  int nq = 0;
  const int32_t* pq0 = nullptr;
  int64_t kvrows = 0;
  const void* kp = nullptr;       // prompt keys kp[(i*P + p)*hkv*hd + g*hd + c]
  const void* vp = nullptr;
  int n = 0, P = 0;
  int kv_dtype = ST_F32;
};
template <typename act_t, typename kv_t>
void attn_simt(const AttnParams& a, cudaStream_t s);
bool attn_tc_supported(int hq, int hkv, int hd);
int attn_tc_eval(const AttnParams& a, int* status, cudaStream_t s);
int attn_tc_prefill(const AttnParams& a, const int32_t* items, int n_items, int* status,
                    cudaStream_t s);

// ---- host sequencing helpers (api.cu): one projection / RMSNorm / attention step
// f16_ops: the BF16 model's operands (IEEE half activations and weights, the
// residual / SwiGLU epilogues writing half); false: caller-given bfloat16 (st_gemm).
int project(st_ctx* ctx, const void* A, const void* W, int M, int N, int K, EpiParams ep, float* tmp,
            void* h_out, cudaStream_t s, bool f16_ops = true);
int rmsnorm(st_ctx* ctx, const float* x, int64_t rows, void* xn, float* inv, cudaStream_t s);
int attention(st_ctx* ctx, const AttnParams& a, const int32_t* items, int n_items, cudaStream_t s);
// The projection reads bf16(x) and scales its rows by 1/rms from `ssq`.
void set_norm_in(EpiParams& ep, const float* ssq, const st_model_cfg& c);
// The residual epilogue also writes bf16(x) to xb and the partial sums of squares.
void set_norm_out(EpiParams& ep, void* xb, float* ssq);

// ---- operator evaluation sequence (api.cu), shared by st_op_eval and st_op_eval_noalloc ----
struct EvalBufs {
  float *x, *tmp, *ssq;
  void *xn, *q, *kp, *vp, *o, *h;
  int32_t *pos, *tok, *rowpair;                       // per prompt row
  int32_t *tup, *len, *nk, *prow, *pP, *pop, *pj;     // per (operator, tuple) pair
  int32_t* order;                                     // attention work list
  // split-KV (with ctx->split_keys > 0): each split (pair, row block)'s first
  // slot, the partial results, the merge list and two counters
  int32_t *psplit, *mlist, *cnt;
  float* part;
};
// Split-KV: partial-result slots per evaluation chunk, floats per row of a slot
// (64 unnormalised output values, the running max, the row sum, padding).
constexpr int SPLIT_SLOTS = 512, SPLIT_STRIDE = 68;
// Lays the buffers for `rows` prompt rows of `pairs` (operator, tuple) pairs out
// from `base` (nullptr: layout only); returns the bytes needed.
size_t eval_bufs(const st_ctx* ctx, int64_t rows, int64_t pairs, char* base, EvalBufs* w);
// Validates the operators of one call and lays them out as an OpSet (operator
// k's pairs follow operator k-1's, its prompt rows likewise).
int make_opset(st_ctx* ctx, const st_kv* kv, int n_ops, const st_operator* const* ops,
               const int32_t* const* tuple_ids, const int32_t* n, float* const* logits,
               int32_t* const* labels, OpSet* os, int64_t* rows_total, int* pairs_total);
// Pairs [p0, p1) of an operator set (their prompt rows start at row_base, `rows`
// of them) through every layer and the label head.
// Greedy decode of one chunk of pairs (the map operator): decode cache, per-pair
// decode arrays and scratch, all device memory.
struct MapCtx {
  int n_gen = 0, S = 0;          // tokens to generate; decode-cache rows per pair (P + n_gen)
  void* K = nullptr;             // [layers][pairs][S][kd] prompt + generated keys (model dtype / f16)
  void* V = nullptr;
  int64_t layer_elems = 0;       // elements per layer of K / V
  int32_t* pq0 = nullptr;        // [pairs]
  int32_t* work = nullptr;       // [pairs][2] attention work list (one query row per pair)
  float* logits = nullptr;       // [pairs][vocab]
  void* xn = nullptr;            // [pairs][d] final-normed rows
  int32_t* tokens = nullptr;     // [pairs][n_gen] output of the chunk
  float* logits_out = nullptr;   // optional [pairs][n_gen][vocab]
};
// mp: the map operator's prompt pass (keeps every layer's prompt K/V, ends
// with the first greedy token instead of the label head); nullptr otherwise.
// qscore: the query-specific scoring pass (one operator, r = 1 cache): every
// layer's prompt attention mass on the document slots into qscore
// [layers][hkv][R]; nullptr otherwise.
int eval_chunk(st_ctx* ctx, const st_kv* kv, const OpSet& os, int p0, int p1, int64_t row_base,
               int64_t rows, const EvalBufs& w, cudaStream_t s, const MapCtx* mp = nullptr,
               float* qscore = nullptr);
// Prompt rows of pairs [p0, p1) of an operator set.
int64_t opset_rows(const OpSet& os, int p0, int p1);
// All pairs of an operator set, in chunks of at most the context's
// eval_rows_cap prompt rows; ws: the workspace (nullptr: the context's, grown
// as needed; otherwise grown as needed too, and owned by the caller).
int run_opset(st_ctx* ctx, const st_kv* kv, const OpSet& os, int pairs, cudaStream_t s, DevBuf* ws,
              float* qscore = nullptr);

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
