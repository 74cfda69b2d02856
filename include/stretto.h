/*
 * stretto.h -- C ABI of the B300 (sm_103a) KV-cache semantic operator library.
 *
 * The library evaluates a KV-cache-enabled semantic operator (filter or
 * classify) over a table of tuples, in the three steps of Sec. 5 of the
 * Stretto paper:
 *
 *   st_kv_build   offline KV-cache creation: every tuple's document is
 *                 prefilled once through the decoder ("Offline: KV Cache
 *                 Creation"); keys/values of every layer and kv head are kept
 *                 with a query-agnostic retention score per slot.
 *   st_kv_retain  query-agnostic compression to a retained fraction r
 *                 (compression ratio 1 - r, the profiles of Sec. 5 and Sec. 6
 *                 "Operators"): the top n_keep(L, r) slots per (layer, kv head),
 *                 in rank order, optionally stored as FP8 E4M3.
 *   st_op_eval    online execution ("Online: Query Execution"): the operator's
 *                 prompt is appended after each cached document and forwarded
 *                 in one batched pass; the logits of the label tokens are read
 *                 at the last prompt position and turned into accept / reject /
 *                 unsure with log-odds thresholds (Sec. 5; temperature-0 form
 *                 of the soft-threshold equation of Sec. 4.1), or into a class.
 *
 * Conventions for every call
 *   - Return value: ST_OK (0) or a positive ST_E* code; the message of the last
 *     failure of a context is st_last_error(ctx).  Nothing aborts the process.
 *   - "dev" pointers are CUDA device pointers owned by the caller; "host"
 *     pointers are ordinary host memory owned by the caller.  The library never
 *     frees caller memory and never keeps a caller pointer past the call,
 *     except where stated.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue work on that stream and return without synchronising, unless
 *     stated; outputs are valid once the stream reaches the enqueued work.
 *   - Handles (st_ctx, st_kv, st_operator) are library-owned and not
 *     thread-safe: use one handle from one host thread at a time.
 *   - Weights, caches and workspaces are allocated by st_create, st_kv_alloc and
 *     st_reserve; st_kv_build / st_kv_retain / st_op_eval allocate only when the
 *     context's workspace must grow (never after st_reserve with the largest
 *     sizes used), and never when the caller provides it (st_set_workspace).
 */
#ifndef STRETTO_H
#define STRETTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define ST_OK 0
#define ST_EINVAL 1        /* invalid argument (message says which) */
#define ST_ENOMEM 2        /* device allocation failed */
#define ST_ECUDA 3         /* a CUDA runtime call failed */
#define ST_ETIMEOUT 4      /* a bounded device wait gave up */
#define ST_ENAN 5          /* a NaN retention score, or NaN map-operator logits */
#define ST_EUNSUPPORTED 6  /* shape not supported by the compiled kernels */
#define ST_ERANGE 7        /* (device status) a tuple id outside [0, T) */
#define ST_ECHECK 8        /* (device status, checked build only) an index or offset check failed */

/* ---- element types ---- */
#define ST_F32 0           /* IEEE float32 */
#define ST_BF16 1          /* bfloat16 */
#define ST_E4M3 2          /* OCP FP8 E4M3 with per-(64-slot block) float32 scales */

/* ---- operator kinds and filter decisions ---- */
#define ST_OP_FILTER 0     /* binary filter: label_ids = {accept token, reject token} */
#define ST_OP_CLASSIFY 1   /* n-way classify: argmax_k (z_k + bias_k), ties to lowest k */
#define ST_REJECT 0
#define ST_ACCEPT 1
#define ST_UNSURE 2

typedef struct st_ctx st_ctx;            /* model weights + workspace */
typedef struct st_kv st_kv;              /* the KV caches of one table */
typedef struct st_operator st_operator;  /* one operator's prompt, labels, r, thresholds */

/* Decoder shape (Llama-style, pre-norm; RMSNorm without gains; RoPE
 * rotate-half with frequencies rope_theta^(-2i/hd); SwiGLU FFN; untied LM head). */
typedef struct {
  int32_t layers;      /* decoder layers */
  int32_t d;           /* model width */
  int32_t hq, hkv;     /* query heads, key/value heads (hq % hkv == 0) */
  int32_t hd;          /* head dim: 32 or 64 (ST_F32), 64 (ST_BF16) */
  int32_t ffn;         /* SwiGLU hidden width (multiple of 128) */
  int32_t vocab;       /* vocabulary size */
  int32_t dtype;       /* ST_F32 or ST_BF16: weights, activations and the full cache */
  int32_t max_pos;     /* largest position + 1 any call may use (document + prompt) */
  float rope_theta;    /* RoPE base (10000) */
  float eps;           /* RMSNorm epsilon (1e-5) */
} st_model_cfg;

/* One operator (Sec. 5 "Online: Query Execution"). */
typedef struct {
  const int32_t* prompt;     /* host [P] prompt token ids, each < vocab */
  int32_t P;                 /* prompt length, 1..256 */
  const int32_t* label_ids;  /* host [n_labels] label token ids; filter: {accept, reject} */
  int32_t n_labels;          /* 2 for ST_OP_FILTER; 2..8 for ST_OP_CLASSIFY */
  int32_t kind;              /* ST_OP_FILTER or ST_OP_CLASSIFY */
  double r;                  /* retained fraction in (0, 1] of the KV profile it reads */
  float theta_pos;           /* filter: accept iff s - theta_pos is the unique largest of
                                (s - theta_pos, theta_neg - s, 0), s = z_accept - z_reject */
  float theta_neg;           /* filter: reject threshold (ties: unsure, then reject) */
  const float* bias;         /* host [n_labels] classify bias, or NULL for zeros */
} st_op;

/* ---- context ---- */

/* Create a context holding a packed copy of the model weights.
 * weights: 2 + 7*layers DEVICE pointers of cfg->dtype elements, row-major
 *   [out][in], in this order: embed [vocab][d]; per layer wq [hq*hd][d],
 *   wk [hkv*hd][d], wv [hkv*hd][d], wo [d][hq*hd], wg [ffn][d], wu [ffn][d],
 *   wd [d][ffn]; then w_lm [vocab][d].  They are copied (the caller may free
 *   them after the stream has passed this call's copies; the call synchronises
 *   `stream` before returning).
 * ST_BF16 contexts keep the projection and LM-head weights as IEEE half (an
 *   exact conversion of the given bf16 values) and run the projections on half
 *   operands (normalised inputs, attention and SwiGLU outputs stored as half,
 *   f32 accumulation); Q, K, V, attention probabilities and the KV cache are
 *   bf16, the residual stream float32.
 * Errors: ST_EINVAL on an unsupported shape, ST_ENOMEM, ST_ECUDA. */
int st_create(const st_model_cfg* cfg, const void* const* weights, void* stream, st_ctx** out);
void st_destroy(st_ctx* ctx);
const char* st_last_error(const st_ctx* ctx);   /* never NULL; "" when no error */
const char* st_version(void);

/* Pre-size the context's workspace for kv_build chunks of up to `build_rows`
 * document tokens and op_eval batches of up to `eval_rows` prompt rows
 * (tuples * P), so that later calls allocate nothing. */
int st_reserve(st_ctx* ctx, int64_t build_rows, int64_t eval_rows);

/* Caller-owned activation workspace (the boundary keeps no hidden device
 * allocation on the hot path when the caller provides it).
 *
 * st_workspace_size: bytes of device workspace that one chunk of `rows` rows
 * needs -- which = ST_WS_BUILD: st_kv_build over chunks of up to `rows`
 * document tokens (a document longer than that is one chunk of its own
 * length); ST_WS_EVAL: st_op_eval / st_op_eval_multi / st_map_eval over chunks
 * of up to `rows` prompt rows (tuples x P).  Returns 0 for a bad argument.
 *
 * st_set_workspace: from now on the context carves that workspace out of the
 * caller's device buffer `dev` of `bytes` bytes (256-byte aligned) instead of
 * allocating its own; the library's own buffer of that kind is freed (which
 * waits for the device).  The buffer is caller-owned: it must stay valid until
 * it is replaced, reset with dev = NULL, bytes = 0 (back to library-owned
 * workspace), or the context is destroyed; the library never frees it.  Calls
 * of the context must not overlap on the GPU (they share it).  A call whose
 * chunk needs more than `bytes` fails with ST_ENOMEM before launching
 * anything; st_reserve fixes the chunk sizes (its own allocation then fails
 * with ST_ENOMEM too if the caller's buffer is smaller).
 * Errors: ST_EINVAL (which, alignment, or dev / bytes not both set or both
 * zero). */
#define ST_WS_BUILD 0
#define ST_WS_EVAL 1
#define ST_WS_ANY 2
size_t st_workspace_size(const st_ctx* ctx, int which, int64_t rows);
int st_set_workspace(st_ctx* ctx, int which, void* dev, size_t bytes);
/* st_workspace_held: device bytes of workspace the context currently owns
 * (allocated by the library, not caller-provided) -- ST_WS_BUILD, ST_WS_EVAL,
 * or ST_WS_ANY for all of its workspaces (build, evaluation, cascade routing,
 * map decode, query scoring).  0 for a NULL context or an unknown kind.  A
 * diagnostic: it shows whether a call grew the library's own memory. */
size_t st_workspace_held(const st_ctx* ctx, int which);

/* ---- KV caches ---- */

/* Allocate the caches of a table of T tuples whose document i spans tokens
 * offsets_host[i] .. offsets_host[i+1]-1 (monotone, offsets_host[0] == 0,
 * every length in 1 .. max_pos-1).  Sizes the full cache (dtype of the model)
 * and the retained cache for any r <= 1 (either dtype).
 * Errors: ST_EINVAL (bad offsets: T < 1, offsets[0] != 0, an empty document
 * or one longer than max_pos - 1), ST_EUNSUPPORTED (a document longer than
 * 16384 tokens), ST_ENOMEM. */
int st_kv_alloc(st_ctx* ctx, const int64_t* offsets_host, int32_t T, st_kv** out);

/* A second retained profile of an existing cache `src` (Sec. 5 keeps several
 * compressed caches -- profiles -- per item, e.g. at two compression ratios or
 * precisions).  The returned handle shares src's document offsets, full cache
 * (K, V, scores) and pooled states -- they are not copied, and src must be
 * built through src and must outlive the profile -- and owns a retained cache
 * of its own, sized for any r <= r_max in either retained dtype
 * (sum over tuples of pad64(n_keep(L, r_max)) slots per layer and kv head).
 * st_kv_retain on it reads src's full cache (src must have been built) and
 * leaves src's own retained profile untouched, so one table can hold, say, a
 * BF16 and an E4M3 profile at once and st_op_eval can read either.
 * st_kv_build, st_kv_import and st_kv_score_query refuse a profile; st_kv_free
 * releases only what it owns.  Errors: ST_EINVAL (src is NULL, of another
 * context or itself a profile; r_max outside (0, 1]; later, st_kv_retain with
 * r > r_max), ST_ENOMEM. */
int st_kv_profile_alloc(st_ctx* ctx, st_kv* src, double r_max, st_kv** out);
void st_kv_free(st_kv* kv);

/* Offline KV-cache creation (Sec. 5).  tokens_dev: DEVICE int32 [offsets[T]]
 * token ids (< vocab; not checked on the device).  Fills, for every layer l,
 * kv head g and document slot j (positions 0..L-1, causal prefill of the
 * document alone): the post-RoPE key and value, the retention score
 *   score = mu.k/sqrt(hd) + sum_c sigma2_c k_c^2/(2 hd) + ln(||v|| + 1e-12)
 * (mu, sigma2: mean and population variance of the group's post-RoPE queries
 * over the document), and the pooled final-normed last-layer state of every
 * tuple.  Processed in chunks of whole tuples. */
int st_kv_build(st_ctx* ctx, st_kv* kv, const int32_t* tokens_dev, void* stream);

/* Process-wide choice of the BF16 projection GEMM for more than 128 rows:
 * on != 0 (default) runs CTA pairs with the 2-SM MMA (256 x 256 tiles, each
 * SM staging half of the A and W tiles); 0 runs one CTA per 128 x 256 tile.
 * Results are identical up to the order of the f32 accumulation (the same K
 * steps in the same order: bit-identical in practice).  Always ST_OK. */
int st_set_gemm_pairs(int32_t on);

/* ---- retention scoring (ablation of Sec. 5's query-agnostic choice) ----
 *
 * ST_SCORE_EA_LITE (default): the score documented at st_kv_build.
 * ST_SCORE_EA_FULL: Expected Attention with the RoPE rotation averaged over
 *   the future positions: per tuple, layer and kv head, mu and Sigma are the
 *   mean and full population covariance of the group's PRE-RoPE queries over
 *   the document; Rbar = (1/F) sum_{p=L}^{L+F-1} R(p) is the mean RoPE
 *   rotation over the horizon of F positions after the document;
 *   m = Rbar mu, M = Rbar Sigma Rbar^T, and slot j scores
 *     m.k_j/sqrt(hd) + k_j^T M k_j/(2 hd) + ln(||v_j|| + 1e-12)
 *   (the log of E[exp(q.k_j/sqrt(hd))] ||v_j|| for q ~ N(m, M)).
 * Query-specific scores: st_kv_score_query. */
#define ST_SCORE_EA_LITE 0
#define ST_SCORE_EA_FULL 1

/* Selects the score of later st_kv_build calls on this context.  horizon: F
 * for ST_SCORE_EA_FULL (1 .. 4096), ignored for EA-lite.  Builds then need
 * hd in {32, 64} (ST_EUNSUPPORTED otherwise) and every document length + F
 * <= max_pos (ST_EINVAL).  Errors: ST_EINVAL (mode, horizon >= max_pos),
 * ST_ENOMEM. */
int st_set_scoring(st_ctx* ctx, int32_t mode, int32_t horizon);

/* Query-specific scores (the contrast of Sec. 5, which keeps a query-agnostic
 * cache): forwards op's prompt against every tuple's whole cache (every slot,
 * whatever op's own r), which must hold a retained profile at r = 1 in the
 * model dtype, and replaces the cache's
 * scores by the attention probability that the prompt's queries (every prompt
 * position and query head of the group) put on each document slot, softmax
 * over the document slots and the visible prompt keys, per layer and kv head.
 * A following st_kv_retain ranks by these scores; st_kv_build restores the
 * query-agnostic ones.  hd must be 32 or 64.
 * Errors: ST_EINVAL (no r = 1 profile in the model dtype), ST_EUNSUPPORTED. */
int st_kv_score_query(st_ctx* ctx, st_kv* kv, const st_operator* op, void* stream);

/* Query-agnostic retention (Sec. 5): per tuple, layer and kv head, rank all
 * slots by (score descending, slot index ascending; -0 == +0) and keep the
 * first n_keep(L, r) = clamp(floor(r*L + 0.5), 1, L) (IEEE double arithmetic)
 * in rank order, as kv_dtype (the model dtype, or ST_E4M3 with one float32
 * scale = amax/448 per 64-slot block for K and for V).  Replaces the previous
 * retained profile of `kv`.  A NaN score sets the device status read by
 * st_kv_status (ST_ENAN). Errors: ST_EINVAL (r outside (0,1], kv_dtype). */
int st_kv_retain(st_ctx* ctx, st_kv* kv, double r, int32_t kv_dtype, void* stream);

/* Device status word of the context: synchronises `stream`, returns the first
 * error a kernel recorded since the last call, and clears it: ST_OK;
 * ST_ETIMEOUT (a tcgen05 pipeline wait gave up; the kernel returned early and
 * its outputs are invalid); ST_EINVAL (a token id outside [0, vocab) was
 * embedded as zeros); ST_ENAN (a map-operator step had no finite logit; its
 * token was set to 0). */
int st_status(st_ctx* ctx, void* stream);

/* Self-test of the failure path (the paper has no counterpart): launches one
 * kernel whose single thread waits on a device barrier that nothing completes,
 * through the same bounded wait as the pipeline kernels, giving up after
 * limit_cycles (1e3 .. 1e9) SM clock cycles and recording ST_ETIMEOUT in the
 * context's device status word; the next st_status reports (and clears) it,
 * and the context stays usable.  Faults and hangs nothing.
 * Errors: ST_EINVAL (limit out of range). */
int st_selftest_wait(st_ctx* ctx, int64_t limit_cycles, void* stream);

/* ---- retained-profile repository (Sec. 5: caches computed offline, stored,
 * and loaded per profile = model + compression ratio at query time) ----
 *
 * A profile blob holds what operator evaluation reads: the rank-ordered
 * retained K / V (used slots only), the E4M3 block scales, the per-tuple
 * retained counts and padded offsets, the pooled document states, and a
 * header (model shape and dtype, retained dtype, r, the table's size and
 * document offsets).  Blobs are plain host memory; the caller stores them.
 * st_kv_profile_bytes: size of the blob of kv's current profile
 *   (ST_EINVAL if kv has none).
 * st_kv_export: writes it to `host` (>= that many bytes); synchronises `stream`.
 * st_kv_import: makes the blob kv's retained profile.  kv must come from
 *   st_kv_alloc with the same document offsets; its full cache is not needed
 *   (operators at r' <= the profile's r evaluate right away), but st_kv_retain
 *   afterwards needs a new st_kv_build.  Synchronises `stream`.
 *   Errors: ST_EINVAL (not a blob, truncated, another model / table, corrupt
 *   counts), ST_ECUDA. */
int st_kv_profile_bytes(const st_kv* kv, size_t* bytes);
int st_kv_export(st_ctx* ctx, const st_kv* kv, void* host, size_t bytes, void* stream);
int st_kv_import(st_ctx* ctx, st_kv* kv, const void* host, size_t bytes, void* stream);

/* The retained slot indices at a fraction r (paper Sec. 5: the retained set
 * of each (tuple, layer, kv head) is the top n_keep(L, r) of its ranking):
 * off_dev (int64 [T+1], caller DEVICE memory) receives the offsets, off[0] = 0
 * and off[t+1] = off[t] + n_keep(L_t, r); idx_dev (int32 [layers][hkv][off[T]],
 * caller DEVICE memory, or NULL for the offsets only) receives, for every
 * (layer, kv head), each tuple's retained slot indices (0 .. L_t - 1) in rank
 * order at idx[l][g][off[t] .. off[t+1]-1].  Any r in (0, 1] (the ranking
 * covers each whole segment, so smaller r read prefixes: the sets are nested).
 * Valid after st_kv_retain and until the next st_kv_build.  Enqueued on
 * `stream`.  Errors: ST_EINVAL (r, no ranking yet, NULL off_dev). */
int st_kv_indices(st_ctx* ctx, const st_kv* kv, double r, int32_t* idx_dev, int64_t* off_dev, void* stream);

/* Device status of the last retain on `kv`: synchronises `stream`, returns
 * ST_OK or ST_ENAN (and clears it). */
int st_kv_status(st_ctx* ctx, st_kv* kv, void* stream);

/* Read-only device views of the cache buffers, for inspection and tests.
 * which: see ST_VIEW_*.  *ptr receives a DEVICE pointer owned by `kv`, *bytes
 * its size.  Layouts:
 *   ST_VIEW_K / ST_VIEW_V        full cache, model dtype [layers][hkv][R][hd], R = offsets[T]
 *   ST_VIEW_SCORES               float32 [layers][hkv][R]
 *   ST_VIEW_POOLED               float32 [T][d]
 *   ST_VIEW_RANK                 int32 [layers][hkv][R]: per tuple segment, slot indices
 *                                (0..L-1) in rank order (valid after st_kv_retain)
 *   ST_VIEW_KR / ST_VIEW_VR      retained cache [layers][hkv][Rp][hd] (model dtype, or one
 *                                byte per E4M3 code); tuple i occupies rows
 *                                offp[i] .. offp[i]+n_i-1, zero-filled to offp[i+1]
 *   ST_VIEW_SCALES               float32 [layers][hkv][Rp/64][2] (K scale, V scale)
 *   ST_VIEW_OFFP                 int64 [T+1] padded offsets (multiples of 64)
 *   ST_VIEW_NKEEP                int32 [T] retained counts n_i */
#define ST_VIEW_K 0
#define ST_VIEW_V 1
#define ST_VIEW_SCORES 2
#define ST_VIEW_POOLED 3
#define ST_VIEW_RANK 4
#define ST_VIEW_KR 5
#define ST_VIEW_VR 6
#define ST_VIEW_SCALES 7
#define ST_VIEW_OFFP 8
#define ST_VIEW_NKEEP 9
int st_kv_view(const st_kv* kv, int32_t which, void** ptr, size_t* bytes);
/* Copy min(bytes, size of the view) bytes of a view into caller DEVICE memory
 * dst_dev, enqueued on `stream`. */
int st_kv_read(const st_kv* kv, int32_t which, void* dst_dev, size_t bytes, void* stream);
/* Copy bytes [offset, offset + bytes) of a view into caller DEVICE memory.
 * Errors: ST_EINVAL (range outside the view). */
int st_kv_read_at(const st_kv* kv, int32_t which, size_t offset, void* dst_dev, size_t bytes, void* stream);

/* ---- operators ---- */

/* Upload an operator's prompt, labels and bias once (synchronous).
 * Errors: ST_EINVAL (P, n_labels, ids out of range, r outside (0,1]). */
int st_op_create(st_ctx* ctx, const st_op* op, st_operator** out);
void st_op_free(st_operator* op);

/* Online execution of one operator (Sec. 5) on the tuples tuple_ids_dev[0..n-1]
 * (DEVICE int32, each in [0, T); an id outside it is evaluated as tuple 0 and
 * recorded in the device status word, which st_status reports as ST_ERANGE)
 * of `kv`, whose retained
 * profile must have r >= op->r (a smaller r reads the rank-order prefix
 * n_keep(L, op->r), which is exactly the smaller profile's set).
 * Outputs: logits_dev DEVICE float32 [n][n_labels] (label-token logits at the
 * last prompt position), labels_dev DEVICE int32 [n] (ST_ACCEPT / ST_REJECT /
 * ST_UNSURE for a filter, the class index for classify).
 * Errors: ST_EINVAL (no retained profile, op->r above it, n < 0). */
int st_op_eval(st_ctx* ctx, const st_kv* kv, const st_operator* op,
               const int32_t* tuple_ids_dev, int32_t n, float* logits_dev,
               int32_t* labels_dev, void* stream);

/* ---- map operator (greedy decode) ----
 *
 * The paper's second operator type (Sec. 6 "Operators": a map generates a
 * value per item): the operator's prompt is forwarded against each tuple's
 * retained cache as in st_op_eval, then n_gen tokens are generated greedily —
 * token t is the argmax over the whole vocabulary (ties to the lowest id) of
 * the logits at the last position of prompt + tokens 0..t-1, and sits at the
 * next position (L + P + t).  Every step attends to the tuple's retained
 * slots (the operator's r) and to all prompt and generated keys, kept per
 * tuple in a decode cache.  op's label ids, kind and thresholds are unused.
 * tokens_dev: DEVICE int32 [n][n_gen]; logits_dev: NULL or DEVICE float32
 * [n][n_gen][vocab] (every step's logits, for inspection).
 * Errors: ST_EINVAL (n_gen outside 1..256, document + P + n_gen > max_pos,
 * op->r above the retained profile's), ST_EUNSUPPORTED (vocab not a multiple of
 * 256 for bf16 / 128 for f32 models). */
int st_map_eval(st_ctx* ctx, const st_kv* kv, const st_operator* op, const int32_t* tuple_ids_dev,
                int32_t n, int32_t n_gen, int32_t* tokens_dev, float* logits_dev, void* stream);

/* ---- batched evaluation of several operators ----
 *
 * Several operators (different prompts, label sets, kinds and retention
 * ratios r_k <= the retained profile's r), each over its own tuple set, in one
 * pass: the (operator, tuple) pairs of all operators share every projection
 * launch and one attention launch per layer; operator k reads the first
 * n_keep(L, r_k) slots of the shared rank-ordered cache (the retained sets
 * are nested in r, Sec. 5 "several profiles per item"; batching over items,
 * Sec. 6).  Results equal n_ops separate st_op_eval calls bit for bit.
 * ST_MAX_OPERATORS operators at most.
 * ops[k], tuple_ids_dev[k] (DEVICE int32 [n[k]]), n[k] (host), logits_dev[k]
 * (DEVICE float32 [n[k]][n_labels of ops[k]]), labels_dev[k] (DEVICE int32
 * [n[k]]): the arrays of pointers are host arrays of n_ops entries, read
 * during the call only.
 * Errors: ST_EINVAL (n_ops outside 1..ST_MAX_OPERATORS, an r above the
 * retained profile's, a NULL buffer with n[k] > 0). */
#define ST_MAX_OPERATORS 8
int st_op_eval_multi(st_ctx* ctx, const st_kv* kv, int32_t n_ops, const st_operator* const* ops,
                     const int32_t* const* tuple_ids_dev, const int32_t* n,
                     float* const* logits_dev, int32_t* const* labels_dev, void* stream);

/* ---- a batched evaluation as a CUDA graph ----
 *
 * st_graph_create records the whole batched evaluation (the same kernels as
 * st_op_eval_multi with these arguments) into a CUDA graph once;
 * st_graph_launch replays it on `stream`, one graph launch instead of one
 * host launch per kernel.  The graph keeps the DEVICE pointers it was
 * created with (tuple ids, outputs, the cache): the caller may change the
 * contents of those buffers between replays (other tuple ids, a new
 * retention of the same cache), not their addresses or counts, and must keep
 * them, the cache and the context alive until st_graph_free.  The graph owns
 * its activation workspace (allocated by st_graph_create, which also runs
 * the evaluation once uncaptured and synchronises).  Replays on one graph
 * must not overlap (they share the workspace).
 * st_graph_launches: kernels per replay.
 * Errors: as st_op_eval_multi; ST_ECUDA if capture or instantiation fails. */
typedef struct st_graph st_graph;
int st_graph_create(st_ctx* ctx, const st_kv* kv, int32_t n_ops, const st_operator* const* ops,
                    const int32_t* const* tuple_ids_dev, const int32_t* n, float* const* logits_dev,
                    int32_t* const* labels_dev, st_graph** out);
int st_graph_launch(st_graph* g, void* stream);
int64_t st_graph_launches(const st_graph* g);
void st_graph_free(st_graph* g);

/* ---- multi-stage cascade ----
 *
 * Sec. 4.1 cascades, any number of stages: stage k runs its filter operator
 * (its own context = model, cache, r, and thresholds theta+ / theta-) on the
 * tuples every earlier stage left unsure; a tuple leaves at the first stage
 * that accepts or rejects it; the last stage's unsure tuples stay ST_UNSURE.
 * All stages run on `stream` on one device.  For each input position i:
 * labels_dev[i] (DEVICE int32 [n]) = the deciding stage's decision,
 * stage_dev[i] (DEVICE int32 [n]) = that stage's index.  counts_host[k] (host,
 * n_stages entries, may be NULL) = tuples sent to stage k; ms_host[k] (may be
 * NULL) = its time (CUDA events: evaluation + routing).  Results equal running
 * st_op_eval stage by stage on the unsure tuples.  Synchronises `stream` once
 * per stage (to size the next stage's evaluation).  The routing buffers (about
 * 30 bytes per tuple) live in stage 0's context.
 * Errors: ST_EINVAL (no stage, a classify operator, a cache of another
 * context), and the errors of st_op_eval (message prefixed with the stage). */
typedef struct {
  st_ctx* ctx;
  const st_kv* kv;
  const st_operator* op;
} st_stage;
int st_cascade_run(int32_t n_stages, const st_stage* stages, const int32_t* tuple_ids_dev, int32_t n,
                   int32_t* labels_dev, int32_t* stage_dev, int32_t* counts_host, float* ms_host,
                   void* stream);

/* The learned-proxy cascade in one call: the proxy (below) as the cheap first
 * stage of the Sec. 4.1 cascade, in front of the operator stages of
 * st_cascade_run.
 *   1. The proxy evaluates the pooled states of the n tuples: row
 *      tuple_ids_dev[i] of x_dev (DEVICE float32 [T][d_in], e.g.
 *      ST_VIEW_POOLED).  Where its confidence is >= tau it decides the tuple.
 *   2. The other tuples, compacted in order, run through
 *      st_cascade_run(n_stages, stages) -- for instance an operator over an
 *      E4M3 profile with an unsure band (theta+ > theta-), then the same
 *      operator over the BF16 profile on what the first leaves unsure.
 *   3. labels_dev[i] (DEVICE int32 [n]): the proxy's label (0 reject,
 *      1 accept) where it decided, else the deciding stage's decision;
 *      stage_dev[i] (DEVICE int32 [n]): 0 for the proxy, k + 1 for stage k.
 * counts_host (optional, [n_stages + 1]): n, then the tuples sent to each
 * operator stage.  Routing buffers are the context's (grown on demand).
 * Synchronises `stream` after the proxy and after each operator stage, to size
 * the next stage's launches.  Errors: ST_EINVAL, ST_ENOMEM, and those of the
 * stages (the message names the stage). */
typedef struct st_proxy st_proxy;
int st_proxy_cascade(st_ctx* ctx, st_proxy* p, const float* x_dev, float tau, int32_t n_stages,
                     const st_stage* stages, const int32_t* tuple_ids_dev, int32_t n,
                     int32_t* labels_dev, int32_t* stage_dev, int32_t* counts_host, void* stream);

/* ---- schedule of operator evaluation, and its autotuner ----
 *
 * eval_rows: prompt rows per pass through the layers (the evaluation is cut
 * into chunks of at most this many rows; 0 = library default 262144);
 * attn_nb: tensor-core attention layout, 1 = two CTAs per SM with single S /
 * P / O buffers (default; 128-key tiles, 64-key tiles with E4M3 KV), 2 = one
 * CTA per SM with double buffers, 3 = as 1 but with 128-key tiles and one f16
 * stage for E4M3 KV (the same as 1 for BF16 KV); longest_first: attention work
 * items ordered by retained document
 * length, longest first (1, default) or in arrival order (0).  ms: measured
 * time of one evaluation (autotuner output).
 * st_autotune_eval times the batched evaluation of its arguments (which it
 * runs, writing the outputs) under candidate schedules — a coordinate search:
 * layout (1, 2, and 3 for E4M3 KV) x order at the current chunk size, then
 * chunk sizes 2^15 .. 2^19, then (when the cache holds documents longer than
 * 2048 slots) split-KV at 2048 retained slots —
 * each one warm-up and three timed runs (CUDA events on `stream`; it
 * synchronises), keeps the fastest in the context for later evaluations and
 * graphs, and returns it in *best; the first max_tried timed candidates go to
 * tried[] and their count to *n_tried (either may be NULL).
 * st_set_schedule sets a schedule directly. */
typedef struct {
  int64_t eval_rows;
  int32_t attn_nb;
  int32_t longest_first;
  int32_t split_keys;   /* split-KV: retained documents longer than this many slots are cut into
                           pieces of this many, each a separate work item whose partial
                           result (unnormalised O, running max, row sum) a merge pass combines
                           (0 = off, else a multiple of 128 up to 65536) */
  float ms;
} st_tune_choice;
int st_autotune_eval(st_ctx* ctx, const st_kv* kv, int32_t n_ops, const st_operator* const* ops,
                     const int32_t* const* tuple_ids_dev, const int32_t* n, float* const* logits_dev,
                     int32_t* const* labels_dev, void* stream, st_tune_choice* best,
                     st_tune_choice* tried, int32_t max_tried, int32_t* n_tried);
int st_set_schedule(st_ctx* ctx, const st_tune_choice* schedule);

/* ---- operator evaluation without device allocation ----
 *
 * The paper has no counterpart to this entry; it exists for callers that
 * cannot let the library allocate device memory: a query executor that keeps
 * several streams busy cannot afford the implicit device synchronisation of
 * cudaFree (and at times cudaMalloc), and a process whose GPU memory is already
 * claimed by another framework's caching allocator can see a fresh cudaMalloc
 * fail although that allocator holds free blocks.
 *
 * st_op_eval_noalloc computes exactly what st_op_eval computes (same kernels,
 * same order) but never allocates: its activations live in one file-scope
 * device array of ST_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until the process exits.  The caller still passes the inputs
 * (context, caches, operator, DEVICE tuple ids) and the outputs (DEVICE logits
 * float32 [n][n_labels], labels int32 [n]).
 *   - Size limit: n * P prompt rows must fit the array (about 16.9 KB per row
 *     for the config-2 decoder: 62 tuples with a 32-token prompt); larger n is
 *     rejected with ST_EINVAL and a message giving the bytes needed.
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array, which keeps the last call's contents (nothing
 *     in it needs to start at zero).  Calls whose work overlaps on the GPU (two
 *     streams or two host threads) race on it: serialise them.
 *   - No profiling events are recorded for this entry (st_prof_read omits it);
 *     its launches are counted by st_launch_count. */
#define ST_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int st_op_eval_noalloc(st_ctx* ctx, const st_kv* kv, const st_operator* op,
                       const int32_t* tuple_ids_dev, int32_t n, float* logits_dev,
                       int32_t* labels_dev, void* stream);

/* The whole path from HOST buffers: copy tokens_host (int32 [offsets[T]]) to
 * the device, st_kv_build, st_kv_retain(op->r, kv_dtype), st_op_eval over all
 * T tuples, and copy logits (float32 [T][n_labels]) and labels (int32 [T]) back
 * to host memory.  Synchronises `stream` before returning. */
int st_run_host(st_ctx* ctx, st_kv* kv, const st_operator* op, int32_t kv_dtype,
                const int32_t* tokens_host, float* logits_host, int32_t* labels_host,
                void* stream);

/* ---- learned proxy and two-stage cascade ----
 *
 * A cheap first stage in front of the operator (the cascade of Sec. 4.1: a
 * stage accepts or rejects a tuple, or marks it unsure and passes it on to the
 * next, more expensive stage).  The proxy is an MLP
 *   Linear(d_in, h1) - GELU(erf) - Linear(h1, h2) - GELU - Linear(h2, 2)
 * over each tuple's pooled last-layer document state (ST_VIEW_POOLED of
 * st_kv_build), trained with softmax cross-entropy and Adam (beta 0.9 / 0.999,
 * eps 1e-8, bias-corrected) against the full operator's labels (0 reject,
 * 1 accept).  float32 parameters, activations and accumulation. */
#define ST_PROXY_PARAMS 0   /* w1 [h1][d_in], b1 [h1], w2 [h2][h1], b2 [h2], w3 [2][h2], b3 [2] */
#define ST_PROXY_GRADS 1    /* the same layout: gradients of the last train step */
#define ST_PROXY_ADAM_M 2
#define ST_PROXY_ADAM_V 3
/* init_host: 6 HOST float32 arrays in the ST_PROXY_PARAMS order (copied). */
int st_proxy_create(st_ctx* ctx, int32_t d_in, int32_t h1, int32_t h2,
                    const float* const* init_host, st_proxy** out);
void st_proxy_free(st_proxy* p);
/* One Adam step on the mini-batch x_dev[batch_dev[b]] (DEVICE float32 [n][d_in]
 * rows, int32 labels y_dev indexed like x); loss_dev (DEVICE float32 [1], or
 * NULL) receives the batch's mean cross-entropy. */
int st_proxy_train_step(st_ctx* ctx, st_proxy* p, const float* x_dev, const int32_t* y_dev,
                        const int32_t* batch_dev, int32_t B, float lr, float* loss_dev,
                        void* stream);
/* Proxy decision for rows x_dev[rows_dev[i]] (rows_dev NULL: rows 0..n-1):
 * conf_dev (float32 [n]) = max softmax probability, label_dev (int32 [n]) =
 * argmax (ties to 0). */
int st_proxy_eval(st_ctx* ctx, st_proxy* p, const float* x_dev, const int32_t* rows_dev, int32_t n,
                  float* conf_dev, int32_t* label_dev, void* stream);
/* Cascade routing: the positions i (or ids_dev[i] when ids_dev is not NULL)
 * with conf_dev[i] < tau, in increasing order, into unsure_dev; their number
 * into count_dev (DEVICE int32 [1]).  One block; n <= 2^31-1. */
int st_cascade_compact(st_ctx* ctx, const float* conf_dev, const int32_t* ids_dev, int32_t n,
                       float tau, int32_t* unsure_dev, int32_t* count_dev, void* stream);
/* Cascade merge: out_dev[i] = proxy_label_dev[i], then
 * out_dev[unsure_pos_dev[j]] = full_label_dev[j] for j < min(*count_dev, n)
 * (a position outside [0, n) is skipped and recorded in the device status
 * word, reported by st_status as ST_ERANGE). */
int st_cascade_merge(st_ctx* ctx, const int32_t* proxy_label_dev, int32_t n,
                     const int32_t* unsure_pos_dev, const int32_t* count_dev,
                     const int32_t* full_label_dev, int32_t* out_dev, void* stream);
/* Copy one of the ST_PROXY_* buffers (float32, ST_PROXY_PARAMS layout) to DEVICE memory. */
int st_proxy_read(const st_proxy* p, int32_t which, void* dst_dev, size_t bytes, void* stream);
/* Checkpoint / resume of training: st_proxy_steps returns the Adam steps taken
 * (-1 for NULL); st_proxy_restore sets the parameters and both Adam moments
 * from caller DEVICE buffers (float32, ST_PROXY_PARAMS layout, n_params each,
 * as st_proxy_read writes them) and the step count, so that the next
 * st_proxy_train_step continues exactly where the saved proxy stopped.
 * `bytes` is the size of EACH of the three buffers and must equal
 * n_params * 4 of this proxy; nothing is read otherwise (a state saved from a
 * proxy of another shape, or a truncated buffer).  Enqueued on `stream`.
 * Errors: ST_EINVAL (NULL buffer, wrong size, steps < 0). */
int64_t st_proxy_steps(const st_proxy* p);
/* Precision of the proxy's contractions: ST_F32 (default; float32 on the CUDA
 * cores) or ST_BF16 (the tensor cores' mma.sync m16n8k16: each operand of
 * every forward and backward product rounded to bfloat16, nearest-even, as it
 * is staged; float32 accumulation).  Parameters, Adam moments, biases, GELU,
 * loss and bias gradients stay float32.  Takes effect from the next call.
 * Errors: ST_EINVAL (NULL proxy, another dtype). */
int st_proxy_set_precision(st_proxy* p, int32_t dtype);
int st_proxy_restore(st_proxy* p, const float* params_dev, const float* m_dev, const float* v_dev,
                     size_t bytes, int64_t steps, void* stream);

/* ---- kernel self-test entry ---- */

/* The projection GEMM of the context's precision with a plain store epilogue:
 * C_dev (float32 [M][N]) = A_dev ([M][K], model dtype) . W_dev ([N][K], model
 * dtype)^T, row-major, on the tcgen05 path for ST_BF16 contexts and the
 * CUDA-core path for ST_F32.  Shapes must satisfy the kernels' tiling (bf16:
 * N % 256 == 0, K % 64 == 0). */
int st_gemm(st_ctx* ctx, const void* A_dev, const void* W_dev, int32_t M, int32_t N, int32_t K,
            float* C_dev, void* stream);

/* ---- per-kernel timing (CUDA events on the launching stream) ---- */

/* When enabled, every launch of the library's kernels is bracketed by CUDA
 * events; st_prof_read sums, per kernel family, the launches, total device
 * milliseconds and the algorithmic FLOPs and bytes of those launches.
 * families: ST_PROF_GEMM, ST_PROF_ATTN, ST_PROF_RETAIN, ST_PROF_OTHER. */
#define ST_PROF_GEMM 0
#define ST_PROF_ATTN 1
#define ST_PROF_RETAIN 2
#define ST_PROF_OTHER 3
#define ST_PROF_N 4
int st_prof_enable(st_ctx* ctx, int32_t on);
/* Synchronises all pending events; out[f] = {launches, ms, flops, bytes}. */
int st_prof_read(st_ctx* ctx, double* out /* [ST_PROF_N][4] */);
int st_prof_reset(st_ctx* ctx);
/* Number of kernel launches the library enqueued since the last reset. */
int64_t st_launch_count(const st_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* STRETTO_H */
