// Attention on the 5th-generation tensor cores (tcgen05) for one kv head and
// 128 query rows per CTA: all G query heads of the group share every key/value
// tile staged in shared memory.
//
//   S = Q K^T   tcgen05.mma M128 K16 x4, N = the tile's visible key columns
//               rounded up to 32; Q and K K-major (128-byte swizzle) in shared
//               memory, f32 accumulator in TMEM (two 128-column buffers).
//   softmax     4 warps, one thread per query row: the row is that thread's TMEM
//               lane, so max / exp2 / sum need no shuffles; P is written back
//               to TMEM (tcgen05.st) as packed 16-bit pairs.
//   O += P V    tcgen05.mma M128 N64 K16, A = P read from TMEM, B = V read
//               MN-major from its [key][dim] shared-memory tile; O accumulates
//               in TMEM (one 64-column buffer per item, two in flight). A row's
//               running max moves only when a tile maximum exceeds it by more
//               than 8 (P <= 256), and then the row of O is rescaled in place
//               (tcgen05.ld / st) before the next P.V; O is read out once, at
//               the end of the item.
//   loads       one thread decodes each work item (into shared memory for the
//               other roles) and issues TMA for its Q (3-D box, two buffers)
//               and its K/V tiles (2-5 stages), in 64-row boxes, so that key
//               rows no query of the item can see are not read.
//   E4M3 KV     raw code tiles land in raw stages; one warp widens the K codes
//               and one the V codes exactly to f16 into the swizzled K/V stage,
//               each as soon as the stage's half is free; Q and the prompt's
//               K/V arrive in f16, both products run as f16 MMAs, the K block
//               scale multiplies the f32 scores and the V block scale P.
//
// Modes: prefill (the document's own keys, causal) and eval (the tuple's
// retained slots, all visible, then the prompt's keys, causal).
// Every mbarrier wait is bounded; a timeout sets the status word.
#include <cudaTypedefs.h>

#include "kernels.h"
#include "ptx.cuh"

namespace st {
namespace {

constexpr int HD = 64;
constexpr int BOX = 64;          // key rows per TMA box
constexpr int ROWS = 128;        // query rows per work item
// Two layouts, by the number NB of S, P and O buffers:
//   NB = 1: two CTAs per SM, each with one S, P and O buffer in 256 TMEM
//           columns, so every SM sub-partition runs two independent softmax
//           warps (the default).  E4M3 KV runs 64-key tiles (two f16 K/V
//           stages, 64 scores per softmax thread), whose register, shared-
//           memory and TMEM budget fits two CTAs per SM; a selectable layout
//           runs 128-key E4M3 tiles with one f16 K/V stage behind two raw code
//           stages (98 KB of shared memory), S read from TMEM in two 64-column
//           passes to fit the 128 registers two CTAs of 256 threads leave the
//           softmax -- measured 30 % slower: with one f16 stage the widening
//           of a tile's V waits for the previous tile's P.V;
//   NB = 2: one CTA per SM with double buffers in 512 TMEM columns.
// K/V stages: 2 (NB = 1; 1 for E4M3 128-key tiles) or 5 (NB = 2; 4 with
// E4M3 KV), and with E4M3 KV two raw code stages.
constexpr int ctas_per_sm(int nb) { return nb == 1 ? 2 : 1; }
constexpr int NKV_MAX = 5, NRAW_MAX = 2;
constexpr int nkv(bool fp8, int nb, int tk) { return nb == 1 ? (fp8 && tk == 128 ? 1 : 2) : (fp8 ? 4 : 5); }
constexpr int nraw(bool fp8, int nb) { return fp8 ? 2 : 0; }
// warps 0-3 softmax, 4 item decode + Q and K/V loads, 5 MMA issue,
// (E4M3 KV) 6 widens the K codes to f16, 7 the V codes
constexpr int nthreads(bool fp8) { return fp8 ? 256 : 192; }
constexpr int OFF_Q = 0;                           // 2 x 16 KB
constexpr int OFF_K = OFF_Q + 2 * ROWS * 128;      // nkv x 16 KB
constexpr int off_v(bool fp8, int nb, int tk) { return OFF_K + nkv(fp8, nb, tk) * tk * 128; }   // nkv x tk x 128 B
constexpr int off_raw(bool fp8, int nb, int tk) { return off_v(fp8, nb, tk) + nkv(fp8, nb, tk) * tk * 128; }
constexpr int raw_bytes(int tk) { return 2 * tk * HD; }   // K + V codes of one tile
constexpr int off_bar(bool fp8, int nb, int tk) { return off_raw(fp8, nb, tk) + nraw(fp8, nb) * raw_bytes(tk); }
constexpr int off_work(bool fp8, int nb, int tk) { return off_bar(fp8, nb, tk) + 512; }   // 2 decoded work items
constexpr size_t smem_bytes(bool fp8, int nb, int tk) { return (size_t)off_work(fp8, nb, tk) + 256 + 1024; }
// TMEM columns: S buffers [0, tk nb), O buffers [tk nb, (tk + 64) nb), P buffers
// [(tk + 64) nb, (1.5 tk + 64) nb) -- within 256 nb for tk <= 128
constexpr uint32_t tmem_cols(int nb) { return 256 * nb; }
constexpr uint32_t col_o(int nb, int tk) { return tk * nb; }
constexpr uint32_t col_p(int nb, int tk) { return (tk + HD) * nb; }

struct Bars {
  // K and V halves of a stage fill and free separately: K after the tile's
  // S = Q K^T, V after its P.V
  uint64_t k_full[NKV_MAX], v_full[NKV_MAX], k_empty[NKV_MAX], v_empty[NKV_MAX], s_full[2], s_free[2], p_full[2], pv_done[2], o_free[2];
  uint64_t q_full[2], q_empty[2];
  // E4M3: K / V halves of a stage widened; raw code stages loaded / free
  uint64_t kc_full[NKV_MAX], vc_full[NKV_MAX], raw_full[NRAW_MAX], raw_empty[NRAW_MAX];
  uint32_t tmem;
};
static_assert(sizeof(Bars) <= 512, "barrier block");

__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 2^x on the special-function unit (flushes subnormal results to zero, which a
// softmax probability can afford).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
  float y;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}
// Two float32 lanes in one 64-bit register (lane 0 low): Blackwell's packed
// FP32 pipe runs fma / add / mul on both with one instruction.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2lo(uint64_t x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float f2hi(uint64_t x) { return __uint_as_float((uint32_t)(x >> 32)); }
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Maximum of the 32 scores of one chunk: four chains of 3-input maxima (few
// live temporaries next to the row's 128 scores).
__device__ __forceinline__ float chunk_max(const uint32_t* v) {
  float m[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) m[q] = fmaxf(__uint_as_float(v[8 * q]), __uint_as_float(v[8 * q + 1]));
#pragma unroll
  for (int k = 2; k < 8; k += 2)
#pragma unroll
    for (int q = 0; q < 4; ++q) m[q] = max3(m[q], __uint_as_float(v[8 * q + k]), __uint_as_float(v[8 * q + k + 1]));
  return fmaxf(max3(m[0], m[1], m[2]), m[3]);
}
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
// MN-major operand with the 128-byte swizzle: 64 elements (128 B) along N per
// row, 8 K-rows per 1024-byte atom; consecutive 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_mnmajor_sw128(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFF);
  d |= (uint64_t)(1024 >> 4) << 16;   // leading byte offset (one 64-wide N atom: unused)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset between 8-row K groups
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

struct TileInfo {
  bool prompt;
  int key0, count;   // first key, keys present in the tile
  int kc;            // keys visible to at least one query row of the item (>= 1)
};

// One work item: 128 query rows of one kv head of one tuple.
template <int MODE, int TK>
struct Work {
  int g, G, rows, row_base, n_tiles, n_doc_tiles;
  int i, n_doc, P;          // eval
  int t, j0, L;             // prefill
  int lim_max;              // largest causal limit (query position) among the rows
  int qoff;                 // (eval) position of the first query among the prompt keys
  int piece, pieces, pslot; // (eval, split-KV) this piece of the pair, their number, its partial-result slot
  int k_lo, k_hi;           // retained slots of the item: [k_lo, k_hi)
  int64_t doc_row0, prompt_row0, qrow0, qbase;

  __device__ void decode(const AttnParams& a, const int32_t* items, int w, int zb_count) {
    G = a.hq / a.hkv;
    if (MODE == 1) {
      // work list record (pair, 128-row block | piece | pieces, P, retained
      // slots, prompt row, partial-result slot, offp of the tuple), longest
      // documents first; kv head fastest
      const int e = w / a.hkv;
      g = w % a.hkv;
      const int4* rec = reinterpret_cast<const int4*>(items + (int64_t)WORK_INTS * e);
      const int4 r0 = rec[0], r1 = rec[1];
      i = r0.x;
      const int zb = r0.y & 0xFF;
      piece = (r0.y >> 8) & 0xFF;
      pieces = max(1, (r0.y >> 16) & 0xFF);
      pslot = r1.y;
      P = r0.z;                                    // prompt keys of the pair
      prompt_row0 = r1.x;
      qbase = prompt_row0;
      if (a.pq0) {
        // decode steps: the prompt grows and moves every step (read live)
        P = a.pP[i];
        prompt_row0 = a.prow[i];
        qbase = a.pq0[i];
      }
      const int nq = a.nq > 0 ? a.nq : P;          // its queries: the last nq positions
      qoff = P - nq;
      row_base = zb * ROWS;
      rows = min(ROWS, nq * G - row_base);
      lim_max = qoff + (row_base + rows - 1) / G;
      n_doc = r0.w;
      doc_row0 = (int64_t)g * a.Rp_cap + (int64_t)(((uint64_t)(uint32_t)r1.w << 32) | (uint32_t)r1.z);
      qrow0 = qbase + row_base / G;
      // a piece of a split pair takes split_keys of the retained slots; the
      // prompt's keys go with the last piece
      k_lo = pieces > 1 ? piece * a.split_keys : 0;
      k_hi = pieces > 1 ? min(n_doc, k_lo + a.split_keys) : n_doc;
      n_doc_tiles = (k_hi - k_lo + TK - 1) / TK;
      n_tiles = n_doc_tiles + (piece == pieces - 1 ? (min(P, lim_max + 1) + TK - 1) / TK : 0);
    } else {
      const int it = w / a.hkv;
      g = w % a.hkv;
      t = items[2 * it];
      j0 = items[2 * it + 1];
      L = (int)(a.off[t + 1] - a.off[t]);
      row_base = 0;
      rows = ROWS;
      doc_row0 = (int64_t)g * a.R + a.off[t];
      qrow0 = a.off[t] - a.r0 + j0;
      lim_max = min(j0 + ROWS / G, L) - 1;
      n_doc_tiles = lim_max / TK + 1;
      n_tiles = n_doc_tiles;
      qoff = 0;
      qbase = 0;
      piece = 0;
      pieces = 1;
      pslot = -1;
      k_lo = 0;
      k_hi = L;
    }
  }
  // Checked build (eval items): the item's retained rows lie in its kv head's
  // plane, its prompt and query rows in their tensors.  A failed check records
  // ST_ECHECK and reduces the item to one query position attending to prompt
  // row 0 (every access then lies inside the tensors; the item's outputs are
  // not meaningful).
  __device__ void check(const AttnParams& a, int* status) {
#ifdef ST_CHECK
    if (MODE != 1) return;
    const int64_t prow_n = a.kvrows > 0 ? a.kvrows : a.qrows;
    const bool ok = n_doc >= 0 && doc_row0 >= (int64_t)g * a.Rp_cap &&
                    doc_row0 + n_doc <= (int64_t)(g + 1) * a.Rp_cap && P >= 1 && prompt_row0 >= 0 &&
                    prompt_row0 + P <= prow_n && qrow0 >= 0 && rows >= 1 && qrow0 + (rows + G - 1) / G <= a.qrows;
    if (!ST_CHECKED(ok, status)) {
      n_doc = 0;
      n_doc_tiles = 0;
      k_lo = k_hi = 0;
      piece = 0;
      pieces = 1;
      pslot = -1;
      doc_row0 = (int64_t)g * a.Rp_cap;
      P = 1;
      qoff = 0;
      row_base = 0;
      rows = G;
      lim_max = 0;
      prompt_row0 = 0;
      qbase = 0;
      qrow0 = 0;
      n_tiles = 1;
    }
#else
    (void)a;
    (void)status;
#endif
  }
  __device__ TileInfo tile(int ti) const {
    TileInfo T;
    if (MODE == 1 && ti >= n_doc_tiles) {
      T.prompt = true;
      T.key0 = (ti - n_doc_tiles) * TK;
      T.count = min(TK, P - T.key0);
    } else {
      T.prompt = false;
      T.key0 = k_lo + ti * TK;
      T.count = min(TK, k_hi - T.key0);
    }
    T.kc = (MODE == 0 || T.prompt) ? min(T.count, lim_max - T.key0 + 1) : T.count;
    return T;
  }
};

// Persistent: CTA b processes work items b, b + gridDim.x, ...; the load,
// MMA, softmax (and E4M3 widening) roles each walk the same sequence,
// connected by mbarrier rings (decoded item + Q: 2 slots, K/V: 3 stages, S, P
// and O: 2 TMEM buffers each), so the next item's loads overlap this item's math.
template <int MODE, bool FP8, int NB, int TK>
__global__ void __launch_bounds__(nthreads(FP8), ctas_per_sm(NB))
    k_attn_tc(AttnParams a, const int32_t* __restrict__ items, int n_work, int zb_count,
              const __grid_constant__ CUtensorMap tmQ,
              const __grid_constant__ CUtensorMap tmK, const __grid_constant__ CUtensorMap tmV,
              const __grid_constant__ CUtensorMap tmKp, const __grid_constant__ CUtensorMap tmVp,
              int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  Bars* bars = reinterpret_cast<Bars*>(smem + off_bar(FP8, NB, TK));
  Work<MODE, TK>* slots = reinterpret_cast<Work<MODE, TK>*>(smem + off_work(FP8, NB, TK));
  static_assert(sizeof(Work<MODE, TK>) <= 128, "work slot");
  // split-KV: the work list's entry count is on the device (the launch used a bound)
  if (MODE == 1 && a.nwork_dev) n_work = min(n_work, *a.nwork_dev * a.hkv);
  const uint32_t sQ0 = ptx::smem_u32(smem + OFF_Q);
  static_assert(TK == 128 || TK == 64, "tile width");
  constexpr int NKV = nkv(FP8, NB, TK), OFF_V = off_v(FP8, NB, TK), OFF_RAW = off_raw(FP8, NB, TK);
  static_assert(smem_bytes(FP8, NB, TK) <= (NB == 1 ? 113u * 1024 : 227u * 1024), "shared memory per CTA");
  constexpr int RAW_BYTES = raw_bytes(TK), NRAW = FP8 ? nraw(FP8, NB) : 1;   // (1: unused with BF16 KV)
  constexpr int NCH = TK / 32, NHALF = TK / 64;   // 32-key chunks, 64-key halves of a tile
  // scores the softmax holds in registers at once (E4M3 128-key tiles with
  // single buffers: two CTAs of 256 threads leave 128 registers a thread)
  constexpr int VW = (FP8 && NB == 1 && TK == 128) ? 64 : TK;
  constexpr int CPP = VW / 32, NPASS = TK / VW;   // chunks per pass, passes over S
  constexpr uint32_t TMEM_COLS = tmem_cols(NB), COL_O = col_o(NB, TK), COL_P = col_p(NB, TK);
  const uint32_t sK0 = ptx::smem_u32(smem + OFF_K), sV0 = ptx::smem_u32(smem + OFF_V);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NKV; ++s) {
      ptx::mbar_init(&bars->k_full[s], 1);
      ptx::mbar_init(&bars->v_full[s], 1);
      ptx::mbar_init(&bars->k_empty[s], 1);
      ptx::mbar_init(&bars->v_empty[s], 1);
      ptx::mbar_init(&bars->kc_full[s], 32);
      ptx::mbar_init(&bars->vc_full[s], 32);
    }
    for (int s = 0; s < NRAW; ++s) {
      ptx::mbar_init(&bars->raw_full[s], 1);
      ptx::mbar_init(&bars->raw_empty[s], 64);
    }
    for (int s = 0; s < 2; ++s) {
      ptx::mbar_init(&bars->s_full[s], 1);
      ptx::mbar_init(&bars->s_free[s], 128);
      ptx::mbar_init(&bars->p_full[s], 128);
      ptx::mbar_init(&bars->pv_done[s], 1);
      ptx::mbar_init(&bars->o_free[s], 128);
      ptx::mbar_init(&bars->q_full[s], 1);
      // the MMA's commit once the item's Q is consumed + every other reader of the slot
      ptx::mbar_init(&bars->q_empty[s], 1 + 128 + (FP8 ? 64 : 0));
    }
    ptx::fence_mbar_init();
  }
  if (warp == 5) {
    ptx::tmem_alloc(&bars->tmem, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = bars->tmem;

  if (warp == 4) {
    // ------------------------------------------------------------ decode + TMA
    if (lane == 0) {
      ptx::tma_prefetch_desc(&tmQ);
      ptx::tma_prefetch_desc(&tmK);
      ptx::tma_prefetch_desc(&tmV);
      int last_kv[NKV];
      uint32_t n_tma[NKV];      // TMA fills of each stage (its k_full / v_full completions)
      for (int s = 0; s < NKV; ++s) {
        last_kv[s] = -1;
        n_tma[s] = 0;
      }
      // L2 prefetch cursor: walks the same (item, tile) sequence PF tiles ahead
      // of the loads, so that a stage's TMA load, issued once the stage is
      // free, finds its rows in L2
      constexpr int PF = 4;
      Work<MODE, TK> PW;
      int pw = blockIdx.x, pti = 0;
      if (pw < n_work) PW.decode(a, items, pw, zb_count);
      auto prefetch_next = [&]() {
        if (pw >= n_work) return;
        const TileInfo T = PW.tile(pti);
        const int nbox = (T.kc + BOX - 1) / BOX;
        for (int h = 0; h < nbox; ++h) {
          if (T.prompt) {
            const int y = (int)(PW.prompt_row0 + T.key0 + h * BOX);
            ptx::tma_prefetch_l2_2d(&tmKp, PW.g * HD, y);
            ptx::tma_prefetch_l2_2d(&tmVp, PW.g * HD, y);
          } else {
            const int y = (int)(PW.doc_row0 + T.key0 + h * BOX);
            ptx::tma_prefetch_l2_2d(&tmK, 0, y);
            ptx::tma_prefetch_l2_2d(&tmV, 0, y);
          }
        }
        if (++pti == PW.n_tiles) {
          pti = 0;
          pw += gridDim.x;
          if (pw < n_work) PW.decode(a, items, pw, zb_count);
        }
      };
      for (int i = 0; i < PF; ++i) prefetch_next();
      bool ok = true;
      uint32_t c = 0, dc = 0, qc = 0;   // tile / E4M3 document-tile / item counters of this CTA
      int last_raw[NRAW_MAX], last_q[2] = {-1, -1};
      for (int s = 0; s < NRAW_MAX; ++s) last_raw[s] = -1;
      // E4M3: widened fills of each stage, and the one whose completion this
      // warp has not observed yet (-1: none)
      uint32_t n_cvt[NKV];
      int pend_cvt[NKV];
      for (int s = 0; s < NKV; ++s) {
        n_cvt[s] = 0;
        pend_cvt[s] = -1;
      }
      for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x, ++qc) {
        // the item into slot qc & 1 once every reader of the item two back is done with it
        const int qb = qc & 1;
        if (!ptx::mbar_wait(&bars->q_empty[qb], ((qc >> 1) & 1) ^ 1)) { ok = false; break; }
        Work<MODE, TK> W;
        W.decode(a, items, w, zb_count);
        W.check(a, status);
        slots[qb] = W;
        ptx::mbar_arrive_expect_tx(&bars->q_full[qb], ROWS * 128);
        ptx::tma_load_3d(smem + OFF_Q + qb * ROWS * 128, &tmQ, &bars->q_full[qb], 0, W.g * W.G,
                         (int)W.qrow0);
        last_q[qb] = (int)((qc >> 1) & 1);
        for (int ti = 0; ti < W.n_tiles; ++ti, ++c) {
          const int s = c % NKV;
          const uint32_t u = c / NKV;
          const TileInfo T = W.tile(ti);
          const int nbox = (T.kc + BOX - 1) / BOX;
          prefetch_next();
          if (FP8) {
            // With E4M3 KV, stage s is filled in turn by this warp (TMA, prompt
            // tiles) and by the widening warps (document tiles).  A parity wait
            // is unambiguous only while the waiter trails the barrier by at most
            // one phase, so before its next fill of stage s this warp observes
            // the completion of the stage's last widened fill: that widening
            // itself waited for the release before it, so the stage's release
            // barriers are then at most one phase ahead of this warp's view.
            if (pend_cvt[s] >= 0) {
              const uint32_t ph = (uint32_t)pend_cvt[s] & 1;
              if (!ptx::mbar_wait(&bars->kc_full[s], ph) || !ptx::mbar_wait(&bars->vc_full[s], ph)) {
                ok = false;
                break;
              }
              pend_cvt[s] = -1;
            }
            if (!T.prompt) {
              // raw codes into a raw stage; the widening warps fill K/V stage s
              const int rs = dc % NRAW;
              if (!ptx::mbar_wait(&bars->raw_empty[rs], ((dc / NRAW) & 1) ^ 1)) { ok = false; break; }
              ptx::mbar_arrive_expect_tx(&bars->raw_full[rs], nbox * 2 * BOX * HD);
              uint8_t* dr = smem + OFF_RAW + rs * RAW_BYTES;
              for (int h = 0; h < nbox; ++h) {
                const int y = (int)(W.doc_row0 + T.key0 + h * BOX);
                ptx::tma_load_2d(dr + h * BOX * HD, &tmK, &bars->raw_full[rs], 0, y);
                ptx::tma_load_2d(dr + TK * HD + h * BOX * HD, &tmV, &bars->raw_full[rs], 0, y);
              }
              last_raw[rs] = (int)((dc / NRAW) & 1);
              pend_cvt[s] = (int)n_cvt[s]++;
              ++dc;
              continue;
            }
          }
          uint8_t* dk = smem + OFF_K + s * TK * 128;
          uint8_t* dv = smem + OFF_V + s * TK * 128;
          const int64_t y0 = (T.prompt ? W.prompt_row0 : W.doc_row0) + T.key0;
          const int x0 = T.prompt ? W.g * HD : 0;
          const CUtensorMap* mk = T.prompt ? &tmKp : &tmK;
          const CUtensorMap* mv = T.prompt ? &tmVp : &tmV;
          if (!ptx::mbar_wait(&bars->k_empty[s], (u & 1) ^ 1)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&bars->k_full[s], nbox * BOX * 128);
          for (int h = 0; h < nbox; ++h)
            ptx::tma_load_2d(dk + h * BOX * 128, mk, &bars->k_full[s], x0, (int)(y0 + h * BOX));
          if (!ptx::mbar_wait(&bars->v_empty[s], (u & 1) ^ 1)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&bars->v_full[s], nbox * BOX * 128);
          for (int h = 0; h < nbox; ++h)
            ptx::tma_load_2d(dv + h * BOX * 128, mv, &bars->v_full[s], x0, (int)(y0 + h * BOX));
          last_kv[s] = (int)(n_tma[s] & 1);
          ++n_tma[s];
        }
      }
      // let every load this CTA issued land before it can exit
      for (int s = 0; s < NKV; ++s)
        if (last_kv[s] >= 0 && (!ptx::mbar_wait(&bars->k_full[s], (uint32_t)last_kv[s], 100000000LL) ||
                                !ptx::mbar_wait(&bars->v_full[s], (uint32_t)last_kv[s], 100000000LL)))
          ok = false;
      for (int s = 0; s < NRAW; ++s)
        if (last_raw[s] >= 0 && !ptx::mbar_wait(&bars->raw_full[s], (uint32_t)last_raw[s], 100000000LL))
          ok = false;
      for (int s = 0; s < 2; ++s)
        if (last_q[s] >= 0 && !ptx::mbar_wait(&bars->q_full[s], (uint32_t)last_q[s], 100000000LL))
          ok = false;
      if (!ok) atomicExch(status, ST_ETIMEOUT);
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issue
    // Two cursors walk the CTA's (item, tile) sequence: the S cursor issues
    // S = Q K^T of tile cs, the P.V cursor issues P.V of tile cp (cp <= cs).
    // Each step issues whichever is ready, tested without blocking, so that a
    // late K of the next tile never holds back the P.V of the current one.
    if (lane == 0) {
      constexpr uint32_t idPV =
          (FP8 ? ptx::idesc_f16_f32(ROWS, HD) : ptx::idesc_bf16_f32(ROWS, HD)) | (1u << 16);
      bool ok = true;
      uint32_t n_tma[NKV] = {}, n_cvt[NKV] = {};   // fills of each stage by kind (parities)
      uint32_t cs = 0, cp = 0;                     // tiles whose S / P.V has been issued
      // parity of each issued-S tile's K/V fill, read by its P.V: the S cursor
      // runs up to NB + 1 tiles ahead, so with fewer stages than that a later
      // fill of the same stage may already be counted when the P.V is checked
      uint32_t vpar = 0;                           // bit (tile & 7)
      int sw = blockIdx.x, sti = 0;                // S cursor: work item, tile
      uint32_t sq = 0;                             //   and its item counter
      bool s_have = false;                         //   its item's slot and Q have landed
      int pw = blockIdx.x, pti = 0;                // P.V cursor
      uint32_t pq = 0;
      long long t_last = clock64();
      while (pw < n_work) {
        bool progressed = false;
        // ---- S of tile cs (the single S buffer: at most one S ahead of the P.V)
        if (sw < n_work && cs <= cp + (uint32_t)NB) {
          const int qb = sq & 1;
          if (!s_have) s_have = ptx::mbar_test(&bars->q_full[qb], (sq >> 1) & 1);
          if (s_have) {
            const Work<MODE, TK>& W = slots[qb];
            const int s = cs % NKV, b = cs % NB;
            const TileInfo T = W.tile(sti);
            const bool widened = FP8 && !T.prompt;
            uint64_t* fb = widened ? &bars->kc_full[s] : &bars->k_full[s];
            uint32_t& nuse = widened ? n_cvt[s] : n_tma[s];
            if (ptx::mbar_test(fb, nuse & 1) && ptx::mbar_test(&bars->s_free[b], ((cs / NB) & 1) ^ 1)) {
              vpar = (vpar & ~(1u << (cs & 7))) | ((nuse & 1u) << (cs & 7));
              ++nuse;
              ptx::tc_fence_after();
              // E4M3 KV runs the products in f16 (codes widen exactly; scales act in f32)
              const int n = ((T.kc + 31) >> 5) * 32;
              const uint32_t idS = FP8 ? ptx::idesc_f16_f32(ROWS, n) : ptx::idesc_bf16_f32(ROWS, n);
              const uint32_t sQ = sQ0 + qb * ROWS * 128, kb = sK0 + s * TK * 128;
#pragma unroll
              for (int k = 0; k < HD / 16; ++k)
                ptx::mma_f16(tmem + b * TK, ptx::desc_kmajor_sw128(sQ + k * 32),
                             ptx::desc_kmajor_sw128(kb + k * 32), idS, k > 0);
              ptx::mma_commit(&bars->s_full[b]);
              ptx::mma_commit(&bars->k_empty[s]);
              ++cs;
              if (++sti == W.n_tiles) {
                sti = 0;
                sw += gridDim.x;
                ++sq;
                s_have = false;
              }
              progressed = true;
            }
          }
        }
        // ---- P.V of tile cp
        if (cp < cs) {
          const int qb = pq & 1, ob = pq % NB;
          const Work<MODE, TK>& W = slots[qb];
          const int b = cp % NB, s = cp % NKV;
          const TileInfo T = W.tile(pti);
          const bool tma_v = !FP8 || T.prompt;
          // the tile's V is in its stage once the fill recorded at its S issue lands
          const uint32_t vp = (vpar >> (cp & 7)) & 1u;   // this tile's V fill
          if ((tma_v ? ptx::mbar_test(&bars->v_full[s], vp) : ptx::mbar_test(&bars->vc_full[s], vp)) &&
              ptx::mbar_test(&bars->p_full[b], (cp / NB) & 1) &&
              (pti != 0 || ptx::mbar_test(&bars->o_free[ob], ((pq / NB) & 1) ^ 1))) {
            ptx::tc_fence_after();
            const int ksteps = ((T.kc + 31) >> 5) * 2;
            const uint32_t vb = sV0 + s * TK * 128;
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk)
              if (kk < ksteps)
                ptx::mma_f16_ta(tmem + COL_O + ob * HD, tmem + COL_P + b * HD + kk * 8,
                                desc_mnmajor_sw128(vb + kk * 2048), idPV, (pti | kk) > 0);
            ptx::mma_commit(&bars->pv_done[b]);
            ptx::mma_commit(&bars->v_empty[s]);
            ++cp;
            if (++pti == W.n_tiles) {
              // the item's last MMA: its Q buffer and decoded slot (which both
              // cursors read) may be refilled once it completes
              ptx::mma_commit(&bars->q_empty[qb]);
              pti = 0;
              pw += gridDim.x;
              ++pq;
            }
            progressed = true;
          }
        }
        if (progressed) {
          t_last = clock64();
        } else if (clock64() - t_last > 4000000000LL) {
          ok = false;
          break;
        }
      }
      if (!ok) atomicExch(status, ST_ETIMEOUT);
      // every commit of this thread has landed once the last stages are released
      if (ok)
        for (uint32_t cc = cp >= NKV ? cp - NKV : 0; cc < cp; ++cc)
          if (!ptx::mbar_wait(&bars->v_empty[cc % NKV], (cc / NKV) & 1, 100000000LL))
            atomicExch(status, ST_ETIMEOUT);
    }
    __syncwarp();
  } else if (FP8 && warp >= 6) {
    // ------------------------------------------------------------ widen E4M3 -> f16
    // Warp 6 widens the K codes of each document tile, warp 7 the V codes, into
    // the swizzled MMA stage (the block scales act later, in f32); lane l takes
    // rows l, l + 32, ...  K is widened once the stage's previous S has read it,
    // V once the previous P.V has, so the next S does not wait for a P.V.
    const int half = warp - 6;   // 0: K, 1: V
    uint64_t* const empty = half == 0 ? bars->k_empty : bars->v_empty;
    uint64_t* const full = half == 0 ? bars->kc_full : bars->vc_full;
    uint8_t* const dst0 = smem + (half == 0 ? OFF_K : OFF_V);
    // a row's four 16-byte code chunks in a lane-dependent order: lane l visits
    // chunk perm[(l >> 1) & 3] ^ j at step j, perm = (0, 2, 3, 1).  Within each
    // group of 8 lanes (8 consecutive rows: code rows 64 B apart, f16 rows 128 B
    // apart under the 128-byte swizzle) that makes the 16-byte code loads and
    // both 16-byte f16 stores of every step hit 8 distinct bank quads, i.e.
    // conflict-free (a plain rotation (j + (l >> 1)) & 3 keeps the loads
    // conflict-free but the swizzle folds the stores onto two quads).
    const int rot = (0x1320 >> (4 * ((lane >> 1) & 3))) & 3;
    bool ok = true;
    uint32_t c = 0, dc = 0, qc = 0;
    for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x, ++qc) {
      const int qb = qc & 1;
      if (!ptx::mbar_wait(&bars->q_full[qb], (qc >> 1) & 1)) { ok = false; break; }
      const Work<MODE, TK> W = slots[qb];
      ptx::mbar_arrive(&bars->q_empty[qb]);
      for (int ti = 0; ti < W.n_tiles; ++ti, ++c) {
        const TileInfo T = W.tile(ti);
        if (T.prompt) continue;
        const int s = c % NKV, rs = dc % NRAW;
        if (!ptx::mbar_wait(&bars->raw_full[rs], (dc / NRAW) & 1)) { ok = false; break; }
        if (!ptx::mbar_wait(&empty[s], ((c / NKV) & 1) ^ 1)) { ok = false; break; }
        const uint8_t* raw = smem + OFF_RAW + rs * RAW_BYTES + half * TK * HD;
        uint8_t* dst = dst0 + s * TK * 128;
#pragma unroll
        for (int i = 0; i < TK / 32; ++i) {
          const int row = lane + 32 * i;
          if (row >= T.count) {
            // past the tuple's retained slots: exact zeros (their codes were
            // not loaded, and their block scale may not exist)
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)
              *reinterpret_cast<uint4*>(dst + swz(row, ch)) = make_uint4(0, 0, 0, 0);
            continue;
          }
          const uint4* src = reinterpret_cast<const uint4*>(raw + row * HD);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int q16 = rot ^ j;
            const uint4 cw = src[q16];
            const uint32_t words[4] = {cw.x, cw.y, cw.z, cw.w};
            uint32_t out[8];
#pragma unroll
            for (int wd = 0; wd < 4; ++wd) {
#pragma unroll
              for (int hw = 0; hw < 2; ++hw) {
                const uint16_t pair = (uint16_t)(words[wd] >> (16 * hw));
                asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(out[2 * wd + hw]) : "h"(pair));
              }
            }
            // 16 codes -> 32 bytes of f16 = chunks 2*q16, 2*q16+1 of the row
            *reinterpret_cast<uint4*>(dst + swz(row, 2 * q16)) = make_uint4(out[0], out[1], out[2], out[3]);
            *reinterpret_cast<uint4*>(dst + swz(row, 2 * q16 + 1)) = make_uint4(out[4], out[5], out[6], out[7]);
          }
        }
        fence_proxy_async();
        ptx::mbar_arrive(&bars->raw_empty[rs]);
        ptx::mbar_arrive(&full[s]);
        ++dc;
      }
    }
    if (!ok) atomicExch(status, ST_ETIMEOUT);
  } else if (warp < 4) {
    // ------------------------------------------------------------ softmax warps
    const int r = threadIdx.x;                 // query row == TMEM lane
    const float sl2 = a.scale * 1.4426950408889634f;
    const uint32_t lane_base = (uint32_t)((warp * 32) << 16);
    __half* og = reinterpret_cast<__half*>(a.o);   // O feeds the half-operand O projection
    bool ok = true;
    uint32_t c = 0, qc = 0;
    // With two O buffers an item's O is read out after the next item's first
    // tile, by when its last P.V has long completed; with one, at its end.
    // O buffer ob of the item whose last tile was cl: wait for its last P.V,
    // release the buffer, write the row normalised by l (orow < 0: no row)
    // (split-KV piece: pidx >= 0 is the row's partial-result index; the
    // unnormalised O, the running max m and the row sum l go there instead)
    auto read_out = [&](int ob, uint32_t cl, float l, int64_t orow, int64_t pidx, float mrow) -> bool {
      if (!ptx::mbar_wait(&bars->pv_done[cl % NB], (cl / NB) & 1)) return false;
      ptx::tc_fence_after();
      const uint32_t o_addr = tmem + lane_base + COL_O + ob * HD;
      const float inv = l > 0.f ? 1.f / l : 0.f;
      uint4* dst = reinterpret_cast<uint4*>(og + (orow >= 0 ? orow : 0) * HD);
      // two 32-column halves (the buffer is released once both are loaded)
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        uint32_t o0[32];
        ST_TMEM_LD32(o_addr + 32 * h, o0);
        ptx::tmem_wait_ld();
        ST_TMEM_TIE32(o0);
        if (h == 1) {
          ptx::tc_fence_before();
          ptx::mbar_arrive(&bars->o_free[ob]);
        }
        if (MODE == 1 && pidx >= 0) {
          float* pr = a.part + pidx * SPLIT_STRIDE;
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<uint4*>(pr + 32 * h + e) = make_uint4(o0[e], o0[e + 1], o0[e + 2], o0[e + 3]);
          if (h == 1) *reinterpret_cast<float2*>(pr + 64) = make_float2(mrow, l);
        } else if (orow >= 0) {
#pragma unroll
          for (int e = 0; e < 32; e += 8)
            dst[4 * h + e / 8] =
                make_uint4(pack_f16(__uint_as_float(o0[e]) * inv, __uint_as_float(o0[e + 1]) * inv),
                           pack_f16(__uint_as_float(o0[e + 2]) * inv, __uint_as_float(o0[e + 3]) * inv),
                           pack_f16(__uint_as_float(o0[e + 4]) * inv, __uint_as_float(o0[e + 5]) * inv),
                           pack_f16(__uint_as_float(o0[e + 6]) * inv, __uint_as_float(o0[e + 7]) * inv));
        }
      }
      return true;
    };
    bool pend_on = false;           // (two O buffers) the item read out after the next one's first tile
    int pend_ob = 0;
    uint32_t pend_cl = 0;
    float pend_l = 0.f;
    int64_t pend_orow = -1, pend_pidx = -1;
    float pend_m = 0.f;
    for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x, ++qc) {
      const int qb = qc & 1;
      if (!ptx::mbar_wait(&bars->q_full[qb], (qc >> 1) & 1)) { ok = false; break; }
      // read in place; the slot is released at the item's end
      const Work<MODE, TK>& W = slots[qb];
      const int pos = (W.row_base + r) / W.G;

      // O accumulates in TMEM (buffer qb); the running max m only moves when a
      // row's tile maximum exceeds it by more than 8 (a factor 256 in P), and
      // then the row's O is rescaled in place before the next P.V is issued.
      float m = -INFINITY, l = 0.f;
      const int ob = qc % NB;
      const uint32_t o_addr = tmem + lane_base + COL_O + ob * HD;
      const int lim = MODE == 0 ? W.j0 + pos : W.qoff + pos;   // causal limit of this row
      for (int ti = 0; ti < W.n_tiles; ++ti, ++c) {
        const int b = c % NB;
        const TileInfo T = W.tile(ti);
        const int nch = (T.kc + 31) >> 5;           // 32-key chunks any row can see
        const bool causal = (MODE == 0) || T.prompt;
        // E4M3 document tiles: one K and one V scale per 64-slot half of the
        // tile, loaded before the wait for S so that their latency overlaps it
        float ks[NHALF], vs[NHALF];
#pragma unroll
        for (int hf = 0; hf < NHALF; ++hf) ks[hf] = vs[hf] = 1.f;
        if (FP8 && !T.prompt) {
          const float* scp = a.scales + ((W.doc_row0 + T.key0) >> 6) * 2;
          ks[0] = scp[0];
          vs[0] = scp[1];
          if (NHALF > 1 && T.count > 64) {
            ks[NHALF - 1] = scp[2];
            vs[NHALF - 1] = scp[3];
          }
        }
        if (!ptx::mbar_wait(&bars->s_full[b], (c / NB) & 1)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t sb = tmem + lane_base + b * TK;
        int nvis = T.count;                          // visible keys of this row in the tile
        if (causal) nvis = min(nvis, lim - T.key0 + 1);
        // The row's visible chunks of S into registers, CPP chunks per pass with
        // one wait, their invisible keys (ragged tail, causal limit) as -inf.
        // With one pass (VW = TK) the TMEM buffer is released at once; with two
        // (E4M3 128-key tiles, whose register budget holds 64 scores) pass 1
        // takes the row maximum and pass 2 reads each half again for the
        // exponentials, releasing the buffer after its last read.
        uint32_t v[VW];
        auto load_pass = [&](int c0) {
#pragma unroll
          for (int q = 0; q < CPP; ++q)
            if (q == 0 || c0 + q < nch) ST_TMEM_LD32(sb + 32 * (c0 + q), (v + 32 * q));
          ptx::tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < CPP; ++q) ST_TMEM_TIE32((v + 32 * q));
#pragma unroll
          for (int q = 0; q < CPP; ++q) {
            const int lo = nvis - 32 * (c0 + q);    // visible keys of this chunk
            if (c0 + q < nch && lo < 32) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (jj >= lo) v[32 * q + jj] = 0xFF800000u;
            }
          }
        };
        auto release_s = [&]() {
          ptx::tc_fence_before();
          ptx::mbar_arrive(&bars->s_free[b]);
        };
        // row maximum of the scaled scores (a positive scale commutes with the max)
        float cm[4];
        if constexpr (NPASS == 1) {
          // every visible chunk with one wait, then the buffer is released
          ST_TMEM_LD32(sb, v);
          if (NCH > 1 && nch > 1) ST_TMEM_LD32(sb + 32, (v + (NCH > 1 ? 32 : 0)));
          if (NCH > 2 && nch > 2) ST_TMEM_LD32(sb + 64, (v + (NCH > 2 ? 64 : 0)));
          if (NCH > 3 && nch > 3) ST_TMEM_LD32(sb + 96, (v + (NCH > 3 ? 96 : 0)));
          ptx::tmem_wait_ld();
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) ST_TMEM_TIE32((v + 32 * ch));
          release_s();
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            const int lo = nvis - 32 * ch;    // visible keys of this chunk
            if (ch < nch && lo < 32) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (jj >= lo) v[32 * ch + jj] = 0xFF800000u;
            }
          }
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            cm[ch] = (ch < NCH && ch < nch) ? chunk_max(v + 32 * (ch < NCH ? ch : 0)) * ks[(ch < NCH ? ch : 0) >> 1]
                                            : -INFINITY;
        } else {
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) cm[ch] = -INFINITY;
#pragma unroll
          for (int p = 0; p < NPASS; ++p) {
            if (p * CPP < nch) {
              load_pass(p * CPP);
#pragma unroll
              for (int q = 0; q < CPP; ++q) {
                const int ch = p * CPP + q;
                if (ch < nch) cm[ch < 4 ? ch : 0] = chunk_max(v + 32 * q) * ks[ch >> 1];
              }
            }
          }
        }
        const float mx = max3(cm[0], cm[1], fmaxf(cm[2], cm[3])) * sl2;
        const bool need = mx > m + 8.f;
        if (__any_sync(0xffffffffu, need)) {
          const float mn = need ? mx : m;
          const float alpha = need ? ex2(m - mn) : 1.f;
          if (ti > 0) {
            // O holds this item's earlier P.V products: scale the row in place
            if (!ptx::mbar_wait(&bars->pv_done[(c - 1) % NB], ((c - 1) / NB) & 1)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint64_t a2 = f2pack(alpha, alpha);
#pragma unroll 1
            for (int part = 0; part < 4; ++part) {
              uint32_t o0[16];
              ST_TMEM_LD16(o_addr + 16 * part, o0);
              ptx::tmem_wait_ld();
              ST_TMEM_TIE16(o0);
#pragma unroll
              for (int e = 0; e < 16; e += 2) {
                const uint64_t x = mul2((uint64_t)o0[e] | ((uint64_t)o0[e + 1] << 32), a2);
                o0[e] = (uint32_t)x;
                o0[e + 1] = (uint32_t)(x >> 32);
              }
              ST_TMEM_ST16(o_addr + 16 * part, o0);
            }
            ptx::tmem_wait_st();
          }
          l *= alpha;
          m = mn;
        }
        const float base = m == -INFINITY ? 0.f : m;
        // the P buffer b was last read by the P.V of tile c - NB
        if (c >= (uint32_t)NB && !ptx::mbar_wait(&bars->pv_done[b], ((c - NB) / NB) & 1)) { ok = false; break; }
        ptx::tc_fence_after();
        // probabilities of the visible chunks, packed in pairs (key 2j low, 2j+1
        // high), 16 TMEM columns per 32-key chunk
        const uint32_t pcol = tmem + lane_base + COL_P + b * HD;
        // p = 2^(s * mul - base), two keys per packed FP32 operation
        const uint64_t nb2 = f2pack(-base, -base);
        uint64_t rs2[2] = {0, 0};           // packed partial row sums (+0.0f lanes)
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          if constexpr (NPASS > 1) {
            if (ch % CPP == 0 && ch < nch) {
              // pass 2: this half of the row again; S is released after its last read
              load_pass(ch);
              if (ch + CPP >= nch) release_s();
            }
          }
          if (ch < nch) {
            const float mul = sl2 * ks[ch >> 1];
            const uint64_t m2 = f2pack(mul, mul), vs2 = f2pack(vs[ch >> 1], vs[ch >> 1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              uint32_t pk[8];
#pragma unroll
              for (int k = 0; k < 16; k += 2) {
                const int kk = 32 * (ch % CPP) + 16 * h + k;
                const uint64_t y = fma2((uint64_t)v[kk] | ((uint64_t)v[kk + 1] << 32), m2, nb2);
                const uint64_t p = f2pack(ex2(f2lo(y)), ex2(f2hi(y)));
                rs2[(k >> 1) & 1] = add2(rs2[(k >> 1) & 1], p);
                if (FP8) {
                  const uint64_t q = mul2(p, vs2);
                  pk[k >> 1] = pack_f16(f2lo(q), f2hi(q));
                } else {
                  pk[k >> 1] = pack_bf16(f2lo(p), f2hi(p));
                }
              }
              ST_TMEM_ST8(pcol + 16 * ch + 8 * h, pk);
            }
          }
        }
        {
          const uint64_t t = add2(rs2[0], rs2[1]);
          l += f2lo(t) + f2hi(t);
        }
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        ptx::mbar_arrive(&bars->p_full[b]);
        if (NB == 2 && ti == 0 && pend_on &&
            !(ok = read_out(pend_ob, pend_cl, pend_l, pend_orow, pend_pidx, pend_m)))
          break;
      }
      if (!ok) break;
      // the output row of this thread (-1: past the item's rows), or for a
      // piece of a split pair its partial-result row
      int64_t orow = -1, pidx = -1;
      {
        const int rr = W.row_base + r, hh = rr % W.G;
        const bool row_ok = r < W.rows && (MODE == 1 || (W.j0 + pos) < W.L);
        if (row_ok) {
          if (MODE == 1 && W.pieces > 1) pidx = ((int64_t)W.pslot * a.hkv + W.g) * ROWS + r;
          else if (MODE == 1) orow = (W.qbase + pos) * a.hq + (int64_t)W.g * W.G + hh;
          else orow = (a.off[W.t] - a.r0 + W.j0 + pos) * a.hq + (int64_t)W.g * W.G + hh;
        }
      }
      ptx::mbar_arrive(&bars->q_empty[qb]);
      if (NB == 1) {
        // a single O buffer is read out at once
        if (!(ok = read_out(ob, c - 1, l, orow, pidx, m))) break;
      } else {
        pend_on = true;
        pend_ob = ob;
        pend_cl = c - 1;
        pend_l = l;
        pend_orow = orow;
        pend_pidx = pidx;
        pend_m = m;
      }
    }
    if (ok && pend_on) ok = read_out(pend_ob, pend_cl, pend_l, pend_orow, pend_pidx, pend_m);
    if (!ok) atomicExch(status, ST_ETIMEOUT);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
}


bool map2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_outer,
           CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)HD, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool map_q(CUtensorMap* m, const void* q, int hq, uint64_t rows, int G,
           CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
            cudaSuccess ||
        qr != cudaDriverEntryPointSuccess)
      return false;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  // q [rows][hq][64] bf16 viewed as (dim, head, row); a box is 128/G rows x G heads x 64 dims,
  // i.e. 128 smem lines ordered (row, head of the group).
  cuuint64_t dims[3] = {(cuuint64_t)HD, (cuuint64_t)hq, rows};
  cuuint64_t strides[2] = {(cuuint64_t)HD * 2, (cuuint64_t)hq * HD * 2};
  cuuint32_t box[3] = {(cuuint32_t)HD, (cuuint32_t)G, (cuuint32_t)(ROWS / G)};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void*>(q), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

bool map2d_u8(CUtensorMap* m, const void* base, uint64_t outer, uint32_t box_outer) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  cuuint64_t dims[2] = {(cuuint64_t)HD, outer};
  cuuint64_t strides[1] = {(cuuint64_t)HD};
  cuuint32_t box[2] = {(cuuint32_t)HD, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, bool FP8, int NB, int TK>
void set_smem_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_attn_tc<MODE, FP8, NB, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_bytes(FP8, NB, TK));
    done = true;
  }
}

template <int MODE, bool FP8, int NB, int TK>
void launch_attn(const AttnParams& a, const int32_t* items, int n_work, int zb, const CUtensorMap& mq,
                 const CUtensorMap& mk, const CUtensorMap& mv, const CUtensorMap& mkp, const CUtensorMap& mvp,
                 int* status, cudaStream_t s) {
  set_smem_attr<MODE, FP8, NB, TK>();
  const int slots = sm_count() * ctas_per_sm(NB);
  const int grid = n_work < slots ? n_work : slots;
  k_attn_tc<MODE, FP8, NB, TK><<<grid, nthreads(FP8), smem_bytes(FP8, NB, TK), s>>>(a, items, n_work, zb, mq, mk,
                                                                                  mv, mkp, mvp, status);
}

}  // namespace

bool attn_tc_supported(int hq, int hkv, int hd) {
  const int G = hq / hkv;
  return hd == HD && G >= 1 && G <= ROWS && ROWS % G == 0;
}

int attn_tc_eval(const AttnParams& a, int* status, cudaStream_t s) {
  if (a.n_work <= 0) return ST_OK;
  if (!attn_tc_supported(a.hq, a.hkv, a.hd) || (a.kv_dtype != ST_BF16 && a.kv_dtype != ST_E4M3))
    return ST_EUNSUPPORTED;
  const bool fp8 = a.kv_dtype == ST_E4M3;
  const int G = a.hq / a.hkv;
  CUtensorMap mq, mk, mv, mkp, mvp;
  const uint64_t planes = (uint64_t)a.hkv * a.Rp_cap;
  const uint64_t prow = (uint64_t)(a.kvrows > 0 ? a.kvrows : a.qrows);
  const CUtensorMapDataType qt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  bool ok = map_q(&mq, a.q, a.hq, (uint64_t)a.qrows, G, qt) &&
            map2d(&mkp, a.kp, (uint64_t)a.hkv * HD, prow, BOX, qt) &&
            map2d(&mvp, a.vp, (uint64_t)a.hkv * HD, prow, BOX, qt);
  if (fp8) ok = ok && map2d_u8(&mk, a.Kr, planes, BOX) && map2d_u8(&mv, a.Vr, planes, BOX);
  else ok = ok && map2d(&mk, a.Kr, HD, planes, BOX) && map2d(&mv, a.Vr, HD, planes, BOX);
  if (!ok) return ST_ECUDA;
  const int n_work = a.n_work * a.hkv;
  const int zb = 1;   // unused in eval (the work list carries the row block)
  // layout by a.nb (0 or 1: two CTAs per SM with single buffers, 2: one CTA with
  // double buffers, 3: E4M3 single buffers with 128-key tiles)
  if (fp8 && a.nb == 2)
    launch_attn<1, true, 2, 128>(a, a.work, n_work, zb, mq, mk, mv, mkp, mvp, status, s);
  else if (fp8 && a.nb == 3)
    launch_attn<1, true, 1, 128>(a, a.work, n_work, zb, mq, mk, mv, mkp, mvp, status, s);
  else if (fp8)
    launch_attn<1, true, 1, 64>(a, a.work, n_work, zb, mq, mk, mv, mkp, mvp, status, s);
  else if (a.nb == 2)
    launch_attn<1, false, 2, 128>(a, a.work, n_work, zb, mq, mk, mv, mkp, mvp, status, s);
  else
    launch_attn<1, false, 1, 128>(a, a.work, n_work, zb, mq, mk, mv, mkp, mvp, status, s);
  return ST_OK;
}

int attn_tc_prefill(const AttnParams& a, const int32_t* items, int n_items, int* status,
                    cudaStream_t s) {
  if (n_items <= 0) return ST_OK;
  if (!attn_tc_supported(a.hq, a.hkv, a.hd)) return ST_EUNSUPPORTED;
  const int G = a.hq / a.hkv;
  CUtensorMap mq, mk, mv;
  const uint64_t planes = (uint64_t)a.hkv * a.R;
  if (!map_q(&mq, a.q, a.hq, (uint64_t)a.rows, G) || !map2d(&mk, a.K, HD, planes, BOX) ||
      !map2d(&mv, a.V, HD, planes, BOX))
    return ST_ECUDA;
  launch_attn<0, false, 1, 128>(a, items, n_items * a.hkv, 1, mq, mk, mv, mk, mv, status, s);
  return ST_OK;
}

}  // namespace st
