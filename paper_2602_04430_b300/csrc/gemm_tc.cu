// BF16 projection GEMM on the 5th-generation tensor cores (tcgen05) for sm_103a.
//
//   C[M][N] = A[M][K] . W[N][K]^T,  A / W bf16 row-major (K-major), f32 accumulate.
//
// Persistent kernel, one CTA per SM (192 KB of shared memory), 128 x 256 output
// tiles with the N index fastest so that CTAs of one wave share the A row block
// through L2.  Warp roles:
//   warp 0      TMA producer: 4-stage ring of (A 128x64, W 256x64) bf16 tiles,
//               128-byte swizzle, mbarrier transaction counts.
//   warp 1      TMEM allocator (512 columns = two 128x256 f32 accumulators) and,
//               on one lane, the tcgen05.mma issuer (M=128, N=256, K=16 steps).
//   warps 2-9   epilogue: tcgen05.ld of the accumulator rows (warp w reads TMEM
//               lanes 32*(w%4) .., warps w and w+4 split the tile's columns),
//               fused epilogue (RoPE + Q/K/V scatter, residual add, SwiGLU).
//               A thread holds one row; each warp turns its 32 rows around in
//               a 4 KB shared-memory buffer so that global loads and stores
//               move whole 128-byte row segments (coalesced).
// The two accumulators let the epilogue of tile i overlap the main loop of
// tile i+1.  Every mbarrier wait is bounded; a timeout sets the status word.
//
// Launches of more than 128 rows run the CTA-pair variant k_gemm_tc2 (2-SM
// MMA on 256 x 256 tiles, described at its definition); k_gemm_tc serves
// the small launches (and st_set_gemm_pairs(0)).
#include <cudaTypedefs.h>

#include "epilogue.cuh"
#include "ptx.cuh"

namespace st {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_THREADS = 320;   // producer, MMA, 8 epilogue warps
constexpr uint32_t TMEM_COLS = 512;
constexpr int STG_BYTES = 4096;     // per epilogue warp: 32 rows x 128 B
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 8 * STG_BYTES + 1024 + 256;

struct Bars {
  uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
  uint32_t tmem_base;
};

// Staging layouts (16-byte chunk j of row r), conflict-free for both the
// row-per-thread side and the row-segment-per-8-threads side.
__device__ __forceinline__ uint32_t sw128(int r, int j) {
  return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4));
}
__device__ __forceinline__ uint32_t sw64(int r, int j) {
  return (uint32_t)(r * 64 + ((j ^ ((r >> 1) & 3)) << 4));
}
// 32 rows x 128 B (or 64 B) from the staging buffer to dst + r * stride; rows
// r >= nrows are past the matrix and skipped.
__device__ __forceinline__ void copy_out128(const uint8_t* st, char* dst, int64_t stride, int nrows,
                                            int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (lane >> 3) + 4 * i, j = lane & 7;
    if (r < nrows)
      *reinterpret_cast<uint4*>(dst + r * stride + j * 16) = *reinterpret_cast<const uint4*>(st + sw128(r, j));
  }
}
__device__ __forceinline__ void copy_out64(const uint8_t* st, char* dst, int64_t stride, int nrows,
                                           int lane) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = (lane >> 2) + 8 * i, j = lane & 3;
    if (r < nrows)
      *reinterpret_cast<uint4*>(dst + r * stride + j * 16) = *reinterpret_cast<const uint4*>(st + sw64(r, j));
  }
}
template <bool F16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if (F16) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// One head (64 columns) of the QKV projection for the warp's 32 rows: RoPE on
// Q and K columns, then the 16-bit head row to Q or to the K / V cache planes.
template <bool F16>
__device__ __forceinline__ void epi_qkv_head(const EpiParams& ep, uint8_t* st, float (&v)[64], int row,
                                             int row0, int nrows, int col0, int lane, int M) {
  const int qcols = ep.hq * 64, kcols = ep.hkv * 64;
  if (col0 < qcols + kcols) {
    const int pos = row < M ? ep.pos[row] : 0;
    const float2* tab = ep.rope_t + pos;
    // eight frequencies per group: bounds the table loads in flight (registers)
#pragma unroll
    for (int i0 = 0; i0 < 32; i0 += 8) {
      float2 cs[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) cs[i] = tab[(int64_t)(i0 + i) * ep.rope_np];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float a = v[i0 + i], b = v[i0 + i + 32];
        v[i0 + i] = a * cs[i].x - b * cs[i].y;
        v[i0 + i + 32] = b * cs[i].x + a * cs[i].y;
      }
      asm volatile("" ::: "memory");
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    *reinterpret_cast<uint4*>(st + sw128(lane, j)) =
        make_uint4(pack2<F16>(v[8 * j], v[8 * j + 1]), pack2<F16>(v[8 * j + 2], v[8 * j + 3]),
                   pack2<F16>(v[8 * j + 4], v[8 * j + 5]), pack2<F16>(v[8 * j + 6], v[8 * j + 7]));
  __syncwarp();
  char* dst;
  int64_t stride;
  if (col0 < qcols) {
    dst = reinterpret_cast<char*>(ep.q) + ((int64_t)row0 * qcols + col0) * 2;
    stride = (int64_t)qcols * 2;
  } else {
    const bool isk = col0 < qcols + kcols;
    const int head = (col0 - qcols - (isk ? 0 : kcols)) / 64;
    dst = reinterpret_cast<char*>(isk ? ep.kbase : ep.vbase) +
          ((int64_t)head * ep.kv_sg + (int64_t)row0 * ep.kv_sr) * 2;
    stride = ep.kv_sr * 2;
  }
  copy_out128(st, dst, stride, nrows, lane);
  __syncwarp();
}

// Columns [half * BN/2, (half + 1) * BN/2) of the tile for the warp's 32 rows
// (SwiGLU: gate columns [half*64, half*64 + 64) with their up columns).
// Residual epilogue: the warp's x rows of 32 columns at col, as the coalesced
// 16-byte pieces this lane moves (row (lane >> 3) + 4 i, piece lane & 7).
__device__ __forceinline__ void resid_load(const EpiParams& ep, uint4 (&pre)[8], int row0, int nrows,
                                           int col, int lane) {
  const int64_t xs = (int64_t)ep.row_mul * ep.ld * 4;
  const char* xc = reinterpret_cast<const char*>(ep.x) +
                   ((int64_t)row0 * ep.row_mul + ep.row_add) * ep.ld * 4 + (int64_t)col * 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int rr = (lane >> 3) + 4 * i, j = lane & 7;
    if (rr < nrows) pre[i] = *reinterpret_cast<const uint4*>(xc + rr * xs + j * 16);
  }
}

// pre: for EPI_RESID, the tile's first x chunk, loaded before the accumulator
// was ready (resid_load at column n0 + half * BN/2).
template <int EPI>
__device__ __forceinline__ void epilogue_tile(const EpiParams& ep, uint8_t* st, int row0, int n0,
                                              uint32_t taddr, int M, int half, int lane,
                                              uint4 (&pre)[8]) {
  const int row = row0 + lane;
  const int nrows = M - row0 < 32 ? M - row0 : 32;
  const float inv = row < M ? row_inv_rms(ep, row) : 1.f;
  if (EPI == EPI_SWIGLU) {
    // columns [0,128) are gate, [128,256) the matching up projections
#pragma unroll 1
    for (int j = half * (BN / 4); j < (half + 1) * (BN / 4); j += 32) {
      uint32_t g[32], u[32];
      ST_TMEM_LD32(taddr + j, g);
      ST_TMEM_LD32(taddr + BN / 2 + j, u);
      ptx::tmem_wait_ld();
      ST_TMEM_TIE32(g);
      ST_TMEM_TIE32(u);
      float hv[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) hv[e] = silu_f(__uint_as_float(g[e]) * inv) * (__uint_as_float(u[e]) * inv);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(st + sw64(lane, q)) =
            ep.act_f16
                ? make_uint4(pack2<true>(hv[8 * q], hv[8 * q + 1]), pack2<true>(hv[8 * q + 2], hv[8 * q + 3]),
                             pack2<true>(hv[8 * q + 4], hv[8 * q + 5]), pack2<true>(hv[8 * q + 6], hv[8 * q + 7]))
                : make_uint4(pack2<false>(hv[8 * q], hv[8 * q + 1]), pack2<false>(hv[8 * q + 2], hv[8 * q + 3]),
                             pack2<false>(hv[8 * q + 4], hv[8 * q + 5]), pack2<false>(hv[8 * q + 6], hv[8 * q + 7]));
      __syncwarp();
      copy_out64(st, reinterpret_cast<char*>(ep.h) + ((int64_t)row0 * ep.ld + n0 / 2 + j) * 2,
                 ep.ld * 2, nrows, lane);
      __syncwarp();
    }
  } else if (EPI == EPI_QKV) {
#pragma unroll 1
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 64) {
      uint32_t r[64];
      uint32_t* r2 = r + 32;
      ST_TMEM_LD32(taddr + c, r);
      ST_TMEM_LD32(taddr + c + 32, r2);
      ptx::tmem_wait_ld();
      ST_TMEM_TIE32(r);
      ST_TMEM_TIE32(r2);
      float v[64];
#pragma unroll
      for (int e = 0; e < 64; ++e) v[e] = __uint_as_float(r[e]) * inv;
      if (ep.qkv_f16) epi_qkv_head<true>(ep, st, v, row, row0, nrows, n0 + c, lane, M);
      else epi_qkv_head<false>(ep, st, v, row, row0, nrows, n0 + c, lane, M);
    }
  } else if (EPI == EPI_RESID) {
    // x[row*row_mul + row_add] += acc, 32 columns at a time through the
    // staging buffer (coalesced float32 read-modify-write, the next chunk's x
    // loads in flight meanwhile); xb = x rounded to the operand type
    const int64_t xs = (int64_t)ep.row_mul * ep.ld * 4;   // byte stride of the warp's x rows
    char* xrow0 = reinterpret_cast<char*>(ep.x) + ((int64_t)row0 * ep.row_mul + ep.row_add) * ep.ld * 4;
    float ss = 0.f;
#pragma unroll 1
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
      uint32_t r[32];
      ST_TMEM_LD32(taddr + c, r);
      char* xc = xrow0 + (int64_t)(n0 + c) * 4;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rr = (lane >> 3) + 4 * i, j = lane & 7;
        if (rr < nrows) *reinterpret_cast<uint4*>(st + sw128(rr, j)) = pre[i];
      }
      if (c + 32 < (half + 1) * (BN / 2)) resid_load(ep, pre, row0, nrows, n0 + c + 32, lane);
      ptx::tmem_wait_ld();
      ST_TMEM_TIE32(r);
      __syncwarp();
      uint32_t xw[16];   // bf16(x) of the row, packed in pairs
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 o = *reinterpret_cast<const float4*>(st + sw128(lane, j));
        o.x += __uint_as_float(r[4 * j]) * inv;
        o.y += __uint_as_float(r[4 * j + 1]) * inv;
        o.z += __uint_as_float(r[4 * j + 2]) * inv;
        o.w += __uint_as_float(r[4 * j + 3]) * inv;
        xw[2 * j] = ep.act_f16 ? pack2<true>(o.x, o.y) : pack2<false>(o.x, o.y);
        xw[2 * j + 1] = ep.act_f16 ? pack2<true>(o.z, o.w) : pack2<false>(o.z, o.w);
        ss += o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
        *reinterpret_cast<float4*>(st + sw128(lane, j)) = o;
      }
      __syncwarp();
      copy_out128(st, xc, xs, nrows, lane);
      __syncwarp();
      if (ep.xb != nullptr) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(st + sw64(lane, q)) =
              make_uint4(xw[4 * q], xw[4 * q + 1], xw[4 * q + 2], xw[4 * q + 3]);
        __syncwarp();
        copy_out64(st, reinterpret_cast<char*>(ep.xb) + ((int64_t)row0 * ep.N + n0 + c) * 2,
                   (int64_t)ep.N * 2, nrows, lane);
        __syncwarp();
      }
    }
    if (ep.ssq_out != nullptr && row < M)
      ep.ssq_out[(int64_t)row * (ep.N / 128) + (n0 + half * (BN / 2)) / 128] = ss;
  } else {
    // EPI_STORE_F32 (self-test path): straight from the row's registers
#pragma unroll 1
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 64) {
      uint32_t r[64];
      uint32_t* r2 = r + 32;
      ST_TMEM_LD32(taddr + c, r);
      ST_TMEM_LD32(taddr + c + 32, r2);
      ptx::tmem_wait_ld();
      ST_TMEM_TIE32(r);
      ST_TMEM_TIE32(r2);
      if (row < M) {
        float* o = ep.out + (int64_t)row * ep.ld + n0 + c;
#pragma unroll
        for (int e = 0; e < 64; e += 4)
          *reinterpret_cast<float4*>(o + e) = make_float4(__uint_as_float(r[e]), __uint_as_float(r[e + 1]),
                                                          __uint_as_float(r[e + 2]), __uint_as_float(r[e + 3]));
      }
    }
  }
}

// One instantiation per epilogue (the launch's EpiParams::mode).
template <int EPI>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int M, int N, int K, EpiParams ep, int* status, uint32_t idesc) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint8_t* stg = smem + STAGES * STAGE_BYTES;   // 8 epilogue staging buffers
  Bars* bars = reinterpret_cast<Bars*>(stg + 8 * STG_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_blocks = (M + BM - 1) / BM, n_blocks = N / BN;
  const int tiles = m_blocks * n_blocks, nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&bars->full[s], 1);
      ptx::mbar_init(&bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&bars->tfull[b], 1);
      ptx::mbar_init(&bars->tempty[b], 256);
    }
    ptx::fence_mbar_init();
    ptx::tma_prefetch_desc(&tmA);
    ptx::tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    ptx::tmem_alloc(&bars->tmem_base, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last_par[STAGES];
      for (int s = 0; s < STAGES; ++s) last_par[s] = -1;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int mb = tile / n_blocks, nb = tile % n_blocks;
        for (int kb = 0; kb < nk; ++kb) {
          if (!ptx::mbar_wait(&bars->empty[stage], phase ^ 1)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&bars->full[stage], STAGE_BYTES);
          ptx::tma_load_2d(sA + stage * A_BYTES, &tmA, &bars->full[stage], kb * BK, mb * BM);
          ptx::tma_load_2d(sB + stage * B_BYTES, &tmB, &bars->full[stage], kb * BK, nb * BN);
          last_par[stage] = (int)phase;
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      // let every load this CTA issued land before the CTA can exit
      for (int s = 0; s < STAGES; ++s)
        if (last_par[s] >= 0 && !ptx::mbar_wait(&bars->full[s], (uint32_t)last_par[s], 100000000LL))
          ok = false;
      if (!ok) atomicExch(status, ST_ETIMEOUT);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int it = 0;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!ptx::mbar_wait(&bars->tempty[buf], (use & 1) ^ 1)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < nk; ++kb) {
          if (!ptx::mbar_wait(&bars->full[stage], phase)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t a0 = ptx::smem_u32(sA + stage * A_BYTES);
          const uint32_t b0 = ptx::smem_u32(sB + stage * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            ptx::mma_f16(dt, ptx::desc_kmajor_sw128(a0 + k * 32), ptx::desc_kmajor_sw128(b0 + k * 32),
                         idesc, (kb | k) != 0);
          ptx::mma_commit(&bars->empty[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit(&bars->tfull[buf]);
      }
      if (!ok) atomicExch(status, ST_ETIMEOUT);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3;          // TMEM lanes 32*quarter .. (warp % 4 rule)
    const int half = (warp - 2) >> 2;      // which half of the tile's columns
    int it = 0;
    uint4 pre[8];
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int buf = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      if (EPI == EPI_RESID) {
        // the residual rows do not depend on the product: fetch the first
        // chunk while the main loop still runs
        const int r0 = (tile / n_blocks) * BM + quarter * 32;
        resid_load(ep, pre, r0, M - r0 < 32 ? M - r0 : 32, (tile % n_blocks) * BN + half * (BN / 2), lane);
      }
      if (!ptx::mbar_wait(&bars->tfull[buf], use & 1)) {
        atomicExch(status, ST_ETIMEOUT);
        break;
      }
      ptx::tc_fence_after();
      const int mb = tile / n_blocks, nb = tile % n_blocks;
      const int row0 = mb * BM + quarter * 32;
      const uint32_t taddr = tmem + (uint32_t)(buf * BN) + ((uint32_t)(quarter * 32) << 16);
      epilogue_tile<EPI>(ep, stg + (warp - 2) * STG_BYTES, row0, nb * BN, taddr, M, half, lane, pre);
      ptx::tc_fence_before();
      ptx::mbar_arrive(&bars->tempty[buf]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- CTA-pair variant
// A cluster of two CTAs (on two SMs) computes 256 x 256 output tiles with the
// 2-SM MMA (tcgen05.mma.cta_group::2, M = 256): CTA rank r stages rows
// [128 r, 128 r + 128) of the A tile and of the W tile, so each SM moves
// 32 KB per 64-deep stage instead of 48 KB for the same tensor work, and
// holds its 128 accumulator rows in its own TMEM (both CTAs' allocations are
// one collective 512-column allocation).  The leader (rank 0) issues the MMAs;
// both CTAs' TMA loads count their bytes on the leader's full barrier; each
// MMA commit arrives on the stage-empty (or accumulator-full) barrier of both
// CTAs; both CTAs' epilogue warps release an accumulator with a remote arrive
// on the leader's barrier.  Same warp roles and epilogues as k_gemm_tc.
constexpr int P_BM = 256, P_HALF = 128, P_STAGES = 6;
constexpr int P_STAGE_BYTES = 2 * P_HALF * BK * 2;   // A half + W half, 32 KB
constexpr size_t P_SMEM_BYTES = (size_t)P_STAGES * P_STAGE_BYTES + 8 * STG_BYTES + 1024 + 256;
static_assert(P_SMEM_BYTES <= 232448, "CTA-pair GEMM shared memory");

struct PairBars {
  uint64_t full[P_STAGES], empty[P_STAGES], tfull[2], tempty[2];
  uint32_t tmem_base;
};

template <int EPI>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_gemm_tc2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int M, int N, int K, EpiParams ep, int* status, uint32_t idesc) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int HALF_BYTES = P_HALF * BK * 2;
  uint8_t* sA = smem;
  uint8_t* sB = smem + P_STAGES * HALF_BYTES;
  uint8_t* stg = smem + P_STAGES * P_STAGE_BYTES;
  PairBars* bars = reinterpret_cast<PairBars*>(stg + 8 * STG_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  const int m_blocks = (M + P_BM - 1) / P_BM, n_blocks = N / BN;
  const int tiles = m_blocks * n_blocks, nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      ptx::mbar_init(&bars->full[s], 1);
      ptx::mbar_init(&bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&bars->tfull[b], 1);
      ptx::mbar_init(&bars->tempty[b], 16);   // 8 epilogue warps in each CTA
    }
    ptx::fence_mbar_init();
    ptx::tma_prefetch_desc(&tmA);
    ptx::tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    ptx::tmem_alloc2(&bars->tmem_base, TMEM_COLS);
    ptx::tmem_relinquish2();
  }
  ptx::tc_fence_before();
  __syncthreads();
  // both CTAs' barriers are initialised and the pair's TMEM allocated before
  // any remote arrive, load completion or MMA
  ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last_par[P_STAGES];
      for (int s = 0; s < P_STAGES; ++s) last_par[s] = -1;
      bool ok = true;
      for (int tile = cluster; tile < tiles && ok; tile += n_clusters) {
        const int mb = tile / n_blocks, nb = tile % n_blocks;
        for (int kb = 0; kb < nk; ++kb) {
          if (!ptx::mbar_wait(&bars->empty[stage], phase ^ 1)) { ok = false; break; }
          if (rank == 0) ptx::mbar_arrive_expect_tx(&bars->full[stage], 2 * P_STAGE_BYTES);
          const uint32_t full_cl = ptx::mapa(ptx::smem_u32(&bars->full[stage]), 0);
          ptx::tma_load_2d_pair(sA + stage * HALF_BYTES, &tmA, full_cl, kb * BK, mb * P_BM + (int)rank * P_HALF);
          ptx::tma_load_2d_pair(sB + stage * HALF_BYTES, &tmB, full_cl, kb * BK, nb * BN + (int)rank * P_HALF);
          last_par[stage] = (int)phase;
          if (++stage == P_STAGES) { stage = 0; phase ^= 1; }
        }
      }
      // every load this CTA issued has landed once the leader's MMAs that read
      // it have completed (their commit arrives on this CTA's empty barrier)
      for (int s = 0; s < P_STAGES; ++s)
        if (last_par[s] >= 0 && !ptx::mbar_wait(&bars->empty[s], (uint32_t)last_par[s], 100000000LL))
          ok = false;
      if (!ok) atomicExch(status, ST_ETIMEOUT);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int it = 0;
      for (int tile = cluster; tile < tiles && ok; tile += n_clusters, ++it) {
        const int buf = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!ptx::mbar_wait(&bars->tempty[buf], (use & 1) ^ 1)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < nk; ++kb) {
          if (!ptx::mbar_wait(&bars->full[stage], phase)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t a0 = ptx::smem_u32(sA + stage * HALF_BYTES);
          const uint32_t b0 = ptx::smem_u32(sB + stage * HALF_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            ptx::mma_f16_pair(dt, ptx::desc_kmajor_sw128(a0 + k * 32), ptx::desc_kmajor_sw128(b0 + k * 32),
                              idesc, (kb | k) != 0);
          ptx::mma_commit_pair(&bars->empty[stage], 0x3);
          if (++stage == P_STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit_pair(&bars->tfull[buf], 0x3);
      }
      if (!ok) atomicExch(status, ST_ETIMEOUT);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3;          // TMEM lanes 32*quarter .. (warp % 4 rule)
    const int half = (warp - 2) >> 2;      // which half of the tile's columns
    const uint32_t tempty_cl[2] = {ptx::mapa(ptx::smem_u32(&bars->tempty[0]), 0),
                                   ptx::mapa(ptx::smem_u32(&bars->tempty[1]), 0)};
    int it = 0;
    uint4 pre[8];
    for (int tile = cluster; tile < tiles; tile += n_clusters, ++it) {
      const int buf = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      const int mb = tile / n_blocks, nb = tile % n_blocks;
      const int row0 = mb * P_BM + (int)rank * P_HALF + quarter * 32;
      if (EPI == EPI_RESID)
        resid_load(ep, pre, row0, M - row0 < 32 ? M - row0 : 32, nb * BN + half * (BN / 2), lane);
      if (!ptx::mbar_wait(&bars->tfull[buf], use & 1)) {
        atomicExch(status, ST_ETIMEOUT);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t taddr = tmem + (uint32_t)(buf * BN) + ((uint32_t)(quarter * 32) << 16);
      epilogue_tile<EPI>(ep, stg + (warp - 2) * STG_BYTES, row0, nb * BN, taddr, M, half, lane, pre);
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive_cluster(tempty_cl[buf]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // neither CTA leaves while the pair's MMAs, loads or arrives may still touch it
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc2(tmem, TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint32_t box_outer,
              uint64_t row_stride, bool f16) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {(row_stride ? row_stride : inner) * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool g_gemm_pairs = true;   // st_set_gemm_pairs: CTA-pair kernel for M > 128

}  // namespace

void set_gemm_pairs(bool on) { g_gemm_pairs = on; }
bool gemm_pair_enabled() { return g_gemm_pairs; }

bool gemm_tc_supported(int M, int N, int K) {
  return M > 0 && N > 0 && K > 0 && N % BN == 0 && K % BK == 0;
}

// CTA-pair launch: clusters of two, as many as can be resident at once (the
// tile loop is persistent, so a cluster that waited for a free SM pair would
// add a second wave).
template <int EPI>
cudaError_t launch_pair(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, const EpiParams& ep,
                        int* status, cudaStream_t s, uint32_t idesc) {
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = P_SMEM_BYTES;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (!max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc2<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2 * (num_sms() / 2));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k_gemm_tc2<EPI>, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_clusters = n;
  }
  const int tiles = ((M + P_BM - 1) / P_BM) * (N / BN);
  cfg.gridDim = dim3(2 * (tiles < max_clusters ? tiles : max_clusters));
  return cudaLaunchKernelEx(&cfg, k_gemm_tc2<EPI>, ma, mb, M, N, K, ep, status, idesc);
}

int gemm_tc(const void* A, const void* W, int M, int N, int K, const EpiParams& ep, int* status,
            cudaStream_t s, bool f16) {
  if (M <= 0) return ST_OK;
  if (!gemm_tc_supported(M, N, K)) return ST_EUNSUPPORTED;
  if (M > BM && gemm_pair_enabled()) {
    // 2-SM MMA: W and A tiles of 128 rows per CTA
    const uint32_t idesc = f16 ? ptx::idesc_f16_f32(P_BM, BN) : ptx::idesc_bf16_f32(P_BM, BN);
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, (uint64_t)K, (uint64_t)M, P_HALF, (uint64_t)ep.a_ld, f16) ||
        !make_map(&mb, W, (uint64_t)K, (uint64_t)N, P_HALF, 0, f16))
      return ST_ECUDA;
    cudaError_t e;
    switch (ep.mode) {
      case EPI_QKV: e = launch_pair<EPI_QKV>(ma, mb, M, N, K, ep, status, s, idesc); break;
      case EPI_RESID: e = launch_pair<EPI_RESID>(ma, mb, M, N, K, ep, status, s, idesc); break;
      case EPI_SWIGLU: e = launch_pair<EPI_SWIGLU>(ma, mb, M, N, K, ep, status, s, idesc); break;
      default: e = launch_pair<EPI_STORE_F32>(ma, mb, M, N, K, ep, status, s, idesc); break;
    }
    return e == cudaSuccess ? ST_OK : ST_ECUDA;
  }
  const uint32_t idesc = f16 ? ptx::idesc_f16_f32(BM, BN) : ptx::idesc_bf16_f32(BM, BN);
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, (uint64_t)K, (uint64_t)M, BM, (uint64_t)ep.a_ld, f16) ||
      !make_map(&mb, W, (uint64_t)K, (uint64_t)N, BN, 0, f16))
    return ST_ECUDA;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<EPI_QKV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    cudaFuncSetAttribute(k_gemm_tc<EPI_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    cudaFuncSetAttribute(k_gemm_tc<EPI_SWIGLU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    cudaFuncSetAttribute(k_gemm_tc<EPI_STORE_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr = true;
  }
  const int tiles = ((M + BM - 1) / BM) * (N / BN);
  const int grid = tiles < num_sms() ? tiles : num_sms();
  switch (ep.mode) {
    case EPI_QKV: k_gemm_tc<EPI_QKV><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, M, N, K, ep, status, idesc); break;
    case EPI_RESID: k_gemm_tc<EPI_RESID><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, M, N, K, ep, status, idesc); break;
    case EPI_SWIGLU: k_gemm_tc<EPI_SWIGLU><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, M, N, K, ep, status, idesc); break;
    default: k_gemm_tc<EPI_STORE_F32><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, M, N, K, ep, status, idesc); break;
  }
  return ST_OK;
}

}  // namespace st
