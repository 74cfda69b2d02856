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
//               fused epilogue (RoPE + Q/K/V scatter, residual add, SwiGLU)
//               straight from registers to global memory.
// The two accumulators let the epilogue of tile i overlap the main loop of
// tile i+1.  Every mbarrier wait is bounded; a timeout sets the status word.
#include <cudaTypedefs.h>

#include "epilogue.cuh"
#include "ptx.cuh"

namespace st {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_THREADS = 320;   // producer, MMA, 8 epilogue warps
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256;

struct Bars {
  uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
  uint32_t tmem_base;
};

// Columns [half * BN/2, (half + 1) * BN/2) of the tile for one accumulator row
// (SwiGLU: gate columns [half*64, half*64 + 64) with their up columns).
__device__ __forceinline__ void epilogue_tile(const EpiParams& ep, int row, int n0,
                                              uint32_t taddr, int M, int half) {
  const float inv = row < M ? row_inv_rms(ep, row) : 1.f;
  if (ep.mode == EPI_SWIGLU) {
    // columns [0,128) are gate, [128,256) the matching up projections
#pragma unroll 1
    for (int j = half * (BN / 4); j < (half + 1) * (BN / 4); j += 32) {
      uint32_t g[32], u[32];
      ST_TMEM_LD32(taddr + j, g);
      ST_TMEM_LD32(taddr + BN / 2 + j, u);
      ptx::tmem_wait_ld();
      if (row < M) {
        float gf[32], uf[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          gf[e] = __uint_as_float(g[e]) * inv;
          uf[e] = __uint_as_float(u[e]) * inv;
        }
        epilogue_swiglu<bf16, 32>(ep, row, n0 / 2 + j, gf, uf);
      }
    }
  } else {
    float ss = 0.f;
#pragma unroll 1
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 64) {
      uint32_t r[64];
      uint32_t* r2 = r + 32;
      ST_TMEM_LD32(taddr + c, r);
      ST_TMEM_LD32(taddr + c + 32, r2);
      ptx::tmem_wait_ld();
      if (row < M) {
        float v[64];
#pragma unroll
        for (int e = 0; e < 64; ++e) v[e] = __uint_as_float(r[e]);
        ss += epilogue_apply<bf16, 64>(ep, row, n0 + c, v, inv);
      }
    }
    if (ep.mode == EPI_RESID && ep.ssq_out != nullptr && row < M)
      ep.ssq_out[(int64_t)row * (ep.N / 128) + (n0 + half * (BN / 2)) / 128] = ss;
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int M, int N, int K, EpiParams ep, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  Bars* bars = reinterpret_cast<Bars*>(smem + STAGES * STAGE_BYTES);
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
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
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
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int buf = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      if (!ptx::mbar_wait(&bars->tfull[buf], use & 1)) {
        atomicExch(status, ST_ETIMEOUT);
        break;
      }
      ptx::tc_fence_after();
      const int mb = tile / n_blocks, nb = tile % n_blocks;
      const int row = mb * BM + quarter * 32 + lane;
      const uint32_t taddr = tmem + (uint32_t)(buf * BN) + ((uint32_t)(quarter * 32) << 16);
      epilogue_tile(ep, row, nb * BN, taddr, M, half);
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
              uint64_t row_stride = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {(row_stride ? row_stride : inner) * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc_supported(int M, int N, int K) {
  return M > 0 && N > 0 && K > 0 && N % BN == 0 && K % BK == 0;
}

int gemm_tc(const bf16* A, const bf16* W, int M, int N, int K, const EpiParams& ep, int* status,
            cudaStream_t s) {
  if (M <= 0) return ST_OK;
  if (!gemm_tc_supported(M, N, K)) return ST_EUNSUPPORTED;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, (uint64_t)K, (uint64_t)M, BM, (uint64_t)ep.a_ld) ||
      !make_map(&mb, W, (uint64_t)K, (uint64_t)N, BN))
    return ST_ECUDA;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr = true;
  }
  const int tiles = ((M + BM - 1) / BM) * (N / BN);
  const int grid = tiles < num_sms() ? tiles : num_sms();
  k_gemm_tc<<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, M, N, K, ep, status);
  return ST_OK;
}

}  // namespace st
