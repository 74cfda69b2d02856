// CUDA-core projection GEMM for the float32 model (true FP32 FMA; TF32 tensor
// cores would not meet a 1e-4 relative error bound).  C = A . W^T with A
// [M][K] row-major and W [N][K] row-major.  Tile 32 rows x 4W columns, one
// thread per (row, W-column chunk); the epilogue runs on the thread's W
// accumulators.
#include "epilogue.cuh"

namespace st {

template <typename act_t, int W>
__global__ void __launch_bounds__(128) k_gemm_simt(const act_t* __restrict__ A,
                                                   const act_t* __restrict__ B, int M, int N,
                                                   int K, EpiParams ep) {
  constexpr int BM = 32, BN = 4 * W, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int64_t lda = ep.a_ld > 0 ? ep.a_ld : K;
  float acc[W];
#pragma unroll
  for (int j = 0; j < W; ++j) acc[j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 128) {
      int r = e / BK, k = e % BK;
      int gr = m0 + r;
      As[k][r] = gr < M ? to_f(A[(int64_t)gr * lda + k0 + k]) : 0.f;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 128) {
      int n = e / BK, k = e % BK;
      Bs[k][n] = to_f(B[(int64_t)(n0 + n) * K + k0 + k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a = As[k][lane];
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j] = fmaf(a, Bs[k][warp * W + j], acc[j]);
    }
    __syncthreads();
  }
  const int row = m0 + lane;
  if (row < M) epilogue_apply<act_t, W>(ep, row, n0 + warp * W, acc);
}

template <typename act_t>
void gemm_simt(const act_t* A, const act_t* W, int M, int N, int K, const EpiParams& ep,
               cudaStream_t s) {
  if (M <= 0) return;
  const int w = (ep.mode == EPI_QKV) ? ep.hd : 32;
  dim3 grid(N / (4 * w), (M + 31) / 32);
  if (w == 64)
    k_gemm_simt<act_t, 64><<<grid, 128, 0, s>>>(A, W, M, N, K, ep);
  else
    k_gemm_simt<act_t, 32><<<grid, 128, 0, s>>>(A, W, M, N, K, ep);
}
template void gemm_simt<float>(const float*, const float*, int, int, int, const EpiParams&,
                               cudaStream_t);
template void gemm_simt<bf16>(const bf16*, const bf16*, int, int, int, const EpiParams&,
                              cudaStream_t);

}  // namespace st
