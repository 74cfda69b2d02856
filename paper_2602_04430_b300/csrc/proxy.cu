// The learned proxy: a cheap first stage of a two-stage cascade in front of
// the KV-cache operator (cascade semantics of Sec. 4.1: a stage accepts or
// rejects a tuple, or marks it unsure and passes it on).
//
// Network  Linear(d, h1) - GELU - Linear(h1, h2) - GELU - Linear(h2, 2) over the
//          pooled final-normed last-layer document state saved by kv_build.
// Training softmax cross-entropy against the full operator's labels, Adam.
// Cascade  tuples whose proxy confidence (max softmax probability) is below tau
//          are compacted, in order, into a list for the full operator; the
//          final labels take the proxy's where it is confident.
//
// Precision (st_proxy_set_precision): float32 contractions on the CUDA cores
// (default), or BF16 contractions on the tensor cores (mma.sync m16n8k16,
// operands rounded to bfloat16, float32 accumulation -- the learned-proxy
// configuration's precision).  Parameters, Adam moments, biases, GELU and the
// loss are float32 either way.  The network is ~2 MFLOP per tuple, far from
// the path's critical time in both.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.h"

namespace {

using namespace st;

enum MmEpi { MM_STORE = 0, MM_BIAS = 1, MM_BIAS_GELU = 2, MM_DGELU = 3 };

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C[m][n] = sum_k A(m, k) B(n, k), A(m, k) = A[m*sam + k*sak], B(n, k) = B[n*sbn + k*sbk].
// 64 x 64 tiles, 256 threads, 4 x 4 outputs per thread.
template <int EPI>
__global__ void __launch_bounds__(256) k_mm(const float* __restrict__ A, int64_t sam, int64_t sak,
                                            const float* __restrict__ B, int64_t sbn, int64_t sbk,
                                            int M, int N, int K, const float* __restrict__ bias,
                                            float* __restrict__ pre, float* __restrict__ C) {
  __shared__ float As[16][64 + 1], Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int i = e >> 4, k = e & 15;
      const int gm = m0 + i, gn = n0 + i, gk = k0 + k;
      As[k][i] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.f;
      Bs[k][i] = (gn < N && gk < K) ? B[gn * sbn + gk * sbk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[k][ty * 4 + i];
        b[i] = Bs[k][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      const int64_t o = (int64_t)m * N + n;
      if (EPI == MM_BIAS || EPI == MM_BIAS_GELU) v += bias[n];
      if (EPI == MM_BIAS_GELU) {
        pre[o] = v;
        v = gelu_f(v);
      }
      if (EPI == MM_DGELU) v *= gelu_grad_f(pre[o]);
      C[o] = v;
    }
  }
}

// The same contraction on the BF16 tensor-core path (the learned-proxy
// configuration's precision): each operand element is rounded from float32 to
// bfloat16 (nearest, ties to even) as it is staged in shared memory, and
// mma.sync m16n8k16 accumulates in float32; the epilogue is k_mm's.
// 64 x 64 tiles over K steps of 32, 4 warps of 32 x 32 (2 x 4 MMA tiles).
constexpr int BM = 64, BK = 32, BKP = BK + 8;   // padded rows: conflict-free fragment loads
template <int EPI>
__global__ void __launch_bounds__(128) k_mm_bf16(const float* __restrict__ A, int64_t sam, int64_t sak,
                                                 const float* __restrict__ B, int64_t sbn, int64_t sbk,
                                                 int M, int N, int K, const float* __restrict__ bias,
                                                 float* __restrict__ pre, float* __restrict__ C) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BKP], Bs[BM][BKP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BM;
  float acc[2][4][4] = {};
  // stage one operand tile, walking the unit-stride index fastest (coalesced)
  auto stage = [&](const float* X, int64_t s_row, int64_t s_k, int rows, int r0, int k0,
                   __nv_bfloat16 (*S)[BKP]) {
    const bool k_fast = s_k == 1;
    for (int e = threadIdx.x; e < BM * BK; e += 128) {
      const int i = k_fast ? e / BK : e % BM;
      const int k = k_fast ? e % BK : e / BM;
      const int gr = r0 + i, gk = k0 + k;
      const float v = (gr < rows && gk < K) ? X[(int64_t)gr * s_row + (int64_t)gk * s_k] : 0.f;
      S[i][k] = __float2bfloat16_rn(v);
    }
  };
  for (int k0 = 0; k0 < K; k0 += BK) {
    stage(A, sam, sak, M, m0, k0, As);
    stage(B, sbn, sbk, N, n0, k0, Bs);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
        a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
        a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + g;
        b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t]);
        b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm + 16 * i + g + (e >> 1) * 8;
        const int n = n0 + wn + 8 * j + 2 * t + (e & 1);
        if (m >= M || n >= N) continue;
        float v = acc[i][j][e];
        const int64_t o = (int64_t)m * N + n;
        if (EPI == MM_BIAS || EPI == MM_BIAS_GELU) v += bias[n];
        if (EPI == MM_BIAS_GELU) {
          pre[o] = v;
          v = gelu_f(v);
        }
        if (EPI == MM_DGELU) v *= gelu_grad_f(pre[o]);
        C[o] = v;
      }
}

template <int EPI>
void mm(bool bf, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbn, int64_t sbk, int M,
        int N, int K, const float* bias, float* pre, float* C, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if (bf)
    k_mm_bf16<EPI><<<grid, 128, 0, s>>>(A, sam, sak, B, sbn, sbk, M, N, K, bias, pre, C);
  else
    k_mm<EPI><<<grid, 256, 0, s>>>(A, sam, sak, B, sbn, sbk, M, N, K, bias, pre, C);
}

__global__ void k_gather(const float* __restrict__ x, const int32_t* __restrict__ rows, int n,
                         int d, float* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * d) return;
  const int64_t r = i / d;
  const int c = (int)(i % d);
  out[i] = x[(int64_t)(rows ? rows[r] : r) * d + c];
}

// Softmax cross-entropy over 2 logits: dz = (p - onehot(y)) / B, loss = mean(-log p_y).
__global__ void k_ce(const float* __restrict__ z, const int32_t* __restrict__ y,
                     const int32_t* __restrict__ rows, int B, float* __restrict__ dz,
                     float* __restrict__ loss) {
  __shared__ float red[1024];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float z0 = z[2 * b], z1 = z[2 * b + 1];
    const float m = fmaxf(z0, z1);
    const float e0 = expf(z0 - m), e1 = expf(z1 - m);
    const float lse = m + logf(e0 + e1);
    const int t = y[rows ? rows[b] : b];
    acc += lse - (t == 1 ? z1 : z0);
    const float p0 = e0 / (e0 + e1), p1 = e1 / (e0 + e1);
    dz[2 * b] = (p0 - (t == 0 ? 1.f : 0.f)) / (float)B;
    dz[2 * b + 1] = (p1 - (t == 1 ? 1.f : 0.f)) / (float)B;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)B;
}

// db[n] = sum_b dA[b][n]
__global__ void k_colsum(const float* __restrict__ dA, int B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int b = 0; b < B; ++b) acc += dA[(int64_t)b * N + n];
  db[n] = acc;
}

// Adam with bias correction (c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t) from the host).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Confidence (max softmax probability) and label (argmax, ties to 0) of each row.
__global__ void k_head(const float* __restrict__ z, int n, float* __restrict__ conf,
                       int32_t* __restrict__ label) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z0 = z[2 * i], z1 = z[2 * i + 1];
  const float m = fmaxf(z0, z1);
  const float e0 = expf(z0 - m), e1 = expf(z1 - m);
  const float p1 = e1 / (e0 + e1), p0 = e0 / (e0 + e1);
  conf[i] = fmaxf(p0, p1);
  label[i] = p1 > p0 ? 1 : 0;
}

// Order-preserving compaction of the unsure rows (conf < tau), one block.
__global__ void k_compact(const float* __restrict__ conf, const int32_t* __restrict__ ids, int n,
                          float tau, int32_t* __restrict__ out, int32_t* __restrict__ count) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int f = (i < n && conf[i] < tau) ? 1 : 0;
    part[threadIdx.x] = f;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (f) out[carry + part[threadIdx.x] - 1] = ids ? ids[i] : i;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

// final labels: the proxy's everywhere, then the full operator's at the unsure rows
__global__ void k_copy_labels(const int32_t* __restrict__ proxy_label, int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = proxy_label[i];
}
// (pos and count are the caller's: a position outside [0, n) is skipped and
// recorded as ST_ERANGE)
__global__ void k_scatter(const int32_t* __restrict__ pos, const int32_t* __restrict__ count,
                          const int32_t* __restrict__ full, int32_t* __restrict__ out, int n, int* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= *count) return;
  const int q = pos[j];
  if ((unsigned)q < (unsigned)n) out[q] = full[j];
  else atomicCAS(status, ST_OK, ST_ERANGE);
}

}  // namespace

// ------------------------------------------------------------------ handle
struct st_proxy {
  st_ctx* ctx = nullptr;
  int d = 0, h1 = 0, h2 = 0;
  int64_t n_params = 0;
  float* params = nullptr;   // w1 b1 w2 b2 w3 b3, contiguous
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int64_t off[7] = {};       // offsets of the six tensors (+ end)
  int64_t t = 0;             // Adam steps taken
  bool bf16 = false;         // contractions on the BF16 tensor-core path (st_proxy_set_precision)
  // activations of the largest batch seen
  float* ws = nullptr;
  int64_t ws_rows = 0;
};

namespace {

int pfail(st_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

struct Act {
  float *xb, *a1, *h1, *a2, *h2, *z, *dz, *d2, *d1, *loss;
};

int proxy_ws(st_proxy* p, int64_t rows, Act* A) {
  const int64_t need = rows * ((int64_t)p->d + 2 * p->h1 + 2 * p->h2 + 4 + p->h1 + p->h2) + 64;
  if (p->ws_rows < rows) {
    cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_rows = 0;
    if (cudaMalloc((void**)&p->ws, need * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return pfail(p->ctx, ST_ENOMEM, "proxy workspace allocation failed");
    }
    p->ws_rows = rows;
  }
  float* q = p->ws;
  A->xb = q; q += rows * p->d;
  A->a1 = q; q += rows * p->h1;
  A->h1 = q; q += rows * p->h1;
  A->a2 = q; q += rows * p->h2;
  A->h2 = q; q += rows * p->h2;
  A->z = q; q += rows * 2;
  A->dz = q; q += rows * 2;
  A->d2 = q; q += rows * p->h2;
  A->d1 = q; q += rows * p->h1;
  A->loss = q;
  return ST_OK;
}

// Forward pass of `rows` gathered rows; leaves pre-activations and activations in A.
void forward(st_proxy* p, const float* x, const int32_t* rows_idx, int n, Act& A, cudaStream_t s) {
  const float* P = p->params;
  const int d = p->d, h1 = p->h1, h2 = p->h2;
  {
    Launch L(p->ctx, s, ST_PROF_OTHER, 0, 0);
    k_gather<<<(unsigned)(((int64_t)n * d + 255) / 256), 256, 0, s>>>(x, rows_idx, n, d, A.xb);
  }
  {
    Launch L(p->ctx, s, ST_PROF_OTHER, 2.0 * n * d * h1, 0);
    mm<MM_BIAS_GELU>(p->bf16, A.xb, d, 1, P + p->off[0], d, 1, n, h1, d, P + p->off[1], A.a1, A.h1, s);
  }
  {
    Launch L(p->ctx, s, ST_PROF_OTHER, 2.0 * n * h1 * h2, 0);
    mm<MM_BIAS_GELU>(p->bf16, A.h1, h1, 1, P + p->off[2], h1, 1, n, h2, h1, P + p->off[3], A.a2, A.h2, s);
  }
  {
    Launch L(p->ctx, s, ST_PROF_OTHER, 4.0 * n * h2, 0);
    mm<MM_BIAS>(p->bf16, A.h2, h2, 1, P + p->off[4], h2, 1, n, 2, h2, P + p->off[5], nullptr, A.z, s);
  }
}

}  // namespace

extern "C" int st_proxy_create(st_ctx* ctx, int32_t d_in, int32_t h1, int32_t h2,
                               const float* const* init_host, st_proxy** out) {
  if (!ctx || !init_host || !out || d_in < 1 || h1 < 1 || h2 < 1)
    return pfail(ctx, ST_EINVAL, "st_proxy_create: bad argument");
  *out = nullptr;
  st_proxy* p = new st_proxy();
  p->ctx = ctx;
  p->d = d_in;
  p->h1 = h1;
  p->h2 = h2;
  const int64_t sizes[6] = {(int64_t)h1 * d_in, h1, (int64_t)h2 * h1, h2, 2LL * h2, 2};
  p->off[0] = 0;
  for (int i = 0; i < 6; ++i) p->off[i + 1] = p->off[i] + sizes[i];
  p->n_params = p->off[6];
  const size_t bytes = p->n_params * sizeof(float);
  float** bufs[4] = {&p->params, &p->grads, &p->m, &p->v};
  for (float** b : bufs) {
    if (cudaMalloc((void**)b, bytes) != cudaSuccess) {
      cudaGetLastError();
      st_proxy_free(p);
      return pfail(ctx, ST_ENOMEM, "st_proxy_create: allocation failed");
    }
    cudaMemset(*b, 0, bytes);
  }
  for (int i = 0; i < 6; ++i)
    cudaMemcpy(p->params + p->off[i], init_host[i], sizes[i] * sizeof(float), cudaMemcpyHostToDevice);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    st_proxy_free(p);
    return pfail(ctx, ST_ECUDA, "st_proxy_create: upload failed");
  }
  *out = p;
  return ST_OK;
}

extern "C" void st_proxy_free(st_proxy* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  cudaFree(p->params);
  cudaFree(p->grads);
  cudaFree(p->m);
  cudaFree(p->v);
  cudaFree(p->ws);
  delete p;
}

extern "C" int st_proxy_train_step(st_ctx* ctx, st_proxy* p, const float* x_dev,
                                   const int32_t* y_dev, const int32_t* batch_dev, int32_t B,
                                   float lr, float* loss_dev, void* stream) {
  ST_TRACE("st_proxy_train_step");
  if (!ctx || !p || p->ctx != ctx || !x_dev || !y_dev || !batch_dev || B < 1)
    return pfail(ctx, ST_EINVAL, "st_proxy_train_step: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Act A;
  int rc = proxy_ws(p, B, &A);
  if (rc != ST_OK) return rc;
  forward(p, x_dev, batch_dev, B, A, s);
  const float* P = p->params;
  float* G = p->grads;
  const int d = p->d, h1 = p->h1, h2 = p->h2;
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_ce<<<1, 1024, 0, s>>>(A.z, y_dev, batch_dev, B, A.dz, loss_dev ? loss_dev : A.loss);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    // dW3 = dz^T h2, db3 = colsum(dz); d2 = (dz W3) * gelu'(a2)
    mm<MM_STORE>(p->bf16, A.dz, 1, 2, A.h2, 1, h2, 2, h2, B, nullptr, nullptr, G + p->off[4], s);
    k_colsum<<<1, 32, 0, s>>>(A.dz, B, 2, G + p->off[5]);
    mm<MM_DGELU>(p->bf16, A.dz, 2, 1, P + p->off[4], 1, h2, B, h2, 2, nullptr, A.a2, A.d2, s);
    // dW2 = d2^T h1, db2; d1 = (d2 W2) * gelu'(a1)
    mm<MM_STORE>(p->bf16, A.d2, 1, h2, A.h1, 1, h1, h2, h1, B, nullptr, nullptr, G + p->off[2], s);
    k_colsum<<<(h2 + 127) / 128, 128, 0, s>>>(A.d2, B, h2, G + p->off[3]);
    mm<MM_DGELU>(p->bf16, A.d2, h2, 1, P + p->off[2], 1, h1, B, h1, h2, nullptr, A.a1, A.d1, s);
    // dW1 = d1^T x, db1
    mm<MM_STORE>(p->bf16, A.d1, 1, h1, A.xb, 1, d, h1, d, B, nullptr, nullptr, G + p->off[0], s);
    k_colsum<<<(h1 + 127) / 128, 128, 0, s>>>(A.d1, B, h1, G + p->off[1]);
  }
  p->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)p->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)p->t)));
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_adam<<<(unsigned)((p->n_params + 255) / 256), 256, 0, s>>>(
        p->params, G, p->m, p->v, p->n_params, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(ctx, ST_ECUDA, cudaGetErrorString(e));
  return ST_OK;
}

extern "C" int st_proxy_eval(st_ctx* ctx, st_proxy* p, const float* x_dev, const int32_t* rows_dev,
                             int32_t n, float* conf_dev, int32_t* label_dev, void* stream) {
  ST_TRACE("st_proxy_eval");
  if (!ctx || !p || p->ctx != ctx || !x_dev || !conf_dev || !label_dev || n < 0)
    return pfail(ctx, ST_EINVAL, "st_proxy_eval: bad argument");
  if (n == 0) return ST_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Act A;
  int rc = proxy_ws(p, n, &A);
  if (rc != ST_OK) return rc;
  forward(p, x_dev, rows_dev, n, A, s);
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_head<<<(n + 255) / 256, 256, 0, s>>>(A.z, n, conf_dev, label_dev);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(ctx, ST_ECUDA, cudaGetErrorString(e));
  return ST_OK;
}

extern "C" int st_cascade_compact(st_ctx* ctx, const float* conf_dev, const int32_t* ids_dev,
                                  int32_t n, float tau, int32_t* unsure_dev, int32_t* count_dev,
                                  void* stream) {
  ST_TRACE("st_cascade_compact");
  if (!ctx || !conf_dev || !unsure_dev || !count_dev || n < 0)
    return pfail(ctx, ST_EINVAL, "st_cascade_compact: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
  k_compact<<<1, 1024, 0, s>>>(conf_dev, ids_dev, n, tau, unsure_dev, count_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(ctx, ST_ECUDA, cudaGetErrorString(e));
  return ST_OK;
}

extern "C" int st_cascade_merge(st_ctx* ctx, const int32_t* proxy_label_dev, int32_t n,
                                const int32_t* unsure_pos_dev, const int32_t* count_dev,
                                const int32_t* full_label_dev, int32_t* out_dev, void* stream) {
  ST_TRACE("st_cascade_merge");
  if (!ctx || !proxy_label_dev || !unsure_pos_dev || !count_dev || !full_label_dev || !out_dev || n < 0)
    return pfail(ctx, ST_EINVAL, "st_cascade_merge: bad argument");
  if (n == 0) return ST_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_copy_labels<<<(n + 255) / 256, 256, 0, s>>>(proxy_label_dev, n, out_dev);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_scatter<<<(n + 255) / 256, 256, 0, s>>>(unsure_pos_dev, count_dev, full_label_dev, out_dev, n, ctx->dstatus);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(ctx, ST_ECUDA, cudaGetErrorString(e));
  return ST_OK;
}

extern "C" int64_t st_proxy_steps(const st_proxy* p) { return p ? p->t : -1; }

extern "C" int st_proxy_set_precision(st_proxy* p, int32_t dtype) {
  if (!p || (dtype != ST_F32 && dtype != ST_BF16))
    return pfail(p ? p->ctx : nullptr, ST_EINVAL, "st_proxy_set_precision: ST_F32 or ST_BF16");
  p->bf16 = dtype == ST_BF16;
  return ST_OK;
}

extern "C" int st_proxy_restore(st_proxy* p, const float* params_dev, const float* m_dev, const float* v_dev,
                                size_t bytes, int64_t steps, void* stream) {
  if (!p || !params_dev || !m_dev || !v_dev || steps < 0)
    return pfail(p ? p->ctx : nullptr, ST_EINVAL, "st_proxy_restore: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = (size_t)p->n_params * sizeof(float);
  // a state saved from a proxy of another shape (or a truncated buffer) is refused
  // before anything is read
  if (bytes != n)
    return pfail(p->ctx, ST_EINVAL, "st_proxy_restore: " + std::to_string(bytes) + " bytes per buffer, this proxy needs " +
                                        std::to_string(n));
  if (cudaMemcpyAsync(p->params, params_dev, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->m, m_dev, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->v, v_dev, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return pfail(p->ctx, ST_ECUDA, "st_proxy_restore: copy failed");
  p->t = steps;
  return ST_OK;
}

extern "C" int st_proxy_read(const st_proxy* p, int32_t which, void* dst_dev, size_t bytes,
                             void* stream) {
  if (!p || !dst_dev) return ST_EINVAL;
  const float* src = nullptr;
  switch (which) {
    case ST_PROXY_PARAMS: src = p->params; break;
    case ST_PROXY_GRADS: src = p->grads; break;
    case ST_PROXY_ADAM_M: src = p->m; break;
    case ST_PROXY_ADAM_V: src = p->v; break;
    default: return pfail(p->ctx, ST_EINVAL, "st_proxy_read: unknown buffer");
  }
  const size_t n = std::min(bytes, (size_t)p->n_params * sizeof(float));
  if (cudaMemcpyAsync(dst_dev, src, n, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return pfail(p->ctx, ST_ECUDA, "st_proxy_read: copy failed");
  return ST_OK;
}
