// Retention scores of the scoring ablation (Sec. 5 "Offline: KV Cache
// Creation" contrasts query-agnostic with query-specific pruning):
//
//  * full Expected Attention -- per (tuple, layer, kv head) the mean mu and the
//    full covariance Sigma of the PRE-RoPE queries of the group over the
//    document, turned into the Gaussian of the expected post-RoPE query at the
//    future positions L .. L+F-1 with the averaged rotation Rbar:
//    m = Rbar mu, M = Rbar Sigma Rbar^T (k_qmoments); every slot then scores
//    m.k/sqrt(hd) + k^T M k/(2 hd) + ln(||v|| + 1e-12) (k_quad_scores);
//  * query-specific -- the attention probability the operator's prompt
//    queries put on each document slot in the r = 1 forward (k_query_mass).
//
// CUDA-core kernels: the moments are a rank-N update of a 64 x 64 matrix per
// (tuple, kv head) and the quadratic form is 4096 FMAs per slot; both run in
// the offline build (or once per operator), next to GEMMs that dominate it.
#include "kernels.h"

namespace st {

namespace {

constexpr int kB = 32;   // query vectors staged per batch (k_qmoments)

// Block per (tuple, kv head), 256 threads.  Pre-RoPE queries come from the
// post-RoPE Q rows by the inverse rotation at the row's document position j
// (pre = R(j)^T post).  One pass, shifted by the group's first query (at
// position 0 RoPE is the identity): S1 = sum(d), S2 = sum(d d^T) with
// d = q_pre - shift; mu = shift + S1/N, Sigma = S2/N - (S1/N)(S1/N)^T.
// S2 in register blocks: thread (rb, cb) of a 16 x 16 grid owns the BLK x BLK
// block at rows BLK*rb, columns BLK*cb (BLK = HD/16), two vector loads of the
// staged item per BLK*BLK FMAs.
template <typename act_t, int HD>
__global__ void __launch_bounds__(256) k_qmoments(const act_t* __restrict__ q, const int64_t* __restrict__ off,
                                                  int t0, int64_t r0, int hq, int hkv,
                                                  const float2* __restrict__ rope,
                                                  const float2* __restrict__ ravg, float* __restrict__ m_out,
                                                  float* __restrict__ M_out) {
  constexpr int H2 = HD / 2, TPR = 256 / HD, EPT = HD / TPR, BLK = HD / 16;
  __shared__ __align__(16) float d[kB][HD];
  __shared__ float shift[HD], mean_d[HD];
  __shared__ float sig[HD][HD + 1];
  const int lt = blockIdx.x / hkv, g = blockIdx.x % hkv, t = t0 + lt;
  const int G = hq / hkv, tid = threadIdx.x;
  const int L = (int)(off[t + 1] - off[t]);
  const int64_t N = (int64_t)L * G;
  const act_t* base = q + (off[t] - r0) * hq * HD + (int64_t)g * G * HD;
  if (tid < HD) shift[tid] = to_f(base[tid]);
  __syncthreads();
  const int rb = tid / 16, cb = tid % 16;
  float acc[BLK][BLK];
#pragma unroll
  for (int x = 0; x < BLK; ++x)
#pragma unroll
    for (int y = 0; y < BLK; ++y) acc[x][y] = 0.f;
  float s1 = 0.f;
  for (int64_t n0 = 0; n0 < N; n0 += kB) {
    for (int idx = tid; idx < kB * H2; idx += 256) {
      const int k = idx / H2, i = idx % H2;
      const int64_t it = n0 + k;
      float x0 = 0.f, x1 = 0.f;                 // items past N contribute nothing
      if (it < N) {
        const int64_t j = it / G;
        const int hh = (int)(it % G);
        const act_t* qp = base + j * hq * HD + hh * HD;
        const float pa = to_f(qp[i]), pb = to_f(qp[i + H2]);
        const float2 cs = rope[j * H2 + i];
        x0 = fmaf(pa, cs.x, pb * cs.y) - shift[i];
        x1 = fmaf(pb, cs.x, -pa * cs.y) - shift[i + H2];
      }
      d[k][i] = x0;
      d[k][i + H2] = x1;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kB; ++k) {
      float ra[BLK], ca[BLK];
      if (BLK == 4) {
        const float4 u = *reinterpret_cast<const float4*>(&d[k][BLK * rb]);
        const float4 w = *reinterpret_cast<const float4*>(&d[k][BLK * cb]);
        ra[0] = u.x; ra[1] = u.y; ra[2] = u.z; ra[3] = u.w;
        ca[0] = w.x; ca[1] = w.y; ca[2] = w.z; ca[3] = w.w;
      } else {
#pragma unroll
        for (int x = 0; x < BLK; ++x) {
          ra[x] = d[k][BLK * rb + x];
          ca[x] = d[k][BLK * cb + x];
        }
      }
#pragma unroll
      for (int x = 0; x < BLK; ++x)
#pragma unroll
        for (int y = 0; y < BLK; ++y) acc[x][y] = fmaf(ra[x], ca[y], acc[x][y]);
    }
    if (tid < HD)
      for (int k = 0; k < kB; ++k) s1 += d[k][tid];
    __syncthreads();
  }
  const float invN = 1.f / (float)N;
  if (tid < HD) mean_d[tid] = s1 * invN;
  __syncthreads();
#pragma unroll
  for (int x = 0; x < BLK; ++x)
#pragma unroll
    for (int y = 0; y < BLK; ++y) {
      const int ra = BLK * rb + x, ca = BLK * cb + y;
      sig[ra][ca] = acc[x][y] * invN - mean_d[ra] * mean_d[ca];
    }
  const int a = tid / TPR, c0 = (tid % TPR) * EPT;   // entries of the rotation steps
  __syncthreads();
  const float2* rv = ravg + (int64_t)L * H2;   // (mean cos, mean sin) of the horizon after L
  float* mo = m_out + ((int64_t)lt * hkv + g) * HD;
  if (tid < H2) {
    const float2 r = rv[tid];
    const float ua = shift[tid] + mean_d[tid], ub = shift[tid + H2] + mean_d[tid + H2];
    mo[tid] = r.x * ua - r.y * ub;
    mo[tid + H2] = r.y * ua + r.x * ub;
  }
  __syncthreads();
  // A = Rbar Sigma (pairs of rows), then M = A Rbar^T (pairs of columns)
  float tmp[EPT];
  {
    const int i = a < H2 ? a : a - H2;
    const float2 r = rv[i];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const float lo = sig[i][c0 + e], hi = sig[i + H2][c0 + e];
      tmp[e] = a < H2 ? r.x * lo - r.y * hi : r.y * lo + r.x * hi;
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < EPT; ++e) sig[a][c0 + e] = tmp[e];
  __syncthreads();
  float* Mo = M_out + ((int64_t)lt * hkv + g) * HD * HD + (int64_t)a * HD;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int c = c0 + e, i = c < H2 ? c : c - H2;
    const float2 r = rv[i];
    const float lo = sig[a][i], hi = sig[a][i + H2];
    Mo[c] = c < H2 ? r.x * lo - r.y * hi : r.y * lo + r.x * hi;
  }
}

// Block per (tuple, kv head): m and M in shared memory, one slot per thread.
template <typename act_t, int HD>
__global__ void __launch_bounds__(256) k_quad_scores(const act_t* __restrict__ K, const act_t* __restrict__ V,
                                                     int64_t R, const int64_t* __restrict__ off, int t0,
                                                     int hkv, const float* __restrict__ m_in,
                                                     const float* __restrict__ M_in, float* __restrict__ scores) {
  constexpr int VN = Vec<act_t>::N;
  __shared__ __align__(16) float Ms[HD][HD];
  __shared__ float ms[HD];
  const int lt = blockIdx.x / hkv, g = blockIdx.x % hkv, t = t0 + lt;
  const float* Mp = M_in + ((int64_t)lt * hkv + g) * HD * HD;
  for (int e = threadIdx.x; e < HD * HD; e += blockDim.x) Ms[e / HD][e % HD] = Mp[e];
  if (threadIdx.x < HD) ms[threadIdx.x] = m_in[((int64_t)lt * hkv + g) * HD + threadIdx.x];
  __syncthreads();
  const int64_t d0 = off[t];
  const int L = (int)(off[t + 1] - d0);
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    // M is re-read from shared memory for every slot (keeps the compiler from
    // hoisting all HD*HD loads of the unrolled form into registers)
    asm volatile("" ::: "memory");
    const int64_t row = (int64_t)g * R + d0 + j;
    float k[HD], vv = 0.f;
#pragma unroll
    for (int c = 0; c < HD; c += VN) {
      float x[VN];
      Vec<act_t>::load(K + row * HD + c, k + c);
      Vec<act_t>::load(V + row * HD + c, x);
#pragma unroll
      for (int e = 0; e < VN; ++e) vv = fmaf(x[e], x[e], vv);
    }
    float lin = 0.f, quad = 0.f;
#pragma unroll
    for (int c = 0; c < HD; ++c) lin = fmaf(ms[c], k[c], lin);
#pragma unroll
    for (int r = 0; r < HD; ++r) {
      float y = 0.f;
#pragma unroll
      for (int c = 0; c < HD; c += 4) {
        const float4 mr = *reinterpret_cast<const float4*>(&Ms[r][c]);
        y = fmaf(mr.x, k[c], y);
        y = fmaf(mr.y, k[c + 1], y);
        y = fmaf(mr.z, k[c + 2], y);
        y = fmaf(mr.w, k[c + 3], y);
      }
      quad = fmaf(k[r], y, quad);
    }
    scores[row] = lin / sqrtf((float)HD) + quad / (2.0f * HD) + logf(sqrtf(vv) + 1e-12f);
  }
}

// q . k for a query in registers and a staged key row (16-byte aligned), four
// independent partial sums.
template <int HD>
__device__ __forceinline__ float dot_row(const float (&qr)[HD], const float* kr) {
  float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < HD; c += 4) {
    const float4 k4 = *reinterpret_cast<const float4*>(kr + c);
    s[0] = fmaf(qr[c], k4.x, s[0]);
    s[1] = fmaf(qr[c + 1], k4.y, s[1]);
    s[2] = fmaf(qr[c + 2], k4.z, s[2]);
    s[3] = fmaf(qr[c + 3], k4.w, s[3]);
  }
  return (s[0] + s[1]) + (s[2] + s[3]);
}

// Block per (pair, kv head), one thread per prompt query row (p, head of the
// group), blockDim.x (<= 256, a multiple of 32) rows per pass.  Pass 1: the
// row's softmax maximum and normaliser over the document slots and its
// visible prompt keys; pass 2:
// each document slot's probability, summed over the rows (warp sums, then
// shared-memory atomics), added into scores.  Keys are staged 64 at a time.
template <typename act_t, int HD>
__global__ void __launch_bounds__(256) k_query_mass(const act_t* __restrict__ q, const act_t* __restrict__ kp,
                                                    const act_t* __restrict__ K, int64_t R,
                                                    const int64_t* __restrict__ off,
                                                    const int32_t* __restrict__ tup,
                                                    const int32_t* __restrict__ prow, int P, int hq, int hkv,
                                                    float scale, float* __restrict__ scores) {
  constexpr int TK = 64;
  __shared__ __align__(16) float ks[TK][HD];   // every thread reads the same key: broadcast
  __shared__ float msum[TK];
  const int i = blockIdx.x / hkv, g = blockIdx.x % hkv, G = hq / hkv;
  const int tid = threadIdx.x, lane = tid & 31;
  const int t = tup[i];
  const int64_t d0 = off[t];
  const int L = (int)(off[t + 1] - d0);
  const int64_t p0 = prow[i];
  const int nrows = P * G;
  auto stage = [&](int k0, int nk) {
    for (int e = tid; e < TK * HD; e += blockDim.x) {
      const int kk = e / HD, c = e % HD, key = k0 + kk;
      float x = 0.f;
      if (kk < nk) {
        x = key < L ? to_f(K[((int64_t)g * R + d0 + key) * HD + c])
                    : to_f(kp[((p0 + key - L) * hkv + g) * HD + c]);
      }
      ks[kk][c] = x;
    }
  };
  for (int rb = 0; rb < nrows; rb += blockDim.x) {
    const int row = rb + tid;
    const bool live = row < nrows;
    const int p = live ? row / G : 0, hh = live ? row % G : 0;
    float qr[HD];
    const act_t* qp = q + ((p0 + p) * hq + (int64_t)g * G + hh) * HD;
#pragma unroll
    for (int c = 0; c < HD; ++c) qr[c] = live ? to_f(qp[c]) * scale : 0.f;
    float m = -INFINITY, l = 0.f;
    for (int k0 = 0; k0 < L + P; k0 += TK) {
      const int nk = min(TK, L + P - k0);
      stage(k0, nk);
      __syncthreads();
      for (int kk = 0; kk < nk; ++kk) {
        const int key = k0 + kk;
        if (live && (key < L || key - L <= p)) {
          const float s = dot_row<HD>(qr, ks[kk]);
          if (s > m) {
            l = l * expf(m - s) + 1.f;
            m = s;
          } else {
            l += expf(s - m);
          }
        }
      }
      __syncthreads();
    }
    const float inv_l = live ? 1.f / l : 0.f;
    for (int k0 = 0; k0 < L; k0 += TK) {
      const int nk = min(TK, L - k0);
      stage(k0, nk);
      for (int e = tid; e < TK; e += blockDim.x) msum[e] = 0.f;
      __syncthreads();
      for (int kk = 0; kk < nk; ++kk) {
        float pv = 0.f;
        if (live) pv = expf(dot_row<HD>(qr, ks[kk]) - m) * inv_l;
        pv = warp_sum(pv);
        if (lane == 0) atomicAdd(&msum[kk], pv);
      }
      __syncthreads();
      for (int e = tid; e < nk; e += blockDim.x) {
        float* o = scores + (int64_t)g * R + d0 + k0 + e;
        *o = (rb == 0 ? 0.f : *o) + msum[e];
      }
      __syncthreads();
    }
  }
}

}  // namespace

bool ea_full_supported(int hd) { return hd == 32 || hd == 64; }

template <typename act_t>
void ea_full_scores(const act_t* q, const act_t* K, const act_t* V, int64_t R, const int64_t* off, int t0,
                    int t1, int64_t r0, int hq, int hkv, int hd, const float2* rope, const float2* ravg,
                    float* m_ws, float* M_ws, float* scores, cudaStream_t s) {
  const int nb = (t1 - t0) * hkv;
  if (nb <= 0) return;
  if (hd == 64) {
    k_qmoments<act_t, 64><<<nb, 256, 0, s>>>(q, off, t0, r0, hq, hkv, rope, ravg, m_ws, M_ws);
    k_quad_scores<act_t, 64><<<nb, 256, 0, s>>>(K, V, R, off, t0, hkv, m_ws, M_ws, scores);
  } else {
    k_qmoments<act_t, 32><<<nb, 256, 0, s>>>(q, off, t0, r0, hq, hkv, rope, ravg, m_ws, M_ws);
    k_quad_scores<act_t, 32><<<nb, 256, 0, s>>>(K, V, R, off, t0, hkv, m_ws, M_ws, scores);
  }
}
template void ea_full_scores<float>(const float*, const float*, const float*, int64_t, const int64_t*, int,
                                    int, int64_t, int, int, int, const float2*, const float2*, float*,
                                    float*, float*, cudaStream_t);
template void ea_full_scores<bf16>(const bf16*, const bf16*, const bf16*, int64_t, const int64_t*, int, int,
                                   int64_t, int, int, int, const float2*, const float2*, float*, float*,
                                   float*, cudaStream_t);

template <typename act_t>
void query_mass(const act_t* q, const act_t* kp, const act_t* K, int64_t R, const int64_t* off,
                const int32_t* tup, const int32_t* prow, int P, int np, int hq, int hkv, int hd, float scale,
                float* scores, cudaStream_t s) {
  const int nb = np * hkv;
  if (nb <= 0) return;
  const int rows = P * (hq / hkv);
  const int threads = rows >= 256 ? 256 : (rows + 31) / 32 * 32;
  if (hd == 64)
    k_query_mass<act_t, 64><<<nb, threads, 0, s>>>(q, kp, K, R, off, tup, prow, P, hq, hkv, scale, scores);
  else
    k_query_mass<act_t, 32><<<nb, threads, 0, s>>>(q, kp, K, R, off, tup, prow, P, hq, hkv, scale, scores);
}
template void query_mass<float>(const float*, const float*, const float*, int64_t, const int64_t*,
                                const int32_t*, const int32_t*, int, int, int, int, int, float, float*,
                                cudaStream_t);
template void query_mass<bf16>(const bf16*, const bf16*, const bf16*, int64_t, const int64_t*,
                               const int32_t*, const int32_t*, int, int, int, int, int, float, float*,
                               cudaStream_t);

}  // namespace st
