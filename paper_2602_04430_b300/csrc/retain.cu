// Query-agnostic retention (Sec. 5): one CTA per (tuple, layer, kv head).
//
// The CTA sorts the segment's float32 scores in shared memory as 64-bit keys
// (order-preserving transform of the negated score in the high word, the slot
// index in the low word), so ascending key order is (score descending, index
// ascending) with -0 == +0; a bitonic network gives a deterministic total
// order.  It writes the full rank order, then gathers the first n_keep slots'
// keys and values into the retained cache in rank order, zero-filling the
// segment up to the next multiple of 64 slots.  With an E4M3 output every
// 64-slot block gets one float32 scale amax/448 for K and one for V and its
// values are encoded round-to-nearest-even, saturating.
#include <cuda_fp8.h>

#include "kernels.h"

namespace st {

constexpr int kRetainThreads = 256;

__device__ __forceinline__ uint64_t score_key(float f, uint32_t idx, int32_t* status) {
  if (f != f) {                       // NaN: report, and rank it last
    atomicExch(status, ST_ENAN);
    return 0xFFFFFFFF00000000ull | idx;
  }
  if (f == 0.0f) f = 0.0f;            // -0 == +0
  uint32_t u = __float_as_uint(f);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // ascending u <=> ascending f
  return ((uint64_t)(~u) << 32) | idx;               // ascending key <=> descending f
}

template <typename in_t>
__device__ void sort_segment(const RetainParams& p, int t, int lg, uint64_t* keys, int& L,
                             int64_t& a) {
  a = p.off[t];
  L = (int)(p.off[t + 1] - a);
  int npow = 1;
  while (npow < L) npow <<= 1;
  const float* sc = p.scores + (int64_t)lg * p.R + a;
  for (int i = threadIdx.x; i < npow; i += blockDim.x)
    keys[i] = i < L ? score_key(sc[i], (uint32_t)i, p.status) : ~0ull;
  __syncthreads();
  for (int k = 2; k <= npow; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t x = keys[i], y = keys[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) { keys[i] = y; keys[ixj] = x; }
        }
      }
      __syncthreads();
    }
  }
  int32_t* rk = p.rank + (int64_t)lg * p.R + a;
  for (int i = threadIdx.x; i < L; i += blockDim.x) rk[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
}

template <typename T>
__global__ void __launch_bounds__(kRetainThreads) k_retain_copy(RetainParams p) {
  extern __shared__ uint64_t keys[];
  const int t = blockIdx.x, lg = blockIdx.y;
  int L;
  int64_t a;
  sort_segment<T>(p, t, lg, keys, L, a);
  const int n = p.nkeep[t];
  // the retained count within the segment, its padded copy within the capacity
  if (!ST_CHECKED(n >= 0 && n <= L && p.offp[t + 1] - p.offp[t] == (int64_t)((n + 63) & ~63) &&
                      p.offp[t + 1] <= p.Rp_cap,
                  p.status))
    return;
  const int npad = (n + 63) & ~63;
  const int hd = p.hd;
  constexpr int VN = 16 / sizeof(T);
  const int per_row = hd / VN;
  const T* K = reinterpret_cast<const T*>(p.K) + ((int64_t)lg * p.R + a) * hd;
  const T* V = reinterpret_cast<const T*>(p.V) + ((int64_t)lg * p.R + a) * hd;
  T* Kr = reinterpret_cast<T*>(p.Kr) + ((int64_t)lg * p.Rp_cap + p.offp[t]) * hd;
  T* Vr = reinterpret_cast<T*>(p.Vr) + ((int64_t)lg * p.Rp_cap + p.offp[t]) * hd;
  for (int e = threadIdx.x; e < npad * per_row; e += blockDim.x) {
    const int i = e / per_row, c = (e % per_row) * VN;
    uint4 kv = make_uint4(0, 0, 0, 0), vv = make_uint4(0, 0, 0, 0);
    if (i < n) {
      const int64_t src = (int64_t)(keys[i] & 0xFFFFFFFFu) * hd + c;
      kv = *reinterpret_cast<const uint4*>(K + src);
      vv = *reinterpret_cast<const uint4*>(V + src);
    }
    *reinterpret_cast<uint4*>(Kr + (int64_t)i * hd + c) = kv;
    *reinterpret_cast<uint4*>(Vr + (int64_t)i * hd + c) = vv;
  }
}

// E4M3 output from a bf16 cache: per 64-slot block, amax -> scale -> codes.
__global__ void __launch_bounds__(kRetainThreads) k_retain_e4m3(RetainParams p) {
  extern __shared__ uint64_t keys[];
  __shared__ float red[2][kRetainThreads / 32];
  const int t = blockIdx.x, lg = blockIdx.y;
  int L;
  int64_t a;
  sort_segment<bf16>(p, t, lg, keys, L, a);
  const int n = p.nkeep[t];
  // the retained count within the segment, its padded copy within the capacity
  if (!ST_CHECKED(n >= 0 && n <= L && p.offp[t + 1] - p.offp[t] == (int64_t)((n + 63) & ~63) &&
                      p.offp[t + 1] <= p.Rp_cap,
                  p.status))
    return;
  const int nblk = (n + 63) >> 6;
  const int hd = p.hd;                // 64: one block = 64 rows x 64 dims = 4096 values
  const bf16* K = reinterpret_cast<const bf16*>(p.K) + ((int64_t)lg * p.R + a) * hd;
  const bf16* V = reinterpret_cast<const bf16*>(p.V) + ((int64_t)lg * p.R + a) * hd;
  uint8_t* Kr = reinterpret_cast<uint8_t*>(p.Kr) + ((int64_t)lg * p.Rp_cap + p.offp[t]) * hd;
  uint8_t* Vr = reinterpret_cast<uint8_t*>(p.Vr) + ((int64_t)lg * p.Rp_cap + p.offp[t]) * hd;
  float* sc = p.scales + ((int64_t)lg * (p.Rp_cap >> 6) + (p.offp[t] >> 6)) * 2;
  const int per_thread = 64 * hd / kRetainThreads;   // 16 for hd = 64
  for (int b = 0; b < nblk; ++b) {
    float kx[16], vx[16];
    float kmax = 0.f, vmax = 0.f;
    const int e0 = threadIdx.x * per_thread;          // 16 consecutive values of one row
    const int i = b * 64 + e0 / hd, c = e0 % hd;
    if (i < n) {
      const int64_t src = (int64_t)(keys[i] & 0xFFFFFFFFu) * hd + c;
      Vec<bf16>::load(K + src, kx);
      Vec<bf16>::load(K + src + 8, kx + 8);
      Vec<bf16>::load(V + src, vx);
      Vec<bf16>::load(V + src + 8, vx + 8);
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e) kx[e] = vx[e] = 0.f;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      kmax = fmaxf(kmax, fabsf(kx[e]));
      vmax = fmaxf(vmax, fabsf(vx[e]));
    }
    kmax = warp_max(kmax);
    vmax = warp_max(vmax);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = kmax;
      red[1][threadIdx.x >> 5] = vmax;
    }
    __syncthreads();
    kmax = 0.f;
    vmax = 0.f;
#pragma unroll
    for (int w = 0; w < kRetainThreads / 32; ++w) {
      kmax = fmaxf(kmax, red[0][w]);
      vmax = fmaxf(vmax, red[1][w]);
    }
    __syncthreads();
    const float ks = kmax == 0.f ? 1.f : kmax / 448.0f;
    const float vs = vmax == 0.f ? 1.f : vmax / 448.0f;
    uint8_t kc[16], vc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      kc[e] = (uint8_t)__nv_cvt_float_to_fp8(kx[e] / ks, __NV_SATFINITE, __NV_E4M3);
      vc[e] = (uint8_t)__nv_cvt_float_to_fp8(vx[e] / vs, __NV_SATFINITE, __NV_E4M3);
    }
    *reinterpret_cast<uint4*>(Kr + (int64_t)i * hd + c) = *reinterpret_cast<uint4*>(kc);
    *reinterpret_cast<uint4*>(Vr + (int64_t)i * hd + c) = *reinterpret_cast<uint4*>(vc);
    if (threadIdx.x == 0) {
      sc[2 * b] = ks;
      sc[2 * b + 1] = vs;
    }
  }
}

int retain(const RetainParams& p, cudaStream_t s) {
  int npow = 1;
  while (npow < p.max_len) npow <<= 1;
  const size_t smem = (size_t)npow * sizeof(uint64_t);
  dim3 grid(p.T, p.layers * p.hkv);
  if (p.out_dtype == ST_E4M3) {
    if (p.in_dtype != ST_BF16 || p.hd != 64) return ST_EUNSUPPORTED;
    cudaFuncSetAttribute(k_retain_e4m3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_retain_e4m3<<<grid, kRetainThreads, smem, s>>>(p);
  } else if (p.in_dtype == ST_BF16) {
    cudaFuncSetAttribute(k_retain_copy<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_retain_copy<bf16><<<grid, kRetainThreads, smem, s>>>(p);
  } else {
    cudaFuncSetAttribute(k_retain_copy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_retain_copy<float><<<grid, kRetainThreads, smem, s>>>(p);
  }
  return ST_OK;
}

// The retained slot indices of every (layer, kv head, tuple) at a fraction r,
// compacted: the first n_t entries of the tuple's rank-ordered segment (the
// ranking covers the whole segment, so every r reads a prefix of it).
__global__ void k_gather_indices(const int32_t* __restrict__ rank, const int64_t* __restrict__ doc_off,
                                 const int64_t* __restrict__ out_off, int64_t R, int64_t Rn,
                                 int32_t* __restrict__ idx, int* status) {
  const int t = blockIdx.x, lg = blockIdx.y;
  const int64_t o = out_off[t];
  const int n = (int)(out_off[t + 1] - o);
  // the indices copied lie in the tuple's rank segment, the output in the index array
  if (!ST_CHECKED(n >= 0 && n <= doc_off[t + 1] - doc_off[t] && o + n <= Rn, status)) return;
  const int32_t* src = rank + (int64_t)lg * R + doc_off[t];
  int32_t* dst = idx + (int64_t)lg * Rn + o;
  for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
}

void gather_indices(const int32_t* rank, const int64_t* doc_off, const int64_t* out_off, int T, int LH,
                    int64_t R, int64_t Rn, int32_t* idx, int* status, cudaStream_t s) {
  if (T <= 0 || LH <= 0 || Rn <= 0) return;
  k_gather_indices<<<dim3((unsigned)T, (unsigned)LH), 128, 0, s>>>(rank, doc_off, out_off, R, Rn, idx, status);
}

}  // namespace st
