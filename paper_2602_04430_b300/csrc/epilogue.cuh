// Projection epilogues shared by the CUDA-core and tcgen05 GEMMs.
//
// A thread holds W consecutive float32 accumulators of one output row.  For the
// QKV projection W equals the head dim, so a thread owns exactly one head and
// the RoPE rotation pairs (i, i + hd/2) are register-local.
#pragma once

#include "kernels.h"

namespace st {

template <typename act_t, int W>
__device__ __forceinline__ void store_act(act_t* dst, const float (&v)[W]) {
  constexpr int VN = Vec<act_t>::N;
#pragma unroll
  for (int j = 0; j < W; j += VN) Vec<act_t>::store(dst + j, v + j);
}

template <int W>
__device__ __forceinline__ void store_half(__half* dst, const float (&v)[W]) {
#pragma unroll
  for (int j = 0; j < W; j += 8) {
    uint4 u;
    __half2* h = reinterpret_cast<__half2*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(v[j + 2 * i], v[j + 2 * i + 1]);
    *reinterpret_cast<uint4*>(dst + j) = u;
  }
}

template <int W>
__device__ __forceinline__ void rope_inplace(float (&v)[W], const float2* __restrict__ tab) {
#pragma unroll
  for (int i = 0; i < W / 2; ++i) {
    float2 cs = tab[i];
    float a = v[i], b = v[i + W / 2];
    v[i] = a * cs.x - b * cs.y;
    v[i + W / 2] = b * cs.x + a * cs.y;
  }
}

// 1 / rms of output row `row` from the partial sums of squares of the previous
// residual epilogue (1 when the A operand is already normalised).
__device__ __forceinline__ float row_inv_rms(const EpiParams& ep, int row) {
  if (ep.ssq_in == nullptr) return 1.f;
  float s = 0.f;
  for (int k = 0; k < ep.ssq_parts; ++k) s += ep.ssq_in[(int64_t)row * ep.ssq_parts + k];
  return 1.0f / sqrtf(s / (float)ep.norm_d + ep.eps);
}

// Apply the epilogue to columns [col0, col0 + W) of output row `row`; `scale`
// multiplies the accumulators first.  Returns, for EPI_RESID, the sum of the
// squares of the new stream values (0 otherwise).
template <typename act_t, int W>
__device__ __forceinline__ float epilogue_apply(const EpiParams& ep, int row, int col0,
                                                float (&v)[W], float scale = 1.f) {
  if (scale != 1.f) {
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] *= scale;
  }
  if (ep.mode == EPI_QKV) {
    const int qcols = ep.hq * W, kcols = ep.hkv * W;
    if (col0 < qcols + kcols) rope_inplace<W>(v, ep.rope + (int64_t)ep.pos[row] * (W / 2));
    int64_t off;
    void* base;
    if (col0 < qcols) {
      base = ep.q;
      off = (int64_t)row * qcols + col0;
    } else if (col0 < qcols + kcols) {
      base = ep.kbase;
      off = ((col0 - qcols) / W) * ep.kv_sg + row * ep.kv_sr;
    } else {
      base = ep.vbase;
      off = ((col0 - qcols - kcols) / W) * ep.kv_sg + row * ep.kv_sr;
    }
    if (ep.qkv_f16) store_half<W>(reinterpret_cast<__half*>(base) + off, v);
    else store_act<act_t, W>(reinterpret_cast<act_t*>(base) + off, v);
  } else if (ep.mode == EPI_RESID) {
    float* x = ep.x + ((int64_t)row * ep.row_mul + ep.row_add) * ep.ld + col0;
    float ss = 0.f;
#pragma unroll
    for (int j = 0; j < W; j += 4) {
      float4 o = *reinterpret_cast<float4*>(x + j);
      o.x += v[j]; o.y += v[j + 1]; o.z += v[j + 2]; o.w += v[j + 3];
      *reinterpret_cast<float4*>(x + j) = o;
      v[j] = o.x; v[j + 1] = o.y; v[j + 2] = o.z; v[j + 3] = o.w;
      ss += o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
    }
    if (ep.xb != nullptr)
      store_act<bf16, W>(reinterpret_cast<bf16*>(ep.xb) + (int64_t)row * ep.N + col0, v);
    return ss;
  } else if (ep.mode == EPI_STORE_F32) {
    float* o = ep.out + (int64_t)row * ep.ld + col0;
#pragma unroll
    for (int j = 0; j < W; j += 4)
      *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  }
  return 0.f;
}

// SwiGLU: gate accumulators g and up accumulators u of FFN columns [f0, f0 + W).
template <typename act_t, int W>
__device__ __forceinline__ void epilogue_swiglu(const EpiParams& ep, int row, int f0,
                                                const float (&g)[W], const float (&u)[W]) {
  float hv[W];
#pragma unroll
  for (int j = 0; j < W; ++j) hv[j] = silu_f(g[j]) * u[j];
  store_act<act_t, W>(reinterpret_cast<act_t*>(ep.h) + (int64_t)row * ep.ld + f0, hv);
}

}  // namespace st
