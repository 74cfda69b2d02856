// CUDA-core attention for the float32 model: one warp per (query row, query
// head); the lanes stride over the visible keys with their own online softmax
// state and merge it at the end.  Serves both the causal document prefill
// (offline cache creation) and the operator evaluation (retained document
// slots, all visible, followed by the prompt's own keys, causal).
#include "kernels.h"

namespace st {

template <typename T, int HD>
__global__ void __launch_bounds__(256) k_attn_simt(AttnParams a) {
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t nrows = a.mode == 0 ? a.rows : a.qrows;
  if (wid >= nrows * a.hq) return;
  const int64_t qrow = wid / a.hq;
  const int h = (int)(wid % a.hq);
  const int g = h / (a.hq / a.hkv);
  const T* qp = reinterpret_cast<const T*>(a.q) + qrow * a.hq * HD + (int64_t)h * HD;
  float q[HD];
#pragma unroll
  for (int c = 0; c < HD; ++c) q[c] = to_f(qp[c]);

  const T *kA, *vA, *kB = nullptr, *vB = nullptr;
  int nA, nB = 0;
  int64_t sB = 0;
  if (a.mode == 0) {
    const int t = a.rowtup[qrow];
    const int64_t base = ((int64_t)g * a.R + a.off[t]) * HD;
    kA = reinterpret_cast<const T*>(a.K) + base;
    vA = reinterpret_cast<const T*>(a.V) + base;
    nA = a.pos[qrow] + 1;
  } else {
    // query position among the pair's prompt keys: the last nq positions
    const int i = a.rowpair[qrow];
    const int64_t qb = a.pq0 ? a.pq0[i] : a.prow[i];
    const int p = (a.pP[i] - (a.nq > 0 ? a.nq : a.pP[i])) + (int)(qrow - qb);
    const int t = a.tup[i];
    const int64_t base = ((int64_t)g * a.Rp_cap + a.offp[t]) * HD;
    kA = reinterpret_cast<const T*>(a.Kr) + base;
    vA = reinterpret_cast<const T*>(a.Vr) + base;
    nA = a.nk[i];
    sB = (int64_t)a.hkv * HD;
    kB = reinterpret_cast<const T*>(a.kp) + (int64_t)a.prow[i] * sB + (int64_t)g * HD;
    vB = reinterpret_cast<const T*>(a.vp) + (int64_t)a.prow[i] * sB + (int64_t)g * HD;
    nB = p + 1;
  }
  float m = -INFINITY, l = 0.f, acc[HD];
#pragma unroll
  for (int c = 0; c < HD; ++c) acc[c] = 0.f;
  for (int kk = lane; kk < nA + nB; kk += 32) {
    const T* kr = kk < nA ? kA + (int64_t)kk * HD : kB + (int64_t)(kk - nA) * sB;
    const T* vr = kk < nA ? vA + (int64_t)kk * HD : vB + (int64_t)(kk - nA) * sB;
    float sc = 0.f;
#pragma unroll
    for (int c = 0; c < HD; ++c) sc = fmaf(q[c], to_f(kr[c]), sc);
    sc *= a.scale;
    if (sc > m) {
      float corr = expf(m - sc);
      l *= corr;
#pragma unroll
      for (int c = 0; c < HD; ++c) acc[c] *= corr;
      m = sc;
    }
    float p = expf(sc - m);
    l += p;
#pragma unroll
    for (int c = 0; c < HD; ++c) acc[c] = fmaf(p, to_f(vr[c]), acc[c]);
  }
  const float M = warp_max(m);
  const float corr = (m == -INFINITY) ? 0.f : expf(m - M);
  l = warp_sum(l * corr);
  T* op = reinterpret_cast<T*>(a.o) + qrow * a.hq * HD + (int64_t)h * HD;
#pragma unroll
  for (int c = 0; c < HD; ++c) {
    float v = warp_sum(acc[c] * corr);
    if (lane == (c & 31)) op[c] = from_f<T>(v / l);
  }
}

template <typename act_t, typename kv_t>
void attn_simt(const AttnParams& a, cudaStream_t s) {
  const int64_t nrows = a.mode == 0 ? a.rows : a.qrows;
  const int64_t warps = nrows * a.hq;
  if (warps <= 0) return;
  const unsigned grid = (unsigned)((warps + 7) / 8);
  if (a.hd == 64)
    k_attn_simt<act_t, 64><<<grid, 256, 0, s>>>(a);
  else
    k_attn_simt<act_t, 32><<<grid, 256, 0, s>>>(a);
}
template void attn_simt<float, float>(const AttnParams&, cudaStream_t);
template void attn_simt<bf16, bf16>(const AttnParams&, cudaStream_t);

}  // namespace st
