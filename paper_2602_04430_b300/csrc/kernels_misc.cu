// Row bookkeeping, embedding, RMSNorm, EA-lite statistics / scores, pooling and
// the label head.  All of these are bandwidth-bound elementwise or reduction
// kernels; the projections and attention live in their own files.
#include "kernels.h"

namespace st {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int n_keep_dev(int L, double r) {
  // clamp(floor(r*L + 0.5), 1, L); the product and the sum are rounded separately
  // (no fused multiply-add) so that host and device agree bit for bit.
  double rl = __dmul_rn(r, (double)L);
  double f = floor(__dadd_rn(rl, 0.5));
  int n = (int)f;
  return n < 1 ? 1 : (n > L ? L : n);
}

template <int BLOCK>
__device__ __forceinline__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = (threadIdx.x < BLOCK / 32) ? red[threadIdx.x] : 0.f;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  return red[0];
}

// ------------------------------------------------------------------ row info
__global__ void k_build_rowinfo(const int64_t* __restrict__ off, int t0, int t1, int64_t r0,
                                int64_t rows, int32_t* __restrict__ rowtup,
                                int32_t* __restrict__ pos) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= rows) return;
  int64_t g = r0 + m;
  int lo = t0, hi = t1 - 1;          // last t with off[t] <= g
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  rowtup[m] = lo;
  pos[m] = (int32_t)(g - off[lo]);
}

void build_rowinfo(const int64_t* off, int t0, int t1, int64_t r0, int64_t rows, int32_t* rowtup,
                   int32_t* pos, cudaStream_t s) {
  if (rows <= 0) return;
  k_build_rowinfo<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(off, t0, t1, r0, rows, rowtup, pos);
}

// Operator k of an operator set owning global pair gp (pairs are laid out
// operator after operator).
__device__ __forceinline__ int op_of_pair(const OpSet& os, int gp) {
  int k = 0;
  while (k + 1 < os.n_ops && gp >= os.op[k + 1].pair0) ++k;
  return k;
}
__device__ __forceinline__ int op_of_row(const OpSet& os, int64_t gr) {
  int k = 0;
  while (k + 1 < os.n_ops && gr >= os.op[k + 1].row0) ++k;
  return k;
}

// The tuple id at position j of operator o, checked against [0, T): an id
// outside it is recorded in *status and evaluated as tuple 0, so that no read
// leaves the cache.
__device__ __forceinline__ int checked_tuple(const OpSet& os, const OpDev& o, int j, int* status) {
  const int t = o.tuple_ids[j];
  if ((unsigned)t < (unsigned)os.T) return t;
  atomicCAS(status, ST_OK, ST_ERANGE);
  return 0;
}

// Thread per pair of [p0, p0 + np): tuple, length, retained count n_keep(L, r)
// of its operator, prompt row (relative to row_base), prompt length, operator,
// index within the operator.
__global__ void k_eval_pairs(OpSet os, int p0, int np, int64_t row_base,
                             const int64_t* __restrict__ off, int32_t* tup, int32_t* len,
                             int32_t* nk, int32_t* prow, int32_t* pP, int32_t* pop, int32_t* pj,
                             int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int gp = p0 + i, k = op_of_pair(os, gp);
  const OpDev& o = os.op[k];
  const int j = gp - o.pair0;
  const int t = checked_tuple(os, o, j, status);
  const int L = (int)(off[t + 1] - off[t]);
  tup[i] = t;
  len[i] = L;
  nk[i] = n_keep_dev(L, o.r);
  prow[i] = (int32_t)(o.row0 + (int64_t)j * o.P - row_base);
  pP[i] = o.P;
  pop[i] = k;
  pj[i] = j;
}

// Thread per prompt row of [row_base, row_base + rows): RoPE position L_t + p,
// the prompt token, and the row's pair (relative to p0).
__global__ void k_eval_rows(OpSet os, int p0, int64_t row_base, int64_t rows,
                            const int64_t* __restrict__ off, int32_t* pos, int32_t* tok,
                            int32_t* rowpair, int* status) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= rows) return;
  const int64_t gr = row_base + m;
  const int k = op_of_row(os, gr);
  const OpDev& o = os.op[k];
  const int j = (int)((gr - o.row0) / o.P), p = (int)((gr - o.row0) % o.P);
  const int t = checked_tuple(os, o, j, status);
  pos[m] = (int32_t)(off[t + 1] - off[t]) + p;
  tok[m] = o.prompt[p];
  rowpair[m] = o.pair0 + j - p0;
}

void eval_pairs(const OpSet& os, int p0, int np, int64_t row_base, const int64_t* off, int32_t* tup,
                int32_t* len, int32_t* nk, int32_t* prow, int32_t* pP, int32_t* pop, int32_t* pj,
                int* status, cudaStream_t s) {
  if (np <= 0) return;
  k_eval_pairs<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(os, p0, np, row_base, off, tup, len, nk,
                                                           prow, pP, pop, pj, status);
}
void eval_rows(const OpSet& os, int p0, int64_t row_base, int64_t rows, const int64_t* off,
               int32_t* pos, int32_t* tok, int32_t* rowpair, int* status, cudaStream_t s) {
  if (rows <= 0) return;
  k_eval_rows<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(os, p0, row_base, rows, off, pos, tok,
                                                             rowpair, status);
}

// Attention work list: every pair contributes ceil(P G / 128) entries (pair,
// 128-row block, as decoded records), grouped longest retained document first (a counting sort on
// the 128-key tile count, capped at 1023), so that a persistent grid walking
// the list ends with its shortest items (sorted = 0: one bucket, arrival
// order).  One block of 1024 threads; the order within a bucket is arbitrary.
__global__ void __launch_bounds__(1024) k_eval_worklist(const int32_t* __restrict__ nk,
                                                        const int32_t* __restrict__ pP,
                                                        const int32_t* __restrict__ tup,
                                                        const int32_t* __restrict__ prow,
                                                        const int64_t* __restrict__ offp, int n, int G,
                                                        int nq, int sorted, int32_t* list, int split_keys,
                                                        int32_t* psplit, int32_t* mlist, int32_t* gcnt) {
  __shared__ int cnt[1024];
  __shared__ int wsum[32];
  __shared__ int slots, merges, total;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  cnt[tid] = 0;
  if (tid == 0) slots = merges = total = 0;
  __syncthreads();
  const bool split = split_keys > 0 && nq == 0;
  auto zblocks = [&](int i) { return ((nq > 0 ? nq : pP[i]) * G + 127) / 128; };
  auto pieces = [&](int i) { return min((nk[i] + split_keys - 1) / split_keys, 255); };
  // split pairs: reserve their partial-result slots (pieces x row blocks) while they last
  if (split)
    for (int i = tid; i < n; i += 1024) {
      int base = -1;
      if (nk[i] > split_keys) {
        const int need = pieces(i) * zblocks(i);
        const int b = atomicAdd(&slots, need);
        if (b + need <= SPLIT_SLOTS) base = b;
      }
      psplit[i] = base;
    }
  __syncthreads();
  auto np_of = [&](int i) { return (split && psplit[i] >= 0) ? pieces(i) : 1; };
  auto bucket = [&](int i) {
    const int keys = np_of(i) > 1 ? split_keys : nk[i];   // the longest piece of the pair
    return sorted ? 1023 - min((keys + 127) / 128, 1023) : 0;
  };
  for (int i = tid; i < n; i += 1024) {
    atomicAdd(&cnt[bucket(i)], zblocks(i) * np_of(i));
    atomicAdd(&total, zblocks(i) * np_of(i));
  }
  __syncthreads();
  // exclusive prefix sum over the buckets
  const int x = cnt[tid];
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int ws = wsum[lane], wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - ws;
  }
  __syncthreads();
  cnt[tid] = wsum[wid] + inc - x;
  __syncthreads();
  for (int i = tid; i < n; i += 1024) {
    const int nz = zblocks(i), npc = np_of(i);
    const int at = atomicAdd(&cnt[bucket(i)], nz * npc);
    const int64_t o = offp[tup[i]];
    const int base = npc > 1 ? psplit[i] : -1;
    for (int z = 0; z < nz; ++z) {
      for (int pc = 0; pc < npc; ++pc) {
        int4* e = reinterpret_cast<int4*>(list + (int64_t)WORK_INTS * (at + z * npc + pc));
        e[0] = make_int4(i, z | (pc << 8) | (npc << 16), pP[i], nk[i]);
        e[1] = make_int4(prow[i], base >= 0 ? base + z * npc + pc : -1, (int)(uint32_t)o, (int)(o >> 32));
      }
      if (base >= 0) {
        const int m = atomicAdd(&merges, 1);
        reinterpret_cast<int4*>(mlist)[m] = make_int4(i, z, base + z * npc, npc);
      }
    }
  }
  __syncthreads();
  if (tid == 0 && gcnt) {
    gcnt[0] = min(slots, SPLIT_SLOTS);
    gcnt[1] = merges;
    gcnt[2] = total;   // entries of the list (the attention's work count)
  }
}

void eval_worklist(const int32_t* nk, const int32_t* pP, const int32_t* tup, const int32_t* prow,
                   const int64_t* offp, int np, int G, int nq, bool longest_first, int32_t* list,
                   int split_keys, int32_t* psplit, int32_t* mlist, int32_t* cnt, cudaStream_t s) {
  if (np <= 0) return;
  if (!psplit || !mlist || !cnt) split_keys = 0;
  k_eval_worklist<<<1, 1024, 0, s>>>(nk, pP, tup, prow, offp, np, G, nq, longest_first ? 1 : 0, list, split_keys,
                                     psplit, mlist, cnt);
}

// Split-KV merge.  Block (merge entry e, kv head g), thread = query row r of
// the entry's row block: the pieces' partial rows (O_s unnormalised, running
// max m_s in the softmax's scaled log2 units, row sum l_s) combine as
// O = sum_s 2^(m_s - M) O_s / sum_s 2^(m_s - M) l_s with M = max_s m_s, written
// as the f16 output row the unsplit item would have written.
__global__ void __launch_bounds__(128) k_split_merge(const int32_t* __restrict__ mlist,
                                                     const int32_t* __restrict__ cnt,
                                                     const float* __restrict__ part,
                                                     const int32_t* __restrict__ prow,
                                                     const int32_t* __restrict__ pP, int G, int hq, int hkv,
                                                     __half* __restrict__ o) {
  const int e = blockIdx.x, g = blockIdx.y, r = threadIdx.x;
  if (e >= cnt[1]) return;
  const int4 m4 = reinterpret_cast<const int4*>(mlist)[e];
  const int i = m4.x, z = m4.y, slot0 = m4.z, ns = m4.w;
  const int rows = min(128, pP[i] * G - z * 128);
  if (r >= rows) return;
  auto row_of = [&](int sidx) { return part + (((int64_t)(slot0 + sidx) * hkv + g) * 128 + r) * SPLIT_STRIDE; };
  float M = -INFINITY;
  for (int sidx = 0; sidx < ns; ++sidx) M = fmaxf(M, row_of(sidx)[64]);
  float acc[64];
#pragma unroll
  for (int c = 0; c < 64; ++c) acc[c] = 0.f;
  float L = 0.f;
  for (int sidx = 0; sidx < ns; ++sidx) {
    const float* pr = row_of(sidx);
    const float w = exp2f(pr[64] - M);
    L += w * pr[65];
#pragma unroll
    for (int c = 0; c < 64; c += 4) {
      const float4 v = *reinterpret_cast<const float4*>(pr + c);
      acc[c] += w * v.x;
      acc[c + 1] += w * v.y;
      acc[c + 2] += w * v.z;
      acc[c + 3] += w * v.w;
    }
  }
  const float inv = L > 0.f ? 1.f / L : 0.f;
  const int rr = z * 128 + r;
  const int64_t orow = ((int64_t)prow[i] + rr / G) * hq + (int64_t)g * G + rr % G;
  __half2* dst = reinterpret_cast<__half2*>(o + orow * 64);
#pragma unroll
  for (int c = 0; c < 64; c += 2) dst[c / 2] = __floats2half2_rn(acc[c] * inv, acc[c + 1] * inv);
}

void split_merge(const int32_t* mlist, const int32_t* cnt, const float* part, const int32_t* prow,
                 const int32_t* pP, int G, int hq, int hkv, __half* o, cudaStream_t s) {
  k_split_merge<<<dim3(SPLIT_SLOTS, (unsigned)hkv), 128, 0, s>>>(mlist, cnt, part, prow, pP, G, hq, hkv, o);
}

// Retained counts and padded (64-slot) offsets of every tuple, one block.
__global__ void k_nkeep_offp(const int64_t* __restrict__ off, int T, double r, int32_t* nkeep,
                             int64_t* offp) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) { carry = 0; offp[0] = 0; }
  __syncthreads();
  for (int base = 0; base < T; base += 1024) {
    int t = base + threadIdx.x;
    int64_t v = 0;
    if (t < T) {
      int L = (int)(off[t + 1] - off[t]);
      int n = n_keep_dev(L, r);
      nkeep[t] = n;
      v = (n + 63) & ~63;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {           // inclusive Hillis-Steele scan
      int64_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (t < T) offp[t + 1] = carry + part[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
}

void nkeep_offp(const int64_t* off, int T, double r, int32_t* nkeep, int64_t* offp,
                cudaStream_t s) {
  k_nkeep_offp<<<1, 1024, 0, s>>>(off, T, r, nkeep, offp);
}

// ------------------------------------------------------------------ embedding
// x[m] = E[tok[m]] (float32 residual stream).  A token id outside
// [0, vocab) embeds as zeros and records ST_EINVAL in *status.
template <typename act_t>
__global__ void k_embed(const int32_t* __restrict__ tok, int64_t rows, const act_t* __restrict__ E, int d,
                        int vocab, float* __restrict__ x, int* status) {
  const int per = d / 4;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * per) return;
  int64_t m = i / per;
  int c = (int)(i % per) * 4;
  const int t = tok[m];
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (t >= 0 && t < vocab) {
    const act_t* e = E + (int64_t)t * d + c;
    v = make_float4(to_f(e[0]), to_f(e[1]), to_f(e[2]), to_f(e[3]));
  } else if (c == 0) {
    atomicCAS(status, ST_OK, ST_EINVAL);
  }
  *reinterpret_cast<float4*>(x + m * d + c) = v;
}

template <typename act_t>
void embed_rows(const int32_t* tok, int64_t rows, const act_t* E, int d, int vocab, float* x, int* status,
                cudaStream_t s) {
  int64_t n = rows * (d / 4);
  if (n <= 0) return;
  k_embed<act_t><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tok, rows, E, d, vocab, x, status);
}
template void embed_rows<float>(const int32_t*, int64_t, const float*, int, int, float*, int*, cudaStream_t);
template void embed_rows<bf16>(const int32_t*, int64_t, const bf16*, int, int, float*, int*, cudaStream_t);

// ------------------------------------------------------------------ RMSNorm
__device__ __forceinline__ void store4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void store4(__half* p, float4 v) {
  __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&a);
  u.y = *reinterpret_cast<uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void store4(bf16* p, float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&a);
  u.y = *reinterpret_cast<uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

// One warp per row; x float32 [rows][d] -> xn = x / sqrt(mean(x^2) + eps) (act type).
template <typename act_t>
__global__ void k_rmsnorm(const float* __restrict__ x, int64_t rows, int d, float eps,
                          act_t* __restrict__ xn, float* __restrict__ inv_rms, int64_t x_ld) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* xr = x + row * x_ld;
  float ss = 0.f;
  for (int c = lane * 4; c < d; c += 128) {
    float4 v = *reinterpret_cast<const float4*>(xr + c);
    ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  ss = warp_sum(ss);
  float inv = 1.0f / sqrtf(ss / (float)d + eps);
  if (inv_rms != nullptr && lane == 0) inv_rms[row] = inv;
  if (xn == nullptr) return;
  act_t* o = xn + row * d;
  for (int c = lane * 4; c < d; c += 128) {
    float4 v = *reinterpret_cast<const float4*>(xr + c);
    store4(o + c, make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv));
  }
}

template <typename act_t>
void rmsnorm_rows(const float* x, int64_t rows, int d, float eps, act_t* xn, float* inv_rms,
                  cudaStream_t s, int64_t x_ld) {
  if (rows <= 0) return;
  k_rmsnorm<act_t><<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(x, rows, d, eps, xn, inv_rms,
                                                              x_ld > 0 ? x_ld : d);
}
template void rmsnorm_rows<float>(const float*, int64_t, int, float, float*, float*, cudaStream_t,
                                  int64_t);
template void rmsnorm_rows<bf16>(const float*, int64_t, int, float, bf16*, float*, cudaStream_t,
                                 int64_t);
template void rmsnorm_rows<__half>(const float*, int64_t, int, float, __half*, float*, cudaStream_t,
                                 int64_t);

// Embedding gather fused with the first layer's RMSNorm (BF16 model), one warp
// per row: x = E[tok] in float32 (the residual stream) and xn = x / rms(x) in
// half.  Each lane sums its squares in k_rmsnorm's order, so xn equals the
// gather followed by k_rmsnorm bit for bit; the second pass re-reads the
// embedding row (an L2 hit) instead of the float32 row just written.
__device__ __forceinline__ float4 load4_bf16(const bf16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__global__ void k_embed_norm(const int32_t* __restrict__ tok, int64_t rows, const bf16* __restrict__ E, int d,
                             int vocab, float eps, float* __restrict__ x, __half* __restrict__ xn,
                             int* status) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const int t = tok[row];
  const bool ok = t >= 0 && t < vocab;
  if (!ok && lane == 0) atomicCAS(status, ST_OK, ST_EINVAL);
  const bf16* er = E + (int64_t)(ok ? t : 0) * d;
  float* xr = x + row * d;
  float ss = 0.f;
  for (int c = lane * 4; c < d; c += 128) {
    const float4 v = ok ? load4_bf16(er + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(xr + c) = v;
    ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  ss = warp_sum(ss);
  const float inv = 1.0f / sqrtf(ss / (float)d + eps);
  __half* o = xn + row * d;
  for (int c = lane * 4; c < d; c += 128) {
    const float4 v = ok ? load4_bf16(er + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    store4(o + c, make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv));
  }
}

void embed_norm_rows(const int32_t* tok, int64_t rows, const bf16* E, int d, int vocab, float eps, float* x,
                     __half* xn, int* status, cudaStream_t s) {
  if (rows <= 0) return;
  k_embed_norm<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(tok, rows, E, d, vocab, eps, x, xn, status);
}

// ------------------------------------------------------------------ EA-lite statistics
// Block per (tuple, kv head): mean and population variance over (document
// position, query head of the group) of every post-RoPE query dimension.
// One pass, shifted by the group's first query vector for stability:
// mean = shift + S1/N, var = S2/N - (S1/N)^2 with S1 = sum(q - shift),
// S2 = sum((q - shift)^2).  Each thread reads 16-byte vectors (VN dims) of
// consecutive (position, head) items, so a warp reads whole rows.
template <typename act_t>
__global__ void __launch_bounds__(256) k_qstats(const act_t* __restrict__ q,
                                                const int64_t* __restrict__ off, int t0, int64_t r0,
                                                int hq, int hkv, int hd, float* __restrict__ mu,
                                                float* __restrict__ s2) {
  constexpr int VN = Vec<act_t>::N;           // dims per 16-byte vector
  __shared__ float red[2][256][VN];
  const int t = t0 + blockIdx.x / hkv, g = blockIdx.x % hkv;
  const int G = hq / hkv;
  const int64_t row0 = off[t] - r0;
  const int L = (int)(off[t + 1] - off[t]);
  const int chunks = hd / VN;                  // threads per item
  const int lanes = blockDim.x / chunks;       // items in flight per iteration
  const int ch = threadIdx.x % chunks, il = threadIdx.x / chunks;
  const int64_t items = (int64_t)L * G;
  const act_t* base = q + row0 * hq * hd + (int64_t)g * G * hd + ch * VN;
  float shift[VN], a1[VN], a2[VN], v[VN];
  Vec<act_t>::load(base, shift);               // the group's first query vector
#pragma unroll
  for (int e = 0; e < VN; ++e) a1[e] = a2[e] = 0.f;
  // eight 16-byte loads per thread in flight (kept raw until accumulated):
  // the kernel is bound by the bytes in flight per SM
  auto acc = [&](const uint4& raw) {
    float w[VN];
    Vec<act_t>::unpack(raw, w);
#pragma unroll
    for (int e = 0; e < VN; ++e) {
      const float dv = w[e] - shift[e];
      a1[e] += dv;
      a2[e] = fmaf(dv, dv, a2[e]);
    }
  };
  int64_t it = il;
  for (; it + 7 * lanes < items; it += 8 * lanes) {
    uint4 raw[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t iu = it + u * lanes, j = iu / G, hh = iu % G;
      raw[u] = ldg_stream(reinterpret_cast<const uint4*>(base + j * hq * hd + hh * hd));
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc(raw[u]);
  }
  for (; it < items; it += lanes) {
    const int64_t j = it / G, hh = it % G;
    acc(ldg_stream(reinterpret_cast<const uint4*>(base + j * hq * hd + hh * hd)));
  }
  (void)v;
#pragma unroll
  for (int e = 0; e < VN; ++e) {
    red[0][threadIdx.x][e] = a1[e];
    red[1][threadIdx.x][e] = a2[e];
  }
  __syncthreads();
  if (il == 0) {
#pragma unroll
    for (int e = 0; e < VN; ++e) {
      float s1 = 0.f, sq = 0.f;
      for (int k = 0; k < lanes; ++k) {
        s1 += red[0][k * chunks + ch][e];
        sq += red[1][k * chunks + ch][e];
      }
      const float m1 = s1 / (float)items;
      const int64_t o = ((int64_t)(t - t0) * hkv + g) * hd + ch * VN + e;
      mu[o] = shift[e] + m1;
      s2[o] = fmaxf(sq / (float)items - m1 * m1, 0.f);
    }
  }
}

template <typename act_t>
void qstats(const act_t* q, const int64_t* off, int t0, int t1, int64_t r0, int hq, int hkv,
            int hd, float* mu, float* s2, cudaStream_t s) {
  int nb = (t1 - t0) * hkv;
  if (nb <= 0) return;
  k_qstats<act_t><<<nb, 256, 0, s>>>(q, off, t0, r0, hq, hkv, hd, mu, s2);
}
template void qstats<float>(const float*, const int64_t*, int, int, int64_t, int, int, int, float*,
                            float*, cudaStream_t);
template void qstats<bf16>(const bf16*, const int64_t*, int, int, int64_t, int, int, int, float*,
                           float*, cudaStream_t);

// score = mu.k/sqrt(hd) + sum sigma2 k^2/(2hd) + ln(||v|| + 1e-12) per (kv head,
// slot).  TPR = hd / VN threads share a slot, each reading one 16-byte vector of
// its K and V rows (a warp reads whole rows); the two terms that are linear in
// the partial sums are combined per thread, so two sums are shuffle-reduced.
template <typename act_t>
__global__ void __launch_bounds__(256) k_scores(const act_t* __restrict__ K, const act_t* __restrict__ V,
                                                int64_t R, int hkv, int hd, int64_t r0, int64_t rows,
                                                const int32_t* __restrict__ rowtup, int t0,
                                                const float* __restrict__ mu, const float* __restrict__ s2,
                                                float* __restrict__ scores) {
  constexpr int VN = Vec<act_t>::N;
  const int tpr = hd / VN;                      // threads per slot (a power of two <= 32)
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / tpr;
  const int c = (threadIdx.x % tpr) * VN;
  const bool live = i < rows * hkv;
  float d1 = 0.f, d2 = 0.f, vv = 0.f;
  const float c1 = 1.f / sqrtf((float)hd), c2 = 1.f / (2.0f * (float)hd);
  int g = 0;
  int64_t m = 0;
  if (live) {
    g = (int)(i / rows);
    m = i % rows;
    const int lt = rowtup[m] - t0;
    float kk[VN], vx[VN];
    Vec<act_t>::load(K + ((int64_t)g * R + r0 + m) * hd + c, kk);
    Vec<act_t>::load(V + ((int64_t)g * R + r0 + m) * hd + c, vx);
    const float* mup = mu + ((int64_t)lt * hkv + g) * hd + c;
    const float* s2p = s2 + ((int64_t)lt * hkv + g) * hd + c;
#pragma unroll
    for (int e = 0; e < VN; ++e) {
      d1 += mup[e] * kk[e];
      d2 += s2p[e] * kk[e] * kk[e];
      vv += vx[e] * vx[e];
    }
  }
  float lin = d1 * c1 + d2 * c2;
  for (int o = tpr / 2; o > 0; o >>= 1) {
    lin += __shfl_xor_sync(0xffffffffu, lin, o);
    vv += __shfl_xor_sync(0xffffffffu, vv, o);
  }
  if (live && c == 0) scores[(int64_t)g * R + r0 + m] = lin + logf(sqrtf(vv) + 1e-12f);
}

template <typename act_t>
void ea_scores(const act_t* K, const act_t* V, int64_t R, int hkv, int hd, int64_t r0,
               int64_t rows, const int32_t* rowtup, int t0, const float* mu, const float* s2,
               float* scores, cudaStream_t s) {
  const int64_t n = rows * hkv * (hd / Vec<act_t>::N);   // threads
  if (n <= 0) return;
  k_scores<act_t><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(K, V, R, hkv, hd, r0, rows, rowtup,
                                                              t0, mu, s2, scores);
}
template void ea_scores<float>(const float*, const float*, int64_t, int, int, int64_t, int64_t,
                               const int32_t*, int, const float*, const float*, float*,
                               cudaStream_t);
template void ea_scores<bf16>(const bf16*, const bf16*, int64_t, int, int, int64_t, int64_t,
                              const int32_t*, int, const float*, const float*, float*,
                              cudaStream_t);

// ------------------------------------------------------------------ pooling
// Block per tuple: pooled[t] = mean over document rows of the final-normed
// state x[m] / rms(x[m]).  1/rms comes from inv_rms, or (inv_rms == nullptr)
// from the residual epilogue's partial sums of squares ssq[m][parts], for 2048
// rows at a time into shared memory.  A thread owns 4 consecutive columns
// (16-byte loads) and keeps four rows in flight.
__global__ void __launch_bounds__(256) k_pool(const float* __restrict__ x, const float* __restrict__ inv_rms,
                                              const float* __restrict__ ssq, int parts, float eps,
                                              const int64_t* __restrict__ off, int t0, int64_t r0, int d,
                                              float* __restrict__ pooled) {
  constexpr int RB = 2048;
  __shared__ float inv_s[RB];
  const int t = t0 + blockIdx.x;
  const int64_t a = off[t] - r0, b = off[t + 1] - r0;
  const int L = (int)(b - a);
  for (int c0 = 0; c0 < d; c0 += blockDim.x * 4) {
    const int c = c0 + threadIdx.x * 4;
    float4 acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int m0 = 0; m0 < L; m0 += RB) {
      const int nb = min(RB, L - m0);
      __syncthreads();
      for (int m = threadIdx.x; m < nb; m += blockDim.x) {
        const int64_t row = a + m0 + m;
        float iv;
        if (inv_rms != nullptr) {
          iv = inv_rms[row];
        } else {
          float sum = 0.f;
          for (int k = 0; k < parts; ++k) sum += ssq[row * parts + k];
          iv = 1.0f / sqrtf(sum / (float)d + eps);
        }
        inv_s[m] = iv;
      }
      __syncthreads();
      if (c < d) {
        const float* xr = x + (a + m0) * d + c;
        int m = 0;
        for (; m + 3 < nb; m += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 v = *reinterpret_cast<const float4*>(xr + (int64_t)(m + u) * d);
            const float iv = inv_s[m + u];
            acc[u].x = fmaf(v.x, iv, acc[u].x);
            acc[u].y = fmaf(v.y, iv, acc[u].y);
            acc[u].z = fmaf(v.z, iv, acc[u].z);
            acc[u].w = fmaf(v.w, iv, acc[u].w);
          }
        }
        for (; m < nb; ++m) {
          const float4 v = *reinterpret_cast<const float4*>(xr + (int64_t)m * d);
          const float iv = inv_s[m];
          acc[0].x = fmaf(v.x, iv, acc[0].x);
          acc[0].y = fmaf(v.y, iv, acc[0].y);
          acc[0].z = fmaf(v.z, iv, acc[0].z);
          acc[0].w = fmaf(v.w, iv, acc[0].w);
        }
      }
    }
    if (c < d) {
      const float inv_l = 1.0f / (float)L;
      float4 o;
      o.x = ((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x)) * inv_l;
      o.y = ((acc[0].y + acc[1].y) + (acc[2].y + acc[3].y)) * inv_l;
      o.z = ((acc[0].z + acc[1].z) + (acc[2].z + acc[3].z)) * inv_l;
      o.w = ((acc[0].w + acc[1].w) + (acc[2].w + acc[3].w)) * inv_l;
      *reinterpret_cast<float4*>(pooled + (int64_t)t * d + c) = o;
    }
  }
}

void pool_rows(const float* x, const float* inv_rms, const float* ssq, int parts, float eps,
               const int64_t* off, int t0, int t1, int64_t r0, int d, float* pooled, cudaStream_t s) {
  if (t1 <= t0) return;
  k_pool<<<t1 - t0, 256, 0, s>>>(x, inv_rms, ssq, parts, eps, off, t0, r0, d, pooled);
}

// ------------------------------------------------------------------ label head
// Block per (operator, tuple) pair: final RMSNorm of its last prompt row, its
// operator's label-token logits, and the decision (filter thresholds or
// classify argmax).
template <typename w_t>
__global__ void k_label_head(const float* __restrict__ x, OpSet os, const int32_t* __restrict__ prow,
                             const int32_t* __restrict__ pP, const int32_t* __restrict__ pop,
                             const int32_t* __restrict__ pj, int d, float eps,
                             const w_t* __restrict__ w_lm, int64_t rows, int* status) {
  __shared__ float red[32];
  __shared__ float z[8];
  const int i = blockIdx.x;
  // the pair's operator, its last prompt row within the chunk's rows
  if (!ST_CHECKED(pop[i] >= 0 && pop[i] < os.n_ops && prow[i] >= 0 && pP[i] >= 1 &&
                      (int64_t)prow[i] + pP[i] <= rows && pj[i] >= 0 && pj[i] < os.op[pop[i]].n,
                  status))
    return;
  const OpDev& o = os.op[pop[i]];
  const float* xr = x + ((int64_t)prow[i] + pP[i] - 1) * d;
  float ss = 0.f;
  for (int c = threadIdx.x; c < d; c += blockDim.x) ss += xr[c] * xr[c];
  ss = block_sum<256>(ss, red);
  const float inv = 1.0f / sqrtf(ss / (float)d + eps);
  for (int k = 0; k < o.n_labels; ++k) {
    const w_t* wr = w_lm + (int64_t)o.labels[k] * d;
    float acc = 0.f;
    for (int c = threadIdx.x; c < d; c += blockDim.x) acc += xr[c] * to_f(wr[c]);
    acc = block_sum<256>(acc, red);
    if (threadIdx.x == 0) z[k] = acc * inv;
  }
  if (threadIdx.x == 0) {
    const int j = pj[i];
    for (int k = 0; k < o.n_labels; ++k) o.logits[(int64_t)j * o.n_labels + k] = z[k];
    int dec;
    if (o.kind == ST_OP_FILTER) {
      float sc = z[0] - z[1];
      float a = sc - o.theta_pos, rj = o.theta_neg - sc, u = 0.f;
      dec = (u >= a && u >= rj) ? ST_UNSURE : (rj >= a ? ST_REJECT : ST_ACCEPT);
    } else {
      dec = 0;
      float best = z[0] + (o.bias ? o.bias[0] : 0.f);
      for (int k = 1; k < o.n_labels; ++k) {
        float v = z[k] + (o.bias ? o.bias[k] : 0.f);
        if (v > best) { best = v; dec = k; }
      }
    }
    o.out_labels[j] = dec;
  }
}

void label_head(const float* x, const OpSet& os, int np, const int32_t* prow, const int32_t* pP,
                const int32_t* pop, const int32_t* pj, int d, float eps, const void* w_lm, int dtype,
                int64_t rows, int* status, cudaStream_t s) {
  if (np <= 0) return;
  if (dtype == ST_BF16)   // the BF16 model holds its LM head as IEEE half
    k_label_head<__half><<<np, 256, 0, s>>>(x, os, prow, pP, pop, pj, d, eps, (const __half*)w_lm, rows, status);
  else
    k_label_head<float><<<np, 256, 0, s>>>(x, os, prow, pP, pop, pj, d, eps, (const float*)w_lm, rows, status);
}

// ------------------------------------------------------------------ weight conversion
__global__ void k_bf16_to_f16(uint32_t* p, size_t n2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = p[i];
    const float lo = __uint_as_float(u << 16), hi = __uint_as_float(u & 0xFFFF0000u);
    __half2 h = __floats2half2_rn(lo, hi);
    p[i] = *reinterpret_cast<uint32_t*>(&h);
  }
}

void bf16_to_f16(void* p, size_t n, cudaStream_t s) {
  // n is even for every weight matrix (dimensions multiples of 64)
  const size_t n2 = n / 2;
  if (n2 == 0) return;
  k_bf16_to_f16<<<(unsigned)std::min<size_t>((n2 + 255) / 256, 4096), 256, 0, s>>>((uint32_t*)p, n2);
}

// ------------------------------------------------------------------ map operator (decode)
// Prompt K/V of one layer from the evaluation layout [pair * P + p][kd] into
// the decode cache [pair][S][kd], 16 bytes per thread: rows p < P copied, rows
// P .. S-1 (the generated tokens' keys, written by later steps) zeroed.  The
// zeros matter: the attention's P.V product runs over whole 32-key chunks of
// the cache, and a zero probability times a non-finite stale value would be NaN.
__global__ void k_copy_prompt_kv(const uint4* __restrict__ src, uint4* __restrict__ dst, int n, int P,
                                 int S, int row_vecs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)n * S * row_vecs;
  if (i >= total) return;
  const int64_t row = i / row_vecs;
  const int c = (int)(i % row_vecs);
  const int64_t pr = row / S, p = row % S;
  dst[i] = p < P ? src[(pr * P + p) * row_vecs + c] : make_uint4(0u, 0u, 0u, 0u);
}

void copy_prompt_kv(const void* src, void* dst, int n, int P, int S, int kd, size_t esz, cudaStream_t s) {
  const int row_vecs = (int)(kd * esz / 16);
  const int64_t total = (int64_t)n * S * row_vecs;
  if (total <= 0) return;
  k_copy_prompt_kv<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const uint4*)src, (uint4*)dst, n, P, S,
                                                                   row_vecs);
}

// Decode step t >= 1 (one query row per pair): pair i's keys are the rows
// i*S .. i*S + P + t - 1 of the decode cache, its query is Q row i at RoPE
// position L_i + P + t - 1, fed the token generated at step t - 1.
__global__ void k_decode_plan(int n, int S, int P, int t, int n_gen, const int32_t* __restrict__ len,
                              const int32_t* __restrict__ tokens, int32_t* prow, int32_t* pP,
                              int32_t* pq0, int32_t* rowpair, int32_t* pos, int32_t* tok) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  prow[i] = i * S;
  pP[i] = P + t;
  pq0[i] = i;
  rowpair[i] = i;
  pos[i] = len[i] + P + t - 1;
  tok[i] = tokens[(int64_t)i * n_gen + t - 1];
}

void decode_plan(int n, int S, int P, int t, int n_gen, const int32_t* len, const int32_t* tokens,
                 int32_t* prow, int32_t* pP, int32_t* pq0, int32_t* rowpair, int32_t* pos, int32_t* tok,
                 cudaStream_t s) {
  if (n <= 0) return;
  k_decode_plan<<<(n + 255) / 256, 256, 0, s>>>(n, S, P, t, n_gen, len, tokens, prow, pP, pq0, rowpair,
                                                pos, tok);
}

// Block per row: the greedy token argmax_v logits[i][v] (ties to the lowest
// v), into tokens[i * n_gen + t]; optionally the row of logits into
// logits_out[(i * n_gen + t) * V ...].  A row without a finite maximum (NaN
// logits) yields token 0 and ST_ENAN in *status, so the next step's embedding
// never reads outside the table.
__global__ void __launch_bounds__(256) k_argmax_rows(const float* __restrict__ logits, int V, int t,
                                                     int n_gen, int32_t* tokens, float* logits_out,
                                                     int* status) {
  __shared__ float bv[256];
  __shared__ int bi[256];
  const int i = blockIdx.x;
  const float* z = logits + (int64_t)i * V;
  float best = -INFINITY;
  int arg = 0x7fffffff;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const float x = z[v];
    if (x > best || (x == best && v < arg)) {
      best = x;
      arg = v;
    }
    if (logits_out) logits_out[((int64_t)i * n_gen + t) * V + v] = x;
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const float x = bv[threadIdx.x + o];
      const int a2 = bi[threadIdx.x + o];
      if (x > bv[threadIdx.x] || (x == bv[threadIdx.x] && a2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = x;
        bi[threadIdx.x] = a2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int tok = bi[0];
    if (tok < 0 || tok >= V) {
      tok = 0;
      atomicCAS(status, ST_OK, ST_ENAN);
    }
    tokens[(int64_t)i * n_gen + t] = tok;
  }
}

void argmax_rows(const float* logits, int n, int V, int t, int n_gen, int32_t* tokens, float* logits_out,
                 int* status, cudaStream_t s) {
  if (n <= 0) return;
  k_argmax_rows<<<n, 256, 0, s>>>(logits, V, t, n_gen, tokens, logits_out, status);
}

// ------------------------------------------------------------------ SwiGLU (float32 path)
// t [rows][2F] with gate/up interleaved in blocks of 128 columns -> h [rows][F].
__global__ void k_swiglu_f32(const float* __restrict__ t, int64_t rows, int ffn,
                             float* __restrict__ h) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ffn) return;
  int64_t m = i / ffn;
  int f = (int)(i % ffn);
  int b = f >> 7, j = f & 127;
  float g = t[m * 2 * ffn + b * 256 + j];
  float u = t[m * 2 * ffn + b * 256 + 128 + j];
  h[i] = silu_f(g) * u;
}

void swiglu_from_f32(const float* t, int64_t rows, int ffn, float* h, cudaStream_t s) {
  int64_t n = rows * ffn;
  if (n <= 0) return;
  k_swiglu_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, rows, ffn, h);
}

}  // namespace st
