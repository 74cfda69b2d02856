// BF16 tensor-core attention (mma.sync m16n8k16, f32 accumulate, online softmax
// in registers) for one kv head at a time, so that every key/value tile staged
// in shared memory serves all G query heads of the group and all query rows of
// the CTA.
//
// Two modes share the kernel body:
//   prefill (offline cache creation): rows = (document position j in a block of
//     128/G positions, query head of the group); keys = the document's own
//     cached keys 0..j (causal).
//   eval (online operator): rows = (prompt position p, query head of the group);
//     keys = the tuple's retained document slots (all visible), then the
//     prompt's own keys 0..p (causal).  Retained slots may be E4M3 codes with one
//     scale per 64-slot block; they are widened exactly to bf16 while staged in
//     shared memory, the K scale multiplies the f32 scores of the tile and the V
//     scale the probabilities fed to the P.V product.
// Shared-memory tiles are 64 rows x 128 bytes with a 16-byte-chunk XOR swizzle
// (chunk ^ row%8) so that ldmatrix is conflict-free.
#include <cuda_fp8.h>

#include "kernels.h"
#include "ptx.cuh"

namespace st {
namespace {

constexpr int HD = 64;
constexpr int KT = 64;            // keys per tile
constexpr int MAX_ROWS = 128;     // query rows per CTA (8 warps x 16)

__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                          uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

struct Tile {
  const void* k;    // first key row of the tile
  const void* v;
  int64_t stride;   // elements between consecutive key rows
  int count;        // valid key rows in this tile (<= 64)
  int key0;         // index of the first key within its segment
  bool prompt;      // keys of the prompt (causal) rather than retained / document slots
  float ks, vs;     // E4M3 block scales (1 for bf16)
};

template <int MODE, bool FP8>
struct Ctx {
  const AttnParams* a;
  int g, rows;
  // eval
  int i, n_doc, P;
  const uint8_t *kr8, *vr8;
  const bf16 *krb, *vrb, *kp, *vp;
  const float* sc;
  // prefill
  int t, j0, L;
  const bf16 *kd, *vd;

  __device__ int n_tiles() const {
    if (MODE == 1) return (n_doc + KT - 1) / KT + (P + KT - 1) / KT;
    const int last = min(j0 + rows / (a->hq / a->hkv), L) - 1;   // last position of the block
    return last / KT + 1;
  }
  __device__ Tile tile(int ti) const {
    Tile T;
    T.ks = T.vs = 1.f;
    if (MODE == 1) {
      const int nd = (n_doc + KT - 1) / KT;
      if (ti < nd) {
        T.prompt = false;
        T.key0 = ti * KT;
        T.count = min(KT, n_doc - T.key0);
        T.stride = HD;
        if (FP8) {
          T.k = kr8 + (int64_t)T.key0 * HD;
          T.v = vr8 + (int64_t)T.key0 * HD;
          T.ks = sc[2 * ti];
          T.vs = sc[2 * ti + 1];
        } else {
          T.k = krb + (int64_t)T.key0 * HD;
          T.v = vrb + (int64_t)T.key0 * HD;
        }
      } else {
        T.prompt = true;
        T.key0 = (ti - nd) * KT;
        T.count = min(KT, P - T.key0);
        T.stride = (int64_t)a->hkv * HD;
        T.k = kp + (int64_t)T.key0 * T.stride;
        T.v = vp + (int64_t)T.key0 * T.stride;
      }
    } else {
      T.prompt = false;
      T.key0 = ti * KT;
      T.count = min(KT, L - T.key0);
      T.stride = HD;
      T.k = kd + (int64_t)T.key0 * HD;
      T.v = vd + (int64_t)T.key0 * HD;
    }
    return T;
  }
};

// Stage one key/value tile into shared memory (bf16, swizzled).  bf16 sources
// go through cp.async; E4M3 sources are widened with their block scale.
template <bool FP8>
__device__ __forceinline__ void stage_tile(const Tile& T, uint32_t sK, uint32_t sV, uint8_t* gK,
                                           uint8_t* gV) {
  if (!FP8 || T.prompt) {
    const bf16* k = reinterpret_cast<const bf16*>(T.k);
    const bf16* v = reinterpret_cast<const bf16*>(T.v);
    for (int e = threadIdx.x; e < KT * 8; e += blockDim.x) {
      const int r = e >> 3, c = e & 7;
      const bool ok = r < T.count;
      const int rr = ok ? r : 0;
      cp_async16(sK + swz(r, c), k + (int64_t)rr * T.stride + c * 8, ok);
      cp_async16(sV + swz(r, c), v + (int64_t)rr * T.stride + c * 8, ok);
    }
  } else {
    const uint8_t* k = reinterpret_cast<const uint8_t*>(T.k);
    const uint8_t* v = reinterpret_cast<const uint8_t*>(T.v);
    for (int e = threadIdx.x; e < KT * 8; e += blockDim.x) {
      const int r = e >> 3, c = e & 7;
      uint2 kc = make_uint2(0, 0), vc = make_uint2(0, 0);
      if (r < T.count) {
        kc = *reinterpret_cast<const uint2*>(k + (int64_t)r * HD + c * 8);
        vc = *reinterpret_cast<const uint2*>(v + (int64_t)r * HD + c * 8);
      }
      const uint8_t* kb = reinterpret_cast<const uint8_t*>(&kc);
      const uint8_t* vb = reinterpret_cast<const uint8_t*>(&vc);
      uint4 ko, vo;
      uint32_t* kw = reinterpret_cast<uint32_t*>(&ko);
      uint32_t* vw = reinterpret_cast<uint32_t*>(&vo);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        __half_raw h0 = __nv_cvt_fp8_to_halfraw(kb[2 * q], __NV_E4M3);
        __half_raw h1 = __nv_cvt_fp8_to_halfraw(kb[2 * q + 1], __NV_E4M3);
        kw[q] = pack_bf16(__half2float(__half(h0)), __half2float(__half(h1)));
        h0 = __nv_cvt_fp8_to_halfraw(vb[2 * q], __NV_E4M3);
        h1 = __nv_cvt_fp8_to_halfraw(vb[2 * q + 1], __NV_E4M3);
        vw[q] = pack_bf16(__half2float(__half(h0)), __half2float(__half(h1)));
      }
      *reinterpret_cast<uint4*>(gK + swz(r, c)) = ko;
      *reinterpret_cast<uint4*>(gV + swz(r, c)) = vo;
    }
  }
  cp_async_commit();
}

template <int MODE, bool FP8>
__global__ void __launch_bounds__(256) k_attn_mma(AttnParams a, const int32_t* items) {
  __shared__ __align__(128) uint8_t sQ[MAX_ROWS * 128];
  __shared__ __align__(128) uint8_t sK[2][KT * 128];
  __shared__ __align__(128) uint8_t sV[2][KT * 128];
  const int G = a.hq / a.hkv;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Ctx<MODE, FP8> C;
  C.a = &a;
  C.g = blockIdx.y;
  int row_base = 0;
  if (MODE == 1) {
    C.i = blockIdx.x;
    C.P = a.P;
    row_base = blockIdx.z * MAX_ROWS;
    C.rows = min(MAX_ROWS, a.P * G - row_base);
    const int t = a.tup[C.i];
    C.n_doc = a.nk[C.i];
    const int64_t seg = (int64_t)C.g * a.Rp_cap + a.offp[t];
    if (FP8) {
      C.kr8 = reinterpret_cast<const uint8_t*>(a.Kr) + seg * HD;
      C.vr8 = reinterpret_cast<const uint8_t*>(a.Vr) + seg * HD;
      C.sc = a.scales + (seg >> 6) * 2;
    } else {
      C.krb = reinterpret_cast<const bf16*>(a.Kr) + seg * HD;
      C.vrb = reinterpret_cast<const bf16*>(a.Vr) + seg * HD;
    }
    const int64_t pb = (int64_t)C.i * a.P * a.hkv * HD + (int64_t)C.g * HD;
    C.kp = reinterpret_cast<const bf16*>(a.kp) + pb;
    C.vp = reinterpret_cast<const bf16*>(a.vp) + pb;
  } else {
    C.t = items[2 * blockIdx.x];
    C.j0 = items[2 * blockIdx.x + 1];
    C.L = (int)(a.off[C.t + 1] - a.off[C.t]);
    C.rows = MAX_ROWS;
    const int64_t seg = (int64_t)C.g * a.R + a.off[C.t];
    C.kd = reinterpret_cast<const bf16*>(a.K) + seg * HD;
    C.vd = reinterpret_cast<const bf16*>(a.V) + seg * HD;
  }
  // ---- stage Q rows: row r -> (position, head of the group)
  const bf16* qg = reinterpret_cast<const bf16*>(a.q);
  const uint32_t sQa = ptx::smem_u32(sQ);
  for (int e = threadIdx.x; e < MAX_ROWS * 8; e += blockDim.x) {
    const int r = e >> 3, c = e & 7;
    const int rr = row_base + r;
    const int pos = rr / G, hh = rr % G;
    bool ok = r < C.rows;
    int64_t qrow = 0;
    if (MODE == 1) {
      qrow = (int64_t)C.i * a.P + pos;
    } else {
      ok = ok && (C.j0 + pos) < C.L;
      qrow = a.off[C.t] - a.r0 + C.j0 + pos;
    }
    const bf16* src = qg + (ok ? (qrow * a.hq + (int64_t)C.g * G + hh) * HD + c * 8 : 0);
    cp_async16(sQa + swz(r, c), src, ok);
  }
  const int ntiles = C.n_tiles();
  const uint32_t sKa[2] = {ptx::smem_u32(sK[0]), ptx::smem_u32(sK[1])};
  const uint32_t sVa[2] = {ptx::smem_u32(sV[0]), ptx::smem_u32(sV[1])};
  stage_tile<FP8>(C.tile(0), sKa[0], sVa[0], sK[0], sV[0]);   // commits Q + tile 0

  // per-thread rows: g8 = lane / 4 -> rows (warp*16 + g8) and (+8)
  const int g8 = lane >> 2, t4 = lane & 3;
  const int r_lo = warp * 16 + g8, r_hi = r_lo + 8;
  const int pos_lo = (row_base + r_lo) / G, pos_hi = (row_base + r_hi) / G;
  const bool warp_active = warp * 16 < C.rows;
  const float sl2 = a.scale * 1.4426950408889634f;   // softmax in base 2
  float m_lo = -INFINITY, m_hi = -INFINITY, l_lo = 0.f, l_hi = 0.f;
  float o[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j][0] = o[j][1] = o[j][2] = o[j][3] = 0.f;
  uint32_t qf[4][4];

  for (int ti = 0; ti < ntiles; ++ti) {
    const int buf = ti & 1;
    const Tile T = C.tile(ti);
    if (ti + 1 < ntiles) {
      stage_tile<FP8>(C.tile(ti + 1), sKa[buf ^ 1], sVa[buf ^ 1], sK[buf ^ 1], sV[buf ^ 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (ti == 0 && warp_active) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int row = warp * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int chunk = ks * 2 + (lane >> 4);
        ldsm_x4(sQa + swz(row, chunk), qf[ks][0], qf[ks][1], qf[ks][2], qf[ks][3]);
      }
    }
    if (warp_active) {
      // ---- S = Q K^T for 16 rows x 64 keys
      float s[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j][0] = s[j][1] = s[j][2] = s[j][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
        for (int nb = 0; nb < 8; nb += 2) {
          const int m = lane >> 3;
          const int key = (nb + (m >> 1)) * 8 + (lane & 7);
          const int chunk = ks * 2 + (m & 1);
          uint32_t b0, b1, b2, b3;
          ldsm_x4(sKa[buf] + swz(key, chunk), b0, b1, b2, b3);
          mma_bf16(s[nb], qf[ks], b0, b1);
          mma_bf16(s[nb + 1], qf[ks], b2, b3);
        }
      }
      // ---- mask, scale, online softmax
      float mx_lo = -INFINITY, mx_hi = -INFINITY;
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kk = nb * 8 + t4 * 2 + e;        // key index within the tile
          const int key = T.key0 + kk;
          bool v_lo = kk < T.count, v_hi = v_lo;
          if (MODE == 0) {
            v_lo = v_lo && key <= C.j0 + pos_lo;
            v_hi = v_hi && key <= C.j0 + pos_hi;
          } else if (T.prompt) {
            v_lo = v_lo && key <= pos_lo;
            v_hi = v_hi && key <= pos_hi;
          }
          s[nb][e] = v_lo ? s[nb][e] * T.ks * sl2 : -INFINITY;
          s[nb][2 + e] = v_hi ? s[nb][2 + e] * T.ks * sl2 : -INFINITY;
          mx_lo = fmaxf(mx_lo, s[nb][e]);
          mx_hi = fmaxf(mx_hi, s[nb][2 + e]);
        }
      }
      mx_lo = fmaxf(mx_lo, __shfl_xor_sync(0xffffffffu, mx_lo, 1));
      mx_lo = fmaxf(mx_lo, __shfl_xor_sync(0xffffffffu, mx_lo, 2));
      mx_hi = fmaxf(mx_hi, __shfl_xor_sync(0xffffffffu, mx_hi, 1));
      mx_hi = fmaxf(mx_hi, __shfl_xor_sync(0xffffffffu, mx_hi, 2));
      const float mn_lo = fmaxf(m_lo, mx_lo), mn_hi = fmaxf(m_hi, mx_hi);
      // rows with nothing visible yet keep a zero state (exp2 of -inf - -inf guarded)
      const float base_lo = mn_lo == -INFINITY ? 0.f : mn_lo;
      const float base_hi = mn_hi == -INFINITY ? 0.f : mn_hi;
      const float c_lo = exp2f(m_lo - base_lo), c_hi = exp2f(m_hi - base_hi);
      m_lo = mn_lo;
      m_hi = mn_hi;
      float rs_lo = 0.f, rs_hi = 0.f;
      uint32_t pf[4][4];
#pragma unroll
      for (int nb = 0; nb < 8; ++nb) {
        const float p0 = exp2f(s[nb][0] - base_lo), p1 = exp2f(s[nb][1] - base_lo);
        const float p2 = exp2f(s[nb][2] - base_hi), p3 = exp2f(s[nb][3] - base_hi);
        rs_lo += p0 + p1;
        rs_hi += p2 + p3;
        // A fragment of P for key step nb/2: a0/a1 from even blocks, a2/a3 from odd
        const int ks = nb >> 1;
        if ((nb & 1) == 0) {
          pf[ks][0] = pack_bf16(p0 * T.vs, p1 * T.vs);
          pf[ks][1] = pack_bf16(p2 * T.vs, p3 * T.vs);
        } else {
          pf[ks][2] = pack_bf16(p0 * T.vs, p1 * T.vs);
          pf[ks][3] = pack_bf16(p2 * T.vs, p3 * T.vs);
        }
      }
      l_lo = l_lo * c_lo + rs_lo;
      l_hi = l_hi * c_hi + rs_hi;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        o[j][0] *= c_lo;
        o[j][1] *= c_lo;
        o[j][2] *= c_hi;
        o[j][3] *= c_hi;
      }
      // ---- O += P V
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
        for (int nd = 0; nd < 8; nd += 2) {
          const int m = lane >> 3;
          const int key = ks * 16 + (m & 1) * 8 + (lane & 7);
          const int chunk = nd + (m >> 1);
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(sVa[buf] + swz(key, chunk), b0, b1, b2, b3);
          mma_bf16(o[nd], pf[ks], b0, b1);
          mma_bf16(o[nd + 1], pf[ks], b2, b3);
        }
      }
    }
    __syncthreads();
  }
  if (!warp_active) return;
  l_lo += __shfl_xor_sync(0xffffffffu, l_lo, 1);
  l_lo += __shfl_xor_sync(0xffffffffu, l_lo, 2);
  l_hi += __shfl_xor_sync(0xffffffffu, l_hi, 1);
  l_hi += __shfl_xor_sync(0xffffffffu, l_hi, 2);
  const float inv_lo = l_lo > 0.f ? 1.f / l_lo : 0.f, inv_hi = l_hi > 0.f ? 1.f / l_hi : 0.f;
  bf16* og = reinterpret_cast<bf16*>(a.o);
  auto out_row = [&](int r, int pos, int64_t& orow, bool& ok) {
    const int hh = (row_base + r) % G;
    ok = r < C.rows;
    if (MODE == 1) {
      orow = ((int64_t)C.i * a.P + pos) * a.hq + (int64_t)C.g * G + hh;
    } else {
      ok = ok && C.j0 + pos < C.L;
      orow = (a.off[C.t] - a.r0 + C.j0 + pos) * a.hq + (int64_t)C.g * G + hh;
    }
  };
  int64_t orow;
  bool ok;
  out_row(r_lo, pos_lo, orow, ok);
  if (ok) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<uint32_t*>(og + orow * HD + j * 8 + t4 * 2) =
          pack_bf16(o[j][0] * inv_lo, o[j][1] * inv_lo);
  }
  out_row(r_hi, pos_hi, orow, ok);
  if (ok) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<uint32_t*>(og + orow * HD + j * 8 + t4 * 2) =
          pack_bf16(o[j][2] * inv_hi, o[j][3] * inv_hi);
  }
}

}  // namespace

void attn_mma_eval(const AttnParams& a, cudaStream_t s) {
  if (a.n <= 0) return;
  const int G = a.hq / a.hkv;
  dim3 grid(a.n, a.hkv, (a.P * G + MAX_ROWS - 1) / MAX_ROWS);
  if (a.kv_dtype == ST_E4M3)
    k_attn_mma<1, true><<<grid, 256, 0, s>>>(a, nullptr);
  else
    k_attn_mma<1, false><<<grid, 256, 0, s>>>(a, nullptr);
}

void attn_mma_prefill(const AttnParams& a, const int32_t* items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return;
  dim3 grid(n_items, a.hkv, 1);
  k_attn_mma<0, false><<<grid, 256, 0, s>>>(a, items);
}

}  // namespace st
