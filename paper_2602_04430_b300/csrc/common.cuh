// Shared device helpers and internal structures of libstretto (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stretto.h"

namespace st {

// NVTX range around one public call (visible in Nsight timelines; a no-op
// when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define ST_TRACE(name) ::st::TraceRange st_trace_range_(name)

typedef __nv_bfloat16 bf16;

// Checked build (-DST_CHECK, libstretto_check.so): the ragged offsets and
// indices the kernels follow are checked before use; a failed check records
// ST_ECHECK in the given status word (first error wins) and the caller skips
// or clamps the access.  In the regular build the condition is not evaluated.
#ifdef ST_CHECK
#define ST_CHECKED(cond, status) ((cond) ? true : (atomicCAS((status), ST_OK, ST_ECHECK), false))
#else
#define ST_CHECKED(cond, status) true
#endif

// ---------------------------------------------------------------- conversions
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<bf16>(bf16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 from_f<bf16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Load / store n consecutive elements as float (n a multiple of 4 for float, 8 for bf16).
template <typename T> struct Vec;
// 16 bytes through the read-only path, not kept in L1 (streamed once).
__device__ __forceinline__ uint4 ldg_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

template <> struct Vec<float> {
  static constexpr int N = 4;
  __device__ __forceinline__ static void unpack(const uint4& v, float* out) {
    out[0] = __uint_as_float(v.x); out[1] = __uint_as_float(v.y);
    out[2] = __uint_as_float(v.z); out[3] = __uint_as_float(v.w);
  }
  __device__ __forceinline__ static void load(const float* p, float* out) {
    float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  }
  __device__ __forceinline__ static void store(float* p, const float* in) {
    *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
  }
};
template <> struct Vec<bf16> {
  static constexpr int N = 8;
  __device__ __forceinline__ static void unpack(const uint4& v, float* out) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      out[2 * i] = f.x; out[2 * i + 1] = f.y;
    }
  }
  __device__ __forceinline__ static void load(const bf16* p, float* out) {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      out[2 * i] = f.x; out[2 * i + 1] = f.y;
    }
  }
  __device__ __forceinline__ static void store(bf16* p, const float* in) {
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(in[2 * i], in[2 * i + 1]);
    *reinterpret_cast<uint4*>(p) = v;
  }
};

// x * sigmoid(x) with the fast reciprocal-based divide (about 2 ulp)
__device__ __forceinline__ float silu_f(float x) { return __fdividef(x, 1.0f + __expf(-x)); }

// ---------------------------------------------------------------- host side
struct LayerW {
  void* wqkv = nullptr;  // [(hq+2hkv)*hd][d]
  void* wo = nullptr;    // [d][hq*hd]
  void* wgu = nullptr;   // [2*ffn][d], gate/up interleaved in blocks of 128 rows
  void* wd = nullptr;    // [d][ffn]
};

// A grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool external = false;   // caller-owned (st_set_workspace): never grown or freed here
};

struct ProfRec {
  int family;
  double flops, bytes;
  cudaEvent_t a, b;
};

struct Prof {
  bool on = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  double acc[ST_PROF_N][4] = {};
};

}  // namespace st

struct st_ctx {
  st_model_cfg cfg;
  int device = 0;
  size_t esz = 4;                 // bytes per weight / activation element
  void* embed = nullptr;
  void* w_lm = nullptr;
  std::vector<st::LayerW> layers;
  float2* rope = nullptr;         // [max_pos][hd/2] (cos, sin)
  float2* rope_t = nullptr;       // the same, [hd/2][max_pos]
  // workspaces
  st::DevBuf ws_build, ws_eval, ws_casc, ws_map;
  int64_t build_rows_cap = 0, eval_rows_cap = 0;
  // operator-evaluation schedule (st_autotune_eval): BF16-KV attention layout
  // (0 / 1 = two CTAs per SM, 2 = one CTA per SM) and longest-first work order
  int attn_nb = 0;
  int longest_first = 1;
  int split_keys = 0;             // split-KV piece length in retained slots (0 = off)
  // retention scores of st_kv_build (st_set_scoring): ST_SCORE_EA_LITE or
  // ST_SCORE_EA_FULL with its horizon F and the averaged rotation table
  // rope_avg[L][hd/2] = (mean cos, mean sin) over positions L .. L+F-1
  int score_mode = ST_SCORE_EA_LITE;
  int score_horizon = 0;
  float2* rope_avg = nullptr;
  st::DevBuf ws_score;            // st_kv_score_query: tuple ids, logits, labels
  st::DevBuf ws_pcasc;            // st_proxy_cascade: confidences and routing
  int32_t* dstatus = nullptr;     // device status word of bounded waits (ST_ETIMEOUT)
  std::string err;
  st::Prof prof;
  int64_t launches = 0;
};

struct st_kv {
  st_ctx* ctx = nullptr;
  int32_t T = 0;
  int64_t R = 0;                  // total document tokens
  int64_t Rp_cap = 0;             // capacity of the retained cache in slots (sum of pad64(L))
  int32_t max_len = 0;
  std::vector<int64_t> off_h;     // host copy of offsets
  int64_t* off = nullptr;         // device [T+1]
  void* K = nullptr;              // [layers][hkv][R][hd]
  void* V = nullptr;
  float* scores = nullptr;        // [layers][hkv][R]
  float* pooled = nullptr;        // [T][d]
  int32_t* rank = nullptr;        // [layers][hkv][R]
  void* Kr = nullptr;             // [layers][hkv][Rp_cap][hd]
  void* Vr = nullptr;
  float* scales = nullptr;        // [layers][hkv][Rp_cap/64][2]
  int64_t* offp = nullptr;        // device [T+1]
  int32_t* nkeep = nullptr;       // device [T]
  int32_t* status = nullptr;      // device status word
  int64_t Rp = 0;                 // used retained slots (sum pad64(n))
  double r = 0.0;                 // retained fraction of the current profile (0 = none)
  int32_t kv_dtype = -1;
  bool built = false;
  int32_t* items = nullptr;       // device [n_items][2] prefill work items (tuple, first position)
  int64_t n_items = 0;
  std::vector<int64_t> item_start;  // first item of each tuple (host)
  int32_t* tok = nullptr;         // device token buffer of st_run_host
  int32_t* iota = nullptr;        // device 0..T-1 of st_run_host
  float* out_logits = nullptr;    // device outputs of st_run_host
  int32_t* out_labels = nullptr;
  // a second retained profile of another cache (st_kv_profile_alloc): shares
  // src's offsets, full cache, scores, pooled states and prefill items, owns
  // its rank, retained cache, scales, offsets, counts and status word
  st_kv* src = nullptr;
  double r_max = 1.0;             // largest r the retained capacity holds
};

struct st_operator {
  st_op desc;
  int32_t* prompt = nullptr;      // device [P]
  int32_t* labels = nullptr;      // device [n_labels]
  float* bias = nullptr;          // device [n_labels]
  float theta_pos = 0, theta_neg = 0;
};
