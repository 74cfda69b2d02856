// Multi-stage operator cascade (Sec. 4.1, generalised to any number of
// stages): stage k evaluates its operator (own model, cache, r and thresholds
// theta+ / theta-) on the tuples every earlier stage left unsure; a tuple
// leaves the cascade at the first stage that accepts or rejects it, and the
// last stage's unsure tuples stay unsure.  Each stage is one st_op_eval on the
// stage's context; a routing kernel records the decided tuples at their
// original positions and compacts the unsure ones, in order, for the next
// stage.  The host reads each stage's unsure count (one synchronisation per
// stage) to size the next evaluation.
#include <string>
#include <vector>

#include "kernels.h"

using namespace st;

namespace {

int cfail(st_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

// One block of 1024 threads.  For i < n: the stage's decision lab[i] of tuple
// ids[i] (original position pos[i], or i when pos is NULL); decided (or last
// stage) -> out_label / out_stage at that position; unsure -> appended, in
// order, to (next_ids, next_pos), their number to *next_n.
__global__ void __launch_bounds__(1024) k_stage_route(const int32_t* __restrict__ lab,
                                                      const int32_t* __restrict__ ids,
                                                      const int32_t* __restrict__ pos, int n, int stage,
                                                      int last, int32_t* __restrict__ out_label,
                                                      int32_t* __restrict__ out_stage,
                                                      int32_t* __restrict__ next_ids,
                                                      int32_t* __restrict__ next_pos,
                                                      int32_t* __restrict__ next_n) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    const bool in = i < n;
    const int l = in ? lab[i] : 0;
    const int p = in ? (pos ? pos[i] : i) : 0;
    const bool go = in && !last && l == ST_UNSURE;
    if (in && !go) {
      out_label[p] = l;
      out_stage[p] = stage;
    }
    // exclusive prefix of `go` over the block
    const unsigned bal = __ballot_sync(0xffffffffu, go);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
      const int v = wsum[lane];
      int inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      wsum[lane] = inc - v;
    }
    __syncthreads();
    const int at = carry + wsum[wid] + before;
    if (go) {
      next_ids[at] = ids[i];
      next_pos[at] = p;
    }
    __syncthreads();
    if (tid == 1023) carry = at + (go ? 1 : 0);
    __syncthreads();
  }
  if (tid == 0) *next_n = carry;
}

// stage of the merged proxy cascade: 0 everywhere (the proxy decided), then,
// in a second launch, k + 1 at the positions operator stage k decided
__global__ void k_stage_zero(int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 0;
}
__global__ void k_scatter_stage(const int32_t* __restrict__ pos, const int32_t* __restrict__ count,
                                const int32_t* __restrict__ op_stage, int32_t* __restrict__ out, int n,
                                int* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < *count && ST_CHECKED((unsigned)pos[j] < (unsigned)n, status)) out[pos[j]] = op_stage[j] + 1;
}

}  // namespace

extern "C" int st_cascade_run(int32_t n_stages, const st_stage* stages, const int32_t* tuple_ids_dev,
                              int32_t n, int32_t* labels_dev, int32_t* stage_dev, int32_t* counts_host,
                              float* ms_host, void* stream) {
  ST_TRACE("st_cascade_run");
  st_ctx* ctx = (n_stages >= 1 && stages) ? stages[0].ctx : nullptr;
  if (!ctx || n < 0 || (n > 0 && (!tuple_ids_dev || !labels_dev || !stage_dev)))
    return cfail(ctx, ST_EINVAL, "st_cascade_run: bad argument");
  for (int k = 0; k < n_stages; ++k) {
    const st_stage& sg = stages[k];
    if (!sg.ctx || !sg.kv || !sg.op || sg.kv->ctx != sg.ctx || sg.ctx->device != ctx->device)
      return cfail(ctx, ST_EINVAL, "st_cascade_run: stage " + std::to_string(k) + ": bad context / cache / operator");
    if (sg.op->desc.kind != ST_OP_FILTER)
      return cfail(ctx, ST_EINVAL, "st_cascade_run: stage " + std::to_string(k) + ": not a filter operator");
  }
  for (int k = 0; k < n_stages; ++k) {
    if (counts_host) counts_host[k] = 0;
    if (ms_host) ms_host[k] = 0.f;
  }
  if (n == 0) return ST_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // routing buffers in the first stage's context: two (ids, pos) sets, the
  // stage's logits and labels, and the unsure count
  const size_t need = (size_t)n * 4 * 4 + (size_t)n * 2 * 4 + (size_t)n * 4 + 256 * 8;
  if (ctx->ws_casc.bytes < need) {
    if (ctx->ws_casc.p) cudaFree(ctx->ws_casc.p);
    ctx->ws_casc.p = nullptr;
    ctx->ws_casc.bytes = 0;
    if (cudaMalloc(&ctx->ws_casc.p, need) != cudaSuccess) {
      cudaGetLastError();
      return cfail(ctx, ST_ENOMEM, "st_cascade_run: routing buffers");
    }
    ctx->ws_casc.bytes = need;
  }
  auto carve = [](char*& p, size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  char* p = (char*)ctx->ws_casc.p;
  int32_t* ids[2] = {(int32_t*)carve(p, (size_t)n * 4), (int32_t*)carve(p, (size_t)n * 4)};
  int32_t* pos[2] = {(int32_t*)carve(p, (size_t)n * 4), (int32_t*)carve(p, (size_t)n * 4)};
  float* logits = (float*)carve(p, (size_t)n * 2 * 4);
  int32_t* lab = (int32_t*)carve(p, (size_t)n * 4);
  int32_t* cnt = (int32_t*)carve(p, 4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms_host && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    return cfail(ctx, ST_ECUDA, "st_cascade_run: events");
  const int32_t* cur_ids = tuple_ids_dev;
  const int32_t* cur_pos = nullptr;   // identity
  int cur_n = n, rc = ST_OK;
  for (int k = 0; k < n_stages && cur_n > 0; ++k) {
    const st_stage& sg = stages[k];
    if (counts_host) counts_host[k] = cur_n;
    if (ms_host) cudaEventRecord(e0, s);
    if ((rc = st_op_eval(sg.ctx, sg.kv, sg.op, cur_ids, cur_n, logits, lab, stream)) != ST_OK) {
      ctx->err = "st_cascade_run: stage " + std::to_string(k) + ": " + sg.ctx->err;
      break;
    }
    const int nb = k & 1;
    k_stage_route<<<1, 1024, 0, s>>>(lab, cur_ids, cur_pos, cur_n, k, k + 1 == n_stages ? 1 : 0,
                                     labels_dev, stage_dev, ids[nb], pos[nb], cnt);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ms_host) e = cudaEventRecord(e1, s);
    int32_t next_n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&next_n, cnt, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cfail(ctx, ST_ECUDA, std::string("st_cascade_run: ") + cudaGetErrorString(e));
      break;
    }
    if (ms_host) cudaEventElapsedTime(&ms_host[k], e0, e1);
    cur_ids = ids[nb];
    cur_pos = pos[nb];
    cur_n = next_n;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

extern "C" int st_proxy_cascade(st_ctx* ctx, st_proxy* p, const float* x_dev, float tau, int32_t n_stages,
                                const st_stage* stages, const int32_t* tuple_ids_dev, int32_t n,
                                int32_t* labels_dev, int32_t* stage_dev, int32_t* counts_host, void* stream) {
  ST_TRACE("st_proxy_cascade");
  if (!ctx || !p || !x_dev || n < 0 || n_stages < 1 || !stages ||
      (n > 0 && (!tuple_ids_dev || !labels_dev || !stage_dev)))
    return cfail(ctx, ST_EINVAL, "st_proxy_cascade: bad argument");
  if (counts_host)
    for (int k = 0; k <= n_stages; ++k) counts_host[k] = 0;
  if (n == 0) return ST_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  {
    // an error left pending by an earlier call is reported as such, not as this call's
    const cudaError_t pend = cudaGetLastError();
    if (pend != cudaSuccess)
      return cfail(ctx, ST_ECUDA, std::string("st_proxy_cascade: pending error from an earlier call: ") +
                                      cudaGetErrorString(pend));
  }
  // routing buffers: confidence, proxy label, unsure ids / positions, the
  // operator stages' labels and stages, the unsure count
  auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t need = 6 * r256((size_t)n * 4) + r256(8);   // exactly what the carving below takes
  if (ctx->ws_pcasc.bytes < need) {
    if (ctx->ws_pcasc.p) cudaFree(ctx->ws_pcasc.p);
    ctx->ws_pcasc.p = nullptr;
    ctx->ws_pcasc.bytes = 0;
    if (cudaMalloc(&ctx->ws_pcasc.p, need) != cudaSuccess) {
      cudaGetLastError();
      return cfail(ctx, ST_ENOMEM, "st_proxy_cascade: routing buffers");
    }
    ctx->ws_pcasc.bytes = need;
  }
  auto carve = [](char*& q, size_t bytes) {
    char* r = q;
    q += (bytes + 255) & ~(size_t)255;
    return r;
  };
  char* q = (char*)ctx->ws_pcasc.p;
  float* conf = (float*)carve(q, (size_t)n * 4);
  int32_t* plab = (int32_t*)carve(q, (size_t)n * 4);
  int32_t* u_ids = (int32_t*)carve(q, (size_t)n * 4);
  int32_t* u_pos = (int32_t*)carve(q, (size_t)n * 4);
  int32_t* u_lab = (int32_t*)carve(q, (size_t)n * 4);
  int32_t* u_stg = (int32_t*)carve(q, (size_t)n * 4);
  int32_t* cnt = (int32_t*)carve(q, 8);
  int rc = st_proxy_eval(ctx, p, x_dev, tuple_ids_dev, n, conf, plab, stream);
  if (rc != ST_OK) return rc;
  if ((rc = st_cascade_compact(ctx, conf, tuple_ids_dev, n, tau, u_ids, cnt, stream)) != ST_OK) return rc;
  if ((rc = st_cascade_compact(ctx, conf, nullptr, n, tau, u_pos, cnt + 1, stream)) != ST_OK) return rc;
  int32_t k = 0;
  cudaError_t e = cudaMemcpyAsync(&k, cnt, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();   // leave no error pending for the next call
    return cfail(ctx, ST_ECUDA, std::string("st_proxy_cascade: proxy stage: ") + cudaGetErrorString(e));
  }
  if (counts_host) counts_host[0] = n;
  if (k > 0 && (rc = st_cascade_run(n_stages, stages, u_ids, k, u_lab, u_stg, counts_host ? counts_host + 1 : nullptr,
                                    nullptr, stream)) != ST_OK) {
    if (stages[0].ctx != ctx) ctx->err = stages[0].ctx->err;
    return rc;
  }
  // the proxy's labels everywhere, then the operator stages' at the unsure positions
  if ((rc = st_cascade_merge(ctx, plab, n, u_pos, cnt, u_lab, labels_dev, stream)) != ST_OK) return rc;
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_stage_zero<<<(n + 255) / 256, 256, 0, s>>>(n, stage_dev);
  }
  {
    Launch L(ctx, s, ST_PROF_OTHER, 0, 0);
    k_scatter_stage<<<(n + 255) / 256, 256, 0, s>>>(u_pos, cnt, u_stg, stage_dev, n, ctx->dstatus);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cfail(ctx, ST_ECUDA, std::string("st_proxy_cascade: merge: ") + cudaGetErrorString(e));
  return ST_OK;
}
