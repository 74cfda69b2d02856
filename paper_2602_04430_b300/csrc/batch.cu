// Batched operator evaluation as a replayable CUDA graph, and the autotuner of
// its schedule.  Both drive the same layer sequence as st_op_eval_multi
// (run_opset in api.cu): the graph captures it once on a private stream with
// its own workspace; the autotuner times it under each candidate schedule.
#include <algorithm>
#include <string>
#include <vector>

#include "kernels.h"
#include "ptx.cuh"

using namespace st;

struct st_graph {
  st_ctx* ctx = nullptr;
  cudaGraphExec_t exec = nullptr;
  DevBuf ws;                 // the captured kernels' activations (owned by the graph)
  int64_t launches = 0;      // kernels per replay
};

namespace {

int bfail(st_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(ctx, ST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

// Schedule of the context while a candidate is timed.
struct Sched {
  int64_t eval_rows;
  int attn_nb, longest_first, split_keys;
};
Sched get(const st_ctx* c) { return {c->eval_rows_cap, c->attn_nb, c->longest_first, c->split_keys}; }
void set(st_ctx* c, const Sched& s) {
  c->eval_rows_cap = s.eval_rows;
  c->attn_nb = s.attn_nb;
  c->longest_first = s.longest_first;
  c->split_keys = s.split_keys;
}

}  // namespace

extern "C" int st_graph_create(st_ctx* ctx, const st_kv* kv, int32_t n_ops,
                               const st_operator* const* ops, const int32_t* const* tuple_ids_dev,
                               const int32_t* n, float* const* logits_dev, int32_t* const* labels_dev,
                               st_graph** out) {
  ST_TRACE("st_graph_create");
  if (!ctx || !out) return bfail(ctx, ST_EINVAL, "st_graph_create: bad argument");
  *out = nullptr;
  OpSet os;
  int64_t rows = 0;
  int pairs = 0;
  int rc = make_opset(ctx, kv, n_ops, ops, tuple_ids_dev, n, logits_dev, labels_dev, &os, &rows, &pairs);
  if (rc != ST_OK) return rc;
  if (pairs == 0) return bfail(ctx, ST_EINVAL, "st_graph_create: no (operator, tuple) pairs");
  st_graph* g = new st_graph();
  g->ctx = ctx;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  const bool prof = ctx->prof.on;
  auto cleanup = [&](int code) {
    ctx->prof.on = prof;
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (code != ST_OK) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      if (g->ws.p) cudaFree(g->ws.p);
      delete g;
    }
    return code;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cleanup(bfail(ctx, ST_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
  // one uncaptured run sizes the graph's workspace and sets every kernel's
  // attributes, so the captured run allocates nothing
  ctx->prof.on = false;
  if ((rc = run_opset(ctx, kv, os, pairs, cs, &g->ws)) != ST_OK) return cleanup(rc);
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess)
    return cleanup(bfail(ctx, ST_ECUDA, std::string("warm-up: ") + cudaGetErrorString(e)));
  const int64_t l0 = ctx->launches;
  if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cleanup(bfail(ctx, ST_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e)));
  rc = run_opset(ctx, kv, os, pairs, cs, &g->ws);
  e = cudaStreamEndCapture(cs, &graph);   // always end the capture
  g->launches = ctx->launches - l0;
  ctx->launches = l0;                    // counted again at every replay
  if (rc != ST_OK) return cleanup(rc);
  if (e != cudaSuccess) return cleanup(bfail(ctx, ST_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e)));
  if ((e = cudaGraphInstantiate(&g->exec, graph, 0)) != cudaSuccess)
    return cleanup(bfail(ctx, ST_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)));
  *out = g;
  return cleanup(ST_OK);
}

extern "C" int st_graph_launch(st_graph* g, void* stream) {
  ST_TRACE("st_graph_launch");
  if (!g || !g->exec) return ST_EINVAL;
  st_ctx* ctx = g->ctx;
  BCK(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
  ctx->launches += g->launches;
  return ST_OK;
}

extern "C" int64_t st_graph_launches(const st_graph* g) { return g ? g->launches : 0; }

extern "C" void st_graph_free(st_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->ws.p) cudaFree(g->ws.p);
  delete g;
}

extern "C" int st_autotune_eval(st_ctx* ctx, const st_kv* kv, int32_t n_ops,
                                const st_operator* const* ops, const int32_t* const* tuple_ids_dev,
                                const int32_t* n, float* const* logits_dev, int32_t* const* labels_dev,
                                void* stream, st_tune_choice* best, st_tune_choice* tried,
                                int32_t max_tried, int32_t* n_tried) {
  ST_TRACE("st_autotune_eval");
  if (!ctx || !best) return bfail(ctx, ST_EINVAL, "st_autotune_eval: bad argument");
  OpSet os;
  int64_t rows = 0;
  int pairs = 0;
  int rc = make_opset(ctx, kv, n_ops, ops, tuple_ids_dev, n, logits_dev, labels_dev, &os, &rows, &pairs);
  if (rc != ST_OK) return rc;
  if (pairs == 0) return bfail(ctx, ST_EINVAL, "st_autotune_eval: no (operator, tuple) pairs");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Sched start = get(ctx);
  const bool prof = ctx->prof.on;
  ctx->prof.on = false;
  cudaEvent_t a = nullptr, b = nullptr;
  BCK(cudaEventCreate(&a));
  BCK(cudaEventCreate(&b));
  std::vector<st_tune_choice> log;
  // one warm-up run and three timed runs of the whole batched evaluation
  auto time_sched = [&](const Sched& sc, float* ms) -> int {
    set(ctx, sc);
    int r = run_opset(ctx, kv, os, pairs, s, nullptr);
    if (r != ST_OK) return r;
    if (cudaEventRecord(a, s) != cudaSuccess) return ST_ECUDA;
    for (int k = 0; k < 3; ++k)
      if ((r = run_opset(ctx, kv, os, pairs, s, nullptr)) != ST_OK) return r;
    if (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
      return bfail(ctx, ST_ECUDA, "st_autotune_eval: timing events");
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    *ms = t / 3.f;
    log.push_back({sc.eval_rows, sc.attn_nb, sc.longest_first, sc.split_keys, *ms});
    return ST_OK;
  };
  // Coordinate search: the attention layout and work order at the default
  // chunk size, then the chunk size (prompt rows per pass of the layers).
  const bool tc_kv = ctx->cfg.dtype == ST_BF16;   // tensor-core attention (BF16 or E4M3 KV)
  Sched bestc{start.eval_rows > 0 ? start.eval_rows : (1LL << 18), 1, 1, 0};
  float best_ms = 1e30f, ms = 0.f;
  // layouts: 1 = two CTAs per SM (E4M3: 64-key tiles), 2 = one CTA per SM with
  // double buffers, 3 = (E4M3 only) two CTAs per SM with 128-key tiles
  for (int nb : {1, 2, 3}) {
    if (nb >= 2 && !tc_kv) continue;
    if (nb == 3 && kv->kv_dtype != ST_E4M3) continue;
    for (int lf : {1, 0}) {
      const Sched sc{bestc.eval_rows, nb, lf, 0};
      if ((rc = time_sched(sc, &ms)) != ST_OK) break;
      if (ms < best_ms) { best_ms = ms; bestc = sc; }
    }
    if (rc != ST_OK) break;
  }
  int maxP = 1;
  for (int k = 0; k < os.n_ops; ++k) maxP = std::max(maxP, os.op[k].P);
  for (int64_t er : {1LL << 15, 1LL << 16, 1LL << 17, 1LL << 18, 1LL << 19}) {
    if (rc != ST_OK) break;
    if (er == bestc.eval_rows || er < maxP || er > 2 * std::max<int64_t>(rows, 1 << 15)) continue;
    const Sched sc{er, bestc.attn_nb, bestc.longest_first, 0};
    if ((rc = time_sched(sc, &ms)) != ST_OK) break;
    if (ms < best_ms) { best_ms = ms; bestc = sc; }
  }
  // split-KV, when some retained document can be longer than a piece
  constexpr int kSplitCandidate = 2048;
  if (rc == ST_OK && tc_kv && kv->max_len > kSplitCandidate) {
    const Sched sc{bestc.eval_rows, bestc.attn_nb, bestc.longest_first, kSplitCandidate};
    if ((rc = time_sched(sc, &ms)) == ST_OK && ms < best_ms) {
      best_ms = ms;
      bestc = sc;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->prof.on = prof;
  if (rc != ST_OK) {
    set(ctx, start);
    return rc;
  }
  set(ctx, bestc);
  *best = {bestc.eval_rows, bestc.attn_nb, bestc.longest_first, bestc.split_keys, best_ms};
  if (n_tried) *n_tried = (int32_t)log.size();
  if (tried)
    for (int k = 0; k < (int)log.size() && k < max_tried; ++k) tried[k] = log[k];
  return ST_OK;
}

extern "C" int st_set_schedule(st_ctx* ctx, const st_tune_choice* sc) {
  if (!ctx || !sc || sc->eval_rows < 0 || sc->attn_nb < 0 || sc->attn_nb > 3 || sc->split_keys < 0 ||
      sc->split_keys % 128 != 0 || sc->split_keys > 65536)
    return bfail(ctx, ST_EINVAL, "st_set_schedule: bad argument");
  ctx->eval_rows_cap = sc->eval_rows;
  ctx->attn_nb = sc->attn_nb;
  ctx->longest_first = sc->longest_first != 0;
  ctx->split_keys = sc->split_keys;
  return ST_OK;
}

// ------------------------------------------------------------------ failure self-test
namespace {
// One thread waits on an mbarrier that nothing arrives on, through the same
// bounded wait as the pipeline kernels, and records the time-out.
__global__ void k_wait_selftest(int* status, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !ptx::mbar_wait(&bar, 0, limit)) atomicExch(status, ST_ETIMEOUT);
}
}  // namespace

extern "C" int st_selftest_wait(st_ctx* ctx, int64_t limit_cycles, void* stream) {
  if (!ctx || limit_cycles < 1000 || limit_cycles > 1000000000LL)
    return bfail(ctx, ST_EINVAL, "st_selftest_wait: limit must lie in 1e3 .. 1e9 cycles");
  k_wait_selftest<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(ctx->dstatus, (long long)limit_cycles);
  BCK(cudaGetLastError());
  ctx->launches += 1;
  return ST_OK;
}
