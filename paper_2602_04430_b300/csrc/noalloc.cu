// Operator evaluation that allocates no device memory.
//
// Some callers of this library cannot let it call cudaMalloc / cudaFree:
// a query executor that keeps several streams busy cannot afford the implicit
// device synchronisation cudaFree (and at times cudaMalloc) performs, and a
// process whose GPU memory is already claimed by another framework's caching
// allocator can see a fresh cudaMalloc fail although that allocator holds free
// blocks.  For them, st_op_eval_noalloc runs the same kernels as st_op_eval but
// takes its activations from one file-scope device array of fixed size instead
// of the context's workspace (the layer sequence itself is st_op_eval's).
//
// The array lives in every GPU that loads the library, for the life of the
// process.  Host code cannot use its name as a device address; the address is
// resolved once per device with cudaGetSymbolAddress on the first call made
// with that device current.  All calls share the array and it keeps the last
// call's contents: nothing in it needs to start at zero (every buffer is fully
// written before it is read), and calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "kernels.h"

using namespace st;

namespace {

constexpr size_t kScratchBytes = ST_NOALLOC_SCRATCH_BYTES;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int na_fail(st_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

// Device address of g_scratch on the current device (resolved once per device).
int scratch_address(st_ctx* ctx, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(ctx, ST_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(ctx, ST_EUNSUPPORTED, "st_op_eval_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return na_fail(ctx, ST_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ST_OK;
}

#define NA_RC(x)                   \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != ST_OK) return rc_;  \
  } while (0)

}  // namespace

extern "C" int st_op_eval_noalloc(st_ctx* ctx, const st_kv* kv, const st_operator* op,
                                  const int32_t* tuple_ids_dev, int32_t n, float* logits_dev,
                                  int32_t* labels_dev, void* stream) {
  ST_TRACE("st_op_eval_noalloc");
  if (!ctx) return ST_EINVAL;
  if (!kv || !op || kv->ctx != ctx || n < 0) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: bad argument");
  if (n == 0) return ST_OK;
  if (!tuple_ids_dev || !logits_dev || !labels_dev) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: NULL buffer");
  if (kv->r <= 0.0) return na_fail(ctx, ST_EINVAL, "st_op_eval_noalloc: no retained profile (call st_kv_retain)");
  OpSet os;
  int64_t M = 0;
  int pairs = 0;
  NA_RC(make_opset(ctx, kv, 1, &op, &tuple_ids_dev, &n, &logits_dev, &labels_dev, &os, &M, &pairs));
  const int P = op->desc.P;
  const size_t need = eval_bufs(ctx, M, n, nullptr, nullptr);
  if (need > kScratchBytes)
    return na_fail(ctx, ST_EINVAL,
                   "st_op_eval_noalloc: " + std::to_string(n) + " tuples x " + std::to_string(P) +
                       " prompt rows need " + std::to_string(need) + " bytes of scratch, more than the " +
                       std::to_string(kScratchBytes) + "-byte static scratch; pass fewer tuples per call");
  void* base = nullptr;
  NA_RC(scratch_address(ctx, &base));
  EvalBufs w;
  eval_bufs(ctx, M, n, (char*)base, &w);
  // the same layer sequence as st_op_eval (one chunk), with profiling events
  // suppressed on this host thread so that this entry creates no CUDA
  // resources (its launches are still counted); the context's own profiling
  // switch is left untouched
  struct NoProf {
    bool old = tls_no_prof;
    NoProf() { tls_no_prof = true; }
    ~NoProf() { tls_no_prof = old; }
  } guard;
  return eval_chunk(ctx, kv, os, 0, n, 0, M, w, reinterpret_cast<cudaStream_t>(stream));
}
