// Pipelined host execution: a stream of one beam's blocks from host memory
// with up to `depth` blocks in flight (Sec. 2.3 block flow). Block k's kernels
// run on the caller's stream while block k + 1 crosses to the device on one
// copy stream and block k - 1's results cross back on another, so a steady
// stream of blocks runs at the kernels' rate whenever the copies take less
// time than the kernels. Host code only: every step of the path is the
// tx_execute of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>

#include "tx_internal.h"

using namespace tx;

#define TX_CUDA(expr)                                                               \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      set_error("%s failed: %s", #expr, cudaGetErrorString(e_));                    \
      return TX_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)

namespace {

constexpr int kMaxDepth = 4;

struct Slot {
  uint8_t* d_block = nullptr;     // staging for the block's input
  void* d_out = nullptr;          // the block's output
  int64_t* d_ncand = nullptr;     // candidate counter (TX_OUT_CANDS)
  int64_t* h_ncand = nullptr;     // pinned copies of the counter and of the beam's give-up count
  cudaEvent_t in = nullptr;       // input on the device
  cudaEvent_t done = nullptr;     // kernels finished
  cudaEvent_t count = nullptr;    // counter copied to the host
  cudaEvent_t out = nullptr;      // results on the host
};

}  // namespace

struct tx_pipeline {
  const tx_plan* plan = nullptr;
  tx_beam* beam = nullptr;
  int device = -1;
  int depth = 0;
  cudaStream_t compute = nullptr;  // the caller's stream
  cudaStream_t h2d = nullptr, d2h = nullptr;
  void* d_ws = nullptr;            // workspace, shared: the blocks' kernels run one after another
  Slot slot[kMaxDepth];
  int64_t pushed = 0, popped = 0;
};

namespace {

void release(tx_pipeline* pl) {
  for (int i = 0; i < kMaxDepth; ++i) {
    Slot& s = pl->slot[i];
    if (s.d_block) cudaFree(s.d_block);
    if (s.d_out) cudaFree(s.d_out);
    if (s.d_ncand) cudaFree(s.d_ncand);
    if (s.h_ncand) cudaFreeHost(s.h_ncand);
    for (cudaEvent_t e : {s.in, s.done, s.count, s.out})
      if (e) cudaEventDestroy(e);
  }
  if (pl->d_ws) cudaFree(pl->d_ws);
  if (pl->h2d) cudaStreamDestroy(pl->h2d);
  if (pl->d2h) cudaStreamDestroy(pl->d2h);
}

// Polls ev until it completes or the deadline passes (timeout_us < 0: none).
int wait_event(cudaEvent_t ev, std::chrono::steady_clock::time_point t0, int64_t timeout_us, const char* what) {
  while (true) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return TX_OK;
    if (e != cudaErrorNotReady) {
      set_error("waiting for %s failed: %s", what, cudaGetErrorString(e));
      return TX_ERR_CUDA;
    }
    const int64_t el =
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_us >= 0 && el >= timeout_us) {
      set_error("%s did not finish within %lld us", what, (long long)timeout_us);
      return TX_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

int32_t tx_pipeline_create(const tx_plan* p, tx_beam* b, int32_t depth, void* stream, tx_pipeline** out) {
  if (!p || !b || !out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (depth < 1 || depth > kMaxDepth) { set_error("depth must be 1..%d", kMaxDepth); return TX_ERR_INVALID_ARG; }
  if (b->plan != p) { set_error("the beam belongs to another plan"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (b->device != dev) { set_error("the beam lives on device %d, the current device is %d", b->device, dev); return TX_ERR_INVALID_ARG; }
  tx_pipeline* pl = new (std::nothrow) tx_pipeline;
  if (!pl) { set_error("host allocation failed"); return TX_ERR_OOM; }
  pl->plan = p;
  pl->beam = b;
  pl->device = dev;
  pl->depth = depth;
  pl->compute = (cudaStream_t)stream;
  auto fail = [&](int rc) { release(pl); delete pl; return rc; };
  auto cuda = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TX_OK;
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TX_ERR_OOM : TX_ERR_CUDA;
  };
  int rc;
  if ((rc = cuda(cudaStreamCreateWithFlags(&pl->h2d, cudaStreamNonBlocking), "copy stream"))) return fail(rc);
  if ((rc = cuda(cudaStreamCreateWithFlags(&pl->d2h, cudaStreamNonBlocking), "copy stream"))) return fail(rc);
  const int64_t ws = b->compact ? p->ws_bytes_compact : p->ws_bytes;
  if ((rc = cuda(cudaMalloc(&pl->d_ws, (size_t)std::max<int64_t>(ws, 256)), "workspace"))) return fail(rc);
  for (int i = 0; i < depth; ++i) {
    Slot& s = pl->slot[i];
    if ((rc = cuda(cudaMalloc((void**)&s.d_block, (size_t)p->nchan * p->T), "staging buffer"))) return fail(rc);
    if ((rc = cuda(cudaMalloc(&s.d_out, (size_t)std::max<int64_t>(p->out_bytes, 16)), "output buffer"))) return fail(rc);
    if ((rc = cuda(cudaMalloc((void**)&s.d_ncand, sizeof(int64_t)), "counter"))) return fail(rc);
    if ((rc = cuda(cudaHostAlloc((void**)&s.h_ncand, 2 * sizeof(int64_t), cudaHostAllocDefault), "pinned counter")))
      return fail(rc);
    for (cudaEvent_t* e : {&s.in, &s.done, &s.count, &s.out})
      if ((rc = cuda(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event"))) return fail(rc);
  }
  *out = pl;
  return TX_OK;
}

int32_t tx_pipeline_push(tx_pipeline* pl, const uint8_t* h_block) {
  if (!pl || !h_block) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (pl->pushed - pl->popped >= pl->depth) {
    set_error("%d blocks already in flight: pop one first", pl->depth);
    return TX_ERR_BUDGET;
  }
  const tx_plan* p = pl->plan;
  Slot& s = pl->slot[pl->pushed % pl->depth];
  // the slot's previous block was popped: its kernels and copies are done
  TX_CUDA(cudaMemcpyAsync(s.d_block, h_block, (size_t)p->nchan * p->T, cudaMemcpyHostToDevice, pl->h2d));
  TX_CUDA(cudaEventRecord(s.in, pl->h2d));
  TX_CUDA(cudaStreamWaitEvent(pl->compute, s.in, 0));
  const int rc = tx_execute(p, pl->beam, s.d_block, s.d_out, p->output == TX_OUT_CANDS ? s.d_ncand : nullptr,
                            pl->d_ws, pl->compute);
  if (rc) return rc;
  TX_CUDA(cudaEventRecord(s.done, pl->compute));
  ++pl->pushed;
  return TX_OK;
}

int32_t tx_pipeline_pop(tx_pipeline* pl, void* h_out, int64_t* h_ncand, int64_t timeout_us) {
  if (!pl || !h_out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  const tx_plan* p = pl->plan;
  if (p->output == TX_OUT_CANDS && !h_ncand) { set_error("candidate mode needs h_ncand"); return TX_ERR_INVALID_ARG; }
  if (pl->popped == pl->pushed) { set_error("no block in flight"); return TX_ERR_INVALID_ARG; }
  Slot& s = pl->slot[pl->popped % pl->depth];
  const auto t0 = std::chrono::steady_clock::now();
  // The result copies are enqueued only once the kernels have finished: a
  // copy waiting on an event in a copy queue could hold back the next block's
  // input copy behind it (the two directions may share a queue).
  int rc;
  if ((rc = wait_event(s.done, t0, timeout_us, "the block's kernels"))) return rc;
  // the beam's count of waits its kernels gave up comes back with the first result copy
  int32_t* h_fail = reinterpret_cast<int32_t*>(s.h_ncand + 1);
  TX_CUDA(cudaMemcpyAsync(h_fail, pl->beam->fail, sizeof(int32_t), cudaMemcpyDeviceToHost, pl->d2h));
  auto gave_up = [&]() -> int {
    if (*h_fail == 0) return TX_OK;
    set_error("the beam's kernels gave up %d waits: results not valid (reset the beam)", *h_fail);
    return TX_ERR_ABORTED;
  };
  if (p->output == TX_OUT_CANDS) {
    TX_CUDA(cudaMemcpyAsync(s.h_ncand, s.d_ncand, sizeof(int64_t), cudaMemcpyDeviceToHost, pl->d2h));
    TX_CUDA(cudaEventRecord(s.count, pl->d2h));
    if ((rc = wait_event(s.count, t0, timeout_us, "the candidate count"))) return rc;
    const int64_t total = *s.h_ncand;
    const int64_t n = std::min<int64_t>(total, p->max_cands);
    if (n > 0) TX_CUDA(cudaMemcpyAsync(h_out, s.d_out, (size_t)n * sizeof(tx_cand), cudaMemcpyDeviceToHost, pl->d2h));
    TX_CUDA(cudaEventRecord(s.out, pl->d2h));
    if ((rc = wait_event(s.out, t0, timeout_us, "the candidate copy"))) return rc;
    *h_ncand = total;
    ++pl->popped;
    if ((rc = gave_up())) return rc;
    if (total > p->max_cands) {
      set_error("%lld candidates, capacity %lld", (long long)total, (long long)p->max_cands);
      return TX_ERR_CAND_OVERFLOW;
    }
    return TX_OK;
  }
  TX_CUDA(cudaMemcpyAsync(h_out, s.d_out, (size_t)p->out_bytes, cudaMemcpyDeviceToHost, pl->d2h));
  TX_CUDA(cudaEventRecord(s.out, pl->d2h));
  if ((rc = wait_event(s.out, t0, timeout_us, "the block's results"))) return rc;
  ++pl->popped;
  return gave_up();
}

void tx_pipeline_destroy(tx_pipeline* pl) {
  if (!pl) return;
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != pl->device) cudaSetDevice(pl->device);
  cudaStreamSynchronize(pl->compute);
  cudaStreamSynchronize(pl->h2d);
  cudaStreamSynchronize(pl->d2h);
  release(pl);
  if (cur >= 0 && cur != pl->device) cudaSetDevice(cur);
  delete pl;
}

}  // extern "C"
