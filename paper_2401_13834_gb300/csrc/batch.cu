// Batched execute: one block of each of many beams of uneven shape (channel
// counts, block lengths, DM grids, widths, output modes) per step, with each
// phase of the hot path run as persistent launches over the concatenated work
// of many beams instead of one launch sequence per beam (Sec. 2.3 blocked
// processing, applied to many beams at once). A step's launches can be
// captured once as a CUDA graph and replayed; what changes from step to step
// (input and output pointers, ring positions) lives in per-beam arguments that
// each wave of the step first copies into a constant-memory slot, where the
// kernels read them as cheaply as the single-beam kernels read parameters.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "kernels.cuh"
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

// Constant-memory argument slots: a batch holds one slot for its lifetime; a
// wave has at most kArgSlotBeams beams.
constexpr int kArgSlots = 2;
constexpr int kArgSlotBeams = 92;
constexpr int kMaxDevices = 64;

}  // namespace

static __constant__ BeamArgs c_args[kArgSlots * kArgSlotBeams];

namespace {

// Batched argument source: member i of a launch is c_args[base + i].
struct SlotArgs {
  static constexpr bool kBatch = true;
  int base;
  __device__ __forceinline__ BeamArgs get(int i) const { return c_args[base + i]; }
};

std::mutex g_slot_mu;
bool g_slot_used[kMaxDevices][kArgSlots] = {};

// Launch kinds: the first five are the phases (TX_PHASE_* order); the compact
// beams' tail copies count as ingest.
enum LaunchKind { kIngest = TX_PHASE_INGEST, kStage1 = TX_PHASE_STAGE1, kStage2 = TX_PHASE_STAGE2,
                  kStats = TX_PHASE_STATS, kBoxcar = TX_PHASE_BOXCAR, kTailIn = 5, kTailOut = 6, kOffsets = 7 };

// compact beams' tail copies count as ingest, half intermediates' offsets as stage 1
int phase_of(int kind) {
  return kind == kTailIn || kind == kTailOut ? TX_PHASE_INGEST : kind == kOffsets ? TX_PHASE_STAGE1 : kind;
}

// Workspace of one execute on beam b of plan p.
int64_t beam_ws(const tx_plan* p, const tx_beam* b) { return b->compact ? p->ws_bytes_compact : p->ws_bytes; }

// One persistent launch of a step over the units of its member beams.
struct BatchLaunch {
  int kind = 0;
  int wave = 0;
  int q1 = 0, split = 0, nwc = 0, mode = 0, half = 0, pipe = 0;  // template selectors
  int grid = 0, threads = 0, smem = 0;
  int nmem = 0, nunits = 0;                  // member beams, work units (stage 1: the plans' items)
  int64_t off = 0, mem = 0;                  // offsets of the unit-offset / member arrays in the table
  int64_t ctr = 0;                           // stage 1: offset of the launch's item counter in the table
  int layout = 0;                            // stage 1 mL, stage 2 slot words, boxcar wmaxL
  int aux = 0;                               // stage 2 words of a group's delays (or chunk sub-bands), boxcar tileL
};

int64_t mod64(int64_t a, int64_t r) { return ((a % r) + r) % r; }

}  // namespace

struct tx_batch {
  int n = 0, device = -1, flags = 0, nwaves = 0, num_sms = 0, slot = -1;
  std::vector<const tx_plan*> plans;
  std::vector<tx_beam*> beams;
  std::vector<int> wave_first;   // first beam of each wave, plus n
  std::vector<int64_t> ws_off;   // per beam, inside the shared workspace (waves reuse it)
  int64_t ws_bytes = 0;
  int64_t dm_samples = 0;
  std::vector<BatchLaunch> launches;  // wave by wave
  BeamArgs* d_slot = nullptr;    // device address of the batch's constant-memory slot
  int32_t* d_tab = nullptr;      // unit offsets and member lists of every launch
  BeamArgs* h_args[2] = {nullptr, nullptr};  // pinned, alternating between steps
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaStream_t cap = nullptr;    // private stream for graph capture
  int64_t nsteps = 0;
  // TX_BATCH_PROFILE: an event before each launch and one after the last
  std::vector<cudaEvent_t> prof_ev;
  bool prof_pending = false;
  double prof_ms[TX_NPHASES] = {0, 0, 0, 0, 0};
  int32_t prof_steps = 0;
};

namespace {

// The kernel a batched launch runs.
const void* launch_kernel(const BatchLaunch& L) {
  switch (L.kind) {
    case kIngest: return (const void*)k_ingest_batch<SlotArgs>;
    case kTailIn:
    case kTailOut: return (const void*)k_tail<SlotArgs>;
    case kOffsets: return (const void*)k_offsets<SlotArgs>;
    case kStage1:
#define TX_K1(Q) (L.half ? (const void*)k_stage1<Q, uint16_t, SlotArgs, true> : (const void*)k_stage1<Q, uint16_t, SlotArgs>)
      switch (L.q1) {
        case 256: return TX_K1(256);
        case 128: return TX_K1(128);
        case 64: return TX_K1(64);
        default: return TX_K1(32);
      }
#undef TX_K1
    case kStage2:
      if (L.pipe) return stage2_pipe_kernel<SlotArgs>(L.split, L.half);
#define TX_K2(NW, SP)                                                        \
  (L.half ? (const void*)k_stage2_u16<NW, 32, SP, SlotArgs, true>            \
          : (const void*)k_stage2_u16<NW, 32, SP, SlotArgs, false>)
      switch (L.split) {
        case 8: return TX_K2(512, 8);
        case 4: return TX_K2(512, 4);
        case 2: return TX_K2(512, 2);
        default: return TX_K2(256, 1);
      }
#undef TX_K2
    case kStats: return (const void*)k_stats<SlotArgs>;
    default: return (const void*)box_kernel<SlotArgs>(L.nwc, L.mode);
  }
}

int build_batch(tx_batch* B, int64_t budget) {
  const int n = B->n;
  // ---- waves: consecutive beams within the workspace budget and a slot --------
  B->ws_off.assign(n, 0);
  B->wave_first.assign(1, 0);
  int64_t cur = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t need = beam_ws(B->plans[i], B->beams[i]);
    if (budget > 0 && need > budget) {
      set_error("beam %d needs %lld workspace bytes, more than the budget %lld", i, (long long)need, (long long)budget);
      return TX_ERR_BUDGET;
    }
    const bool full = i - B->wave_first.back() == kArgSlotBeams;
    if (i > 0 && (full || (budget > 0 && cur + need > budget))) {
      B->wave_first.push_back(i);
      cur = 0;
    }
    B->ws_off[i] = cur;
    cur += need;
    B->ws_bytes = std::max(B->ws_bytes, cur);
    B->dm_samples += (int64_t)B->plans[i]->ndm * B->plans[i]->T;
  }
  B->wave_first.push_back(n);
  B->nwaves = (int)B->wave_first.size() - 1;

  std::vector<int32_t> tab;
  // unit offsets and member list (wave-local indices) of one launch
  auto add_members = [&](BatchLaunch& L, const std::vector<int>& mem, int first, auto units_of) -> int {
    L.nmem = (int)mem.size();
    L.off = (int64_t)tab.size();
    int64_t total = 0;
    for (int b : mem) {
      tab.push_back((int32_t)total);
      total += units_of(b);
    }
    tab.push_back((int32_t)total);
    if (total >= INT32_MAX) { set_error("a batched launch has too many work units (%lld)", (long long)total); return TX_ERR_UNSUPPORTED; }
    L.mem = (int64_t)tab.size();
    for (int b : mem) tab.push_back(b - first);
    L.nunits = (int)total;
    return TX_OK;
  };
  const int nsm = std::max(B->num_sms, 1);
  int rc;

  for (int wv = 0; wv < B->nwaves; ++wv) {
    const int first = B->wave_first[wv];
    std::vector<int> mem;
    for (int i = first; i < B->wave_first[wv + 1]; ++i) mem.push_back(i);
    // ---- compact beams: tails into their borrowed rings ---------------------------
    std::vector<int> compact;
    for (int b : mem)
      if (B->beams[b]->compact && B->plans[b]->L > 0) compact.push_back(b);
    auto tail_launch = [&](int kind) -> int {
      BatchLaunch L;
      L.kind = kind;
      L.wave = wv;
      const int r = add_members(L, compact, first, [&](int b) -> int64_t {
        const tx_plan* p = B->plans[b];
        return (int64_t)p->nchan * ((p->tail_pitch + 4095) / 4096);
      });
      if (r) return r;
      L.threads = 256;
      L.grid = std::min(L.nunits, nsm * 8);
      if (L.nunits > 0) B->launches.push_back(L);
      return TX_OK;
    };
    if (!compact.empty() && (rc = tail_launch(kTailIn))) return rc;
    // ---- ingest: every beam of the wave ------------------------------------------
    {
      BatchLaunch L;
      L.kind = kIngest;
      L.wave = wv;
      rc = add_members(L, mem, first, [&](int b) -> int64_t {
        const tx_plan* p = B->plans[b];
        return p->layout == TX_LAYOUT_TF ? ((p->T + 63) / 64) * ((p->nchan + 63) / 64)
                                         : (int64_t)p->nchan * ((p->T + 4095) / 4096);
      });
      if (rc) return rc;
      L.threads = 256;
      L.grid = std::min(L.nunits, nsm * 8);
      if (L.nunits > 0) B->launches.push_back(L);
    }
    // ---- compact beams: the new tails out ------------------------------------------
    if (!compact.empty() && (rc = tail_launch(kTailOut))) return rc;
    // ---- half intermediates: the block's per-sub-band offsets (ingest zeroed them) ----
    {
      std::vector<int> hm;
      for (int b : mem)
        if (B->plans[b]->interm == TX_INTERM_F16) hm.push_back(b);
      if (!hm.empty()) {
        BatchLaunch L;
        L.kind = kOffsets;
        L.wave = wv;
        if ((rc = add_members(L, hm, first, [&](int b) -> int64_t { return B->plans[b]->nchan; }))) return rc;
        L.threads = 256;
        L.grid = std::min(L.nunits, nsm * 8);
        B->launches.push_back(L);
      }
    }
    // ---- stage 1, one launch per (tile length, channels per sub-band): the shared
    // memory of a launch is laid out for its largest sub-band, and a mix would
    // take carve-out from L1 for the smaller ones
    std::map<std::tuple<int, int, int>, std::vector<int>> by_q;
    for (int b : mem)
      by_q[{B->plans[b]->q1, B->plans[b]->m, B->plans[b]->interm == TX_INTERM_F16}].push_back(b);
    for (auto& kv : by_q) {
      BatchLaunch L;
      L.kind = kStage1;
      L.wave = wv;
      L.q1 = std::get<0>(kv.first);
      L.half = std::get<2>(kv.first);
      if ((rc = add_members(L, kv.second, first, [&](int b) -> int64_t { return (int64_t)B->plans[b]->items1.size(); })))
        return rc;
      L.layout = std::get<1>(kv.first);  // channels per sub-band of every member
      const int mL = L.layout;
      L.smem = (int)stage1_smem_bytes(mL, L.q1);
      if (L.smem > kSmemMax) { set_error("stage-1 shared memory for %d channels per sub-band exceeds the limit", mL); return TX_ERR_UNSUPPORTED; }
      L.threads = kStage1Warps * 32;
      L.grid = std::min(L.nunits, nsm);
      L.ctr = (int64_t)tab.size();
      tab.push_back(0);
      if (L.nunits > 0) B->launches.push_back(L);
    }
    // ---- stage 2, one launch per (warp split, sub-bands per chunk, block size) -------
    // Shared memory is laid out for the largest staged chunk and table of the
    // launch (which the plans size to fit, with room for the static sums); a
    // block as large as its largest group would idle warps of smaller groups.
    std::map<std::tuple<int, int, int, int, int, int>, std::vector<int>> by_split;
    for (int b : mem)
      by_split[{B->plans[b]->pipe2, stage2_split(B->plans[b]), B->plans[b]->nsub_chunk2, stage2_threads(B->plans[b]),
                B->plans[b]->interm == TX_INTERM_F16, B->plans[b]->e2w2}].push_back(b);
    auto s2_smem = [&](const std::vector<int>& g) {
      int slot = 0, sc = 0, e2w = 0;
      for (int b : g) {
        slot = std::max(slot, B->plans[b]->nsub_chunk2 * B->plans[b]->sww2);
        sc = std::max(sc, B->plans[b]->nsub_chunk2);
        e2w = std::max(e2w, B->plans[b]->e2w2);
      }
      return std::make_tuple(slot, stage2_u16_smem_for(slot, sc, e2w), e2w);
    };
    for (auto& kv : by_split) {
      BatchLaunch L;
      L.kind = kStage2;
      L.wave = wv;
      L.pipe = std::get<0>(kv.first);
      L.split = std::get<1>(kv.first);
      L.half = std::get<4>(kv.first);
      if ((rc = add_members(L, kv.second, first,
                            [&](int b) -> int64_t { return (int64_t)B->plans[b]->nk * B->plans[b]->ntile2; })))
        return rc;
      int threads = 0;
      for (int b : kv.second) threads = std::max(threads, stage2_threads(B->plans[b]));
      const auto sm = s2_smem(kv.second);
      L.layout = std::get<0>(sm);
      L.smem = std::get<1>(sm);
      L.aux = std::get<2>(sm);
      if (L.pipe) {   // stages of the largest chunk (slot words) and address table (aux: sub-bands per chunk)
        int sc = 0;
        for (int b : kv.second) sc = std::max(sc, B->plans[b]->nsub_chunk2);
        L.aux = sc;
        L.smem = (int)((int64_t)kPipeStages2 * (2 * (int64_t)L.layout + (int64_t)(kPipeMaxGroup2 + 1) * ((sc + 3) & ~3)) * 4);
      }
      if (L.smem > kSmemMax - 1024) { set_error("batched stage-2 shared memory (%d bytes) exceeds the limit", L.smem); return TX_ERR_UNSUPPORTED; }
      L.threads = threads;
      L.grid = std::min(L.nunits, nsm);
      if (L.nunits > 0) B->launches.push_back(L);
    }
    // ---- statistics, then boxcar per (width class, output mode) ----------------------
    std::vector<int> filt;
    for (int b : mem)
      if (B->plans[b]->output != TX_OUT_SERIES) filt.push_back(b);
    if (!filt.empty()) {
      BatchLaunch L;
      L.kind = kStats;
      L.wave = wv;
      if ((rc = add_members(L, filt, first, [&](int b) -> int64_t { return B->plans[b]->ndm; }))) return rc;
      L.threads = 128;                   // one warp per DM
      L.grid = (L.nunits + 3) / 4;
      B->launches.push_back(L);
    }
    std::map<std::pair<int, int>, std::vector<int>> by_box;
    for (int b : filt) by_box[{box_class(B->plans[b]->nw), B->plans[b]->output}].push_back(b);
    for (auto& kv : by_box) {
      BatchLaunch L;
      L.kind = kBoxcar;
      L.wave = wv;
      L.nwc = kv.first.first;
      L.mode = kv.first.second;
      if ((rc = add_members(L, kv.second, first,
                            [&](int b) -> int64_t { return (int64_t)B->plans[b]->ndm * B->plans[b]->ntile3; })))
        return rc;
      int wm = 0, tl = kBoxTile;
      for (int b : kv.second) {
        wm = std::max(wm, B->plans[b]->wmax);
        tl = std::max(tl, B->plans[b]->box_tile);
      }
      L.layout = wm;
      L.aux = tl;
      L.smem = box_smem_for(tl, wm);
      const void* k = launch_kernel(L);
      TX_CUDA(raise_smem_limit(k, L.smem));  // before the occupancy query
      int bps = 1;
      TX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kBoxThreads, L.smem));
      L.threads = kBoxThreads;
      L.grid = std::min(L.nunits, nsm * std::max(bps, 1));
      if (L.nunits > 0) B->launches.push_back(L);
    }
  }

  // ---- shared memory limit of each batched kernel: the most any launch asks --------
  std::map<const void*, int> need;
  for (const BatchLaunch& L : B->launches) {
    const void* k = launch_kernel(L);
    need[k] = std::max(need[k], L.smem);
  }
  for (auto& kv : need) TX_CUDA(raise_smem_limit(kv.first, kv.second));

  // ---- device tables, pinned argument buffers ----------------------------------
  void* sym = nullptr;
  TX_CUDA(cudaGetSymbolAddress(&sym, c_args));
  B->d_slot = static_cast<BeamArgs*>(sym) + (size_t)B->slot * kArgSlotBeams;
  TX_CUDA(cudaMalloc((void**)&B->d_tab, std::max<size_t>(tab.size(), 1) * 4));
  if (!tab.empty()) TX_CUDA(cudaMemcpy(B->d_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice));
  for (int i = 0; i < 2; ++i) {
    TX_CUDA(cudaHostAlloc((void**)&B->h_args[i], (size_t)n * sizeof(BeamArgs), cudaHostAllocDefault));
    std::memset(B->h_args[i], 0, (size_t)n * sizeof(BeamArgs));
    TX_CUDA(cudaEventCreateWithFlags(&B->done[i], cudaEventDisableTiming));
  }
  TX_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  if (B->flags & TX_BATCH_PROFILE) {
    B->prof_ev.assign(B->launches.size() + 1, nullptr);
    for (auto& e : B->prof_ev) TX_CUDA(cudaEventCreate(&e));
  }
  return TX_OK;
}

// Adds the previous profiled step's launch times to the per-phase sums.
int collect_profile(tx_batch* B) {
  if (!B->prof_pending) return TX_OK;
  TX_CUDA(cudaEventSynchronize(B->prof_ev.back()));
  for (size_t i = 0; i < B->launches.size(); ++i) {
    float ms = 0.f;
    TX_CUDA(cudaEventElapsedTime(&ms, B->prof_ev[i], B->prof_ev[i + 1]));
    B->prof_ms[phase_of(B->launches[i].kind)] += ms;
  }
  ++B->prof_steps;
  B->prof_pending = false;
  return TX_OK;
}

// Enqueues one step: per wave, the copy of its beams' arguments into the
// batch's constant slot, then the wave's launches in order.
int enqueue(tx_batch* B, const BeamArgs* h_src, cudaStream_t st) {
  const bool prof = (B->flags & TX_BATCH_PROFILE) != 0;
  const SlotArgs src{B->slot * kArgSlotBeams};
  int wave = -1;
  for (size_t li = 0; li < B->launches.size(); ++li) {
    const BatchLaunch& L = B->launches[li];
    if (L.wave != wave) {
      wave = L.wave;
      const int first = B->wave_first[wave], cnt = B->wave_first[wave + 1] - first;
      TX_CUDA(cudaMemcpyAsync(B->d_slot, h_src + first, (size_t)cnt * sizeof(BeamArgs), cudaMemcpyHostToDevice, st));
    }
    if (prof) TX_CUDA(cudaEventRecord(B->prof_ev[li], st));
    const int32_t* off = B->d_tab + L.off;
    const int32_t* mem = B->d_tab + L.mem;
    switch (L.kind) {
      case kIngest:
        k_ingest_batch<SlotArgs><<<L.grid, L.threads, 0, st>>>(src, off, mem, L.nmem, L.nunits);
        break;
      case kTailIn:
      case kTailOut:
        k_tail<SlotArgs><<<L.grid, L.threads, 0, st>>>(src, L.kind == kTailOut, off, mem, L.nmem, L.nunits);
        break;
      case kOffsets:
        k_offsets<SlotArgs><<<L.grid, L.threads, 0, st>>>(src, off, mem, L.nmem, L.nunits);
        break;
      case kStage1: {
        int32_t* ictr = B->d_tab + L.ctr;
        TX_CUDA(cudaMemsetAsync(ictr, 0, sizeof(int32_t), st));
#define TX_B1(Q)                                                                                                \
  do {                                                                                                           \
    if (L.half)                                                                                                  \
      k_stage1<Q, uint16_t, SlotArgs, true><<<L.grid, L.threads, L.smem, st>>>(src, off, mem, L.nmem, L.nunits,   \
                                                                               L.layout, 1u, ictr);              \
    else                                                                                                         \
      k_stage1<Q, uint16_t, SlotArgs><<<L.grid, L.threads, L.smem, st>>>(src, off, mem, L.nmem, L.nunits,         \
                                                                         L.layout, 1u, ictr);                    \
  } while (0)
        switch (L.q1) {
          case 256: TX_B1(256); break;
          case 128: TX_B1(128); break;
          case 64: TX_B1(64); break;
          default: TX_B1(32); break;
        }
#undef TX_B1
        break;
      }
      case kStage2:
        if (L.pipe) {
          launch_stage2_pipe<SlotArgs>(L.split, L.half, L.grid, L.threads, L.smem, st, src, off, mem, L.nmem, L.nunits,
                                       L.aux, L.layout);
          break;
        }
#define TX_B2(NW, SP)                                                                                          \
  do {                                                                                                         \
    if (L.half)                                                                                                \
      k_stage2_u16<NW, 32, SP, SlotArgs, true><<<L.grid, L.threads, L.smem, st>>>(src, off, mem, L.nmem,       \
                                                                                  L.nunits, L.layout, L.aux);  \
    else                                                                                                       \
      k_stage2_u16<NW, 32, SP, SlotArgs, false><<<L.grid, L.threads, L.smem, st>>>(src, off, mem, L.nmem,      \
                                                                                   L.nunits, L.layout, L.aux); \
  } while (0)
        switch (L.split) {
          case 8: TX_B2(512, 8); break;
          case 4: TX_B2(512, 4); break;
          case 2: TX_B2(512, 2); break;
          default: TX_B2(256, 1); break;
        }
#undef TX_B2
        break;
      case kStats:
        k_stats<SlotArgs><<<L.grid, L.threads, 0, st>>>(src, off, mem, L.nmem, L.nunits);
        break;
      default:
        box_kernel<SlotArgs>(L.nwc, L.mode)<<<L.grid, L.threads, L.smem, st>>>(src, off, mem, L.nmem, L.nunits,
                                                                               L.aux, L.layout);
        break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, launch_kernel(L));
      set_error("batched launch (phase %d, grid %d, %d threads, %d + %zu bytes shared; kernel allows %d threads, "
                "%d dynamic bytes) failed: %s", L.kind, L.grid, L.threads, L.smem, fa.sharedSizeBytes,
                fa.maxThreadsPerBlock, fa.maxDynamicSharedSizeBytes, cudaGetErrorString(e));
      return TX_ERR_CUDA;
    }
  }
  if (prof) {
    TX_CUDA(cudaEventRecord(B->prof_ev.back(), st));
    B->prof_pending = true;
  }
  return TX_OK;
}

}  // namespace

extern "C" {

int32_t tx_batch_create(int32_t n, const tx_plan* const* plans, tx_beam* const* beams, int64_t workspace_budget,
                        int32_t flags, tx_batch** out) {
  if (!out || !plans || !beams || n < 1) { set_error("need n >= 1 plans and beams and an output handle"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  if (flags & ~(TX_BATCH_GRAPH | TX_BATCH_PROFILE)) { set_error("unknown batch flags 0x%x", flags); return TX_ERR_INVALID_ARG; }
  if ((flags & TX_BATCH_GRAPH) && (flags & TX_BATCH_PROFILE)) { set_error("TX_BATCH_PROFILE needs direct launches (no TX_BATCH_GRAPH)"); return TX_ERR_INVALID_ARG; }
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device %d out of range", dev); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < n; ++i) {
    const tx_plan* p = plans[i];
    const tx_beam* b = beams[i];
    if (!p || !b) { set_error("null plan or beam at %d", i); return TX_ERR_INVALID_ARG; }
    if (b->plan != p) { set_error("beam %d was created for another plan", i); return TX_ERR_INVALID_ARG; }
    if (b->device != dev) { set_error("beam %d lives on device %d, current device is %d", i, b->device, dev); return TX_ERR_INVALID_ARG; }
    if (p->interm == TX_INTERM_I32 || p->interm == TX_INTERM_F32) { set_error("batched execute needs 16-bit intermediates (beam %d)", i); return TX_ERR_UNSUPPORTED; }
    for (int j = 0; j < i; ++j)
      if (beams[j] == b) { set_error("beam %d appears twice in the batch", i); return TX_ERR_INVALID_ARG; }
    int rc = tx_upload_plan(p);
    if (rc) return rc;
  }
  tx_batch* B = new (std::nothrow) tx_batch();
  if (!B) { set_error("out of host memory"); return TX_ERR_OOM; }
  B->n = n;
  B->device = dev;
  B->flags = flags;
  B->plans.assign(plans, plans + n);
  B->beams.assign(beams, beams + n);
  {
    std::lock_guard<std::mutex> g(g_slot_mu);
    for (int s = 0; s < kArgSlots; ++s)
      if (!g_slot_used[dev][s]) {
        g_slot_used[dev][s] = true;
        B->slot = s;
        break;
      }
  }
  if (B->slot < 0) {
    delete B;
    set_error("all %d batch argument slots of device %d are in use (destroy a batch first)", kArgSlots, dev);
    return TX_ERR_BUDGET;
  }
  int rc = TX_OK;
  if (cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("cudaDeviceGetAttribute failed");
    rc = TX_ERR_CUDA;
  }
  if (rc == TX_OK) {
    try {
      rc = build_batch(B, workspace_budget);
    } catch (const std::bad_alloc&) {
      set_error("out of host memory");
      rc = TX_ERR_OOM;
    }
  }
  if (rc) { tx_batch_destroy(B); return rc; }
  *out = B;
  return TX_OK;
}

int32_t tx_batch_get_info(const tx_batch* B, tx_batch_info* info) {
  if (!B || !info) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  std::memset(info, 0, sizeof(*info));
  info->nbeams = B->n;
  info->nwaves = B->nwaves;
  info->nlaunches = (int32_t)B->launches.size();
  info->flags = B->flags;
  info->workspace_bytes = B->ws_bytes;
  info->dm_trial_samples = B->dm_samples;
  return TX_OK;
}

int32_t tx_execute_batch(tx_batch* B, const uint8_t* const* d_blocks, void* const* d_outs, int64_t* const* d_ncands,
                         void* d_workspace, void* stream) {
  if (!B || !d_blocks || !d_outs || !d_workspace) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev != B->device) { set_error("batch lives on device %d, current device is %d", B->device, dev); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < B->n; ++i) {
    if (!d_blocks[i] || !d_outs[i]) { set_error("null block or output of beam %d", i); return TX_ERR_INVALID_ARG; }
    if (B->plans[i]->output == TX_OUT_CANDS && (!d_ncands || !d_ncands[i])) { set_error("beam %d is in candidate mode and needs d_ncands", i); return TX_ERR_INVALID_ARG; }
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = collect_profile(B);
  if (rc) return rc;
  const int slot = (int)(B->nsteps & 1);
  if (B->used[slot]) TX_CUDA(cudaEventSynchronize(B->done[slot]));  // the step that last read this buffer
  BeamArgs* h = B->h_args[slot];
  uint8_t* ws = static_cast<uint8_t*>(d_workspace);
  for (int i = 0; i < B->n; ++i) {
    const tx_plan* p = B->plans[i];
    tx_beam* b = B->beams[i];
    const int64_t start = mod64(b->head - p->L, p->R);
    h[i] = make_args(p, b, d_blocks[i], d_outs[i], d_ncands ? d_ncands[i] : nullptr, ws + B->ws_off[i], b->head,
                     start);
  }
  if (B->flags & TX_BATCH_GRAPH) {
    if (!B->exec[slot]) {
      cudaGraph_t g = nullptr;
      TX_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
      rc = enqueue(B, h, B->cap);
      const cudaError_t e = cudaStreamEndCapture(B->cap, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      TX_CUDA(e);
      const cudaError_t ei = cudaGraphInstantiate(&B->exec[slot], g, 0);
      cudaGraphDestroy(g);
      TX_CUDA(ei);
    }
    TX_CUDA(cudaGraphLaunch(B->exec[slot], st));
  } else {
    rc = enqueue(B, h, st);
    if (rc) return rc;
  }
  TX_CUDA(cudaEventRecord(B->done[slot], st));
  B->used[slot] = true;
  ++B->nsteps;
  for (int i = 0; i < B->n; ++i) {
    tx_beam* b = B->beams[i];
    if (!b->compact) b->head = mod64(b->head + B->plans[i]->T, B->plans[i]->R);
    ++b->nblocks;
  }
  return TX_OK;
}

}  // extern "C"

int batch_wait_timeouts(int64_t* n) {
  int v = 0;
  TX_CUDA(cudaMemcpyFromSymbol(&v, g_tx_wait_timeouts, sizeof(int)));
  *n = v;
  return TX_OK;
}

extern "C" {

int32_t tx_batch_wait(tx_batch* B, int64_t timeout_us) {
  if (!B) { set_error("null batch"); return TX_ERR_INVALID_ARG; }
  if (!B->nsteps) return TX_OK;
  const cudaEvent_t ev = B->done[(B->nsteps - 1) & 1];
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) {
      // the members' counts of waits their kernels gave up
      // (copied on the batch's private non-blocking stream: nothing else waits)
      for (int i = 0; i < B->n; ++i) {
        int32_t v = 0;
        TX_CUDA(cudaMemcpyAsync(&v, B->beams[i]->fail, sizeof(v), cudaMemcpyDeviceToHost, B->cap));
        TX_CUDA(cudaStreamSynchronize(B->cap));
        if (v) {
          set_error("the kernels of beam %d gave up %d waits: its results are not valid (reset the beam)", i, v);
          return TX_ERR_ABORTED;
        }
      }
      return TX_OK;
    }
    if (e != cudaErrorNotReady) {
      set_error("waiting for the batch failed: %s", cudaGetErrorString(e));
      return TX_ERR_CUDA;
    }
    const int64_t el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_us >= 0 && el >= timeout_us) {
      set_error("the batch's last step did not finish within %lld us", (long long)timeout_us);
      return TX_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int32_t tx_batch_read_profile(tx_batch* B, double* h_ms, int32_t* nsteps) {
  if (!B || !h_ms) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (!(B->flags & TX_BATCH_PROFILE)) { set_error("the batch was created without TX_BATCH_PROFILE"); return TX_ERR_INVALID_ARG; }
  const int rc = collect_profile(B);
  if (rc) return rc;
  for (int i = 0; i < TX_NPHASES; ++i) h_ms[i] = B->prof_ms[i];
  if (nsteps) *nsteps = B->prof_steps;
  return TX_OK;
}

void tx_batch_destroy(tx_batch* B) {
  if (!B) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (B->device >= 0) cudaSetDevice(B->device);
  for (int i = 0; i < 2; ++i) {
    if (B->used[i]) cudaEventSynchronize(B->done[i]);
    if (B->exec[i]) cudaGraphExecDestroy(B->exec[i]);
    if (B->done[i]) cudaEventDestroy(B->done[i]);
    if (B->h_args[i]) cudaFreeHost(B->h_args[i]);
  }
  if (B->cap) cudaStreamDestroy(B->cap);
  for (auto e : B->prof_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(B->d_tab);
  if (B->slot >= 0 && B->device >= 0) {
    std::lock_guard<std::mutex> g(g_slot_mu);
    g_slot_used[B->device][B->slot] = false;
  }
  cudaSetDevice(prev);
  delete B;
}

}  // extern "C"
