// Device kernels (sm_103a) of the hot path: ingest, two-stage sub-band
// de-dispersion (Sec. 2.3), block statistics, and the boxcar matched filter
// with its outputs (Sec. 2.4, 2.5). Included by kernels.cu (one beam per
// execute) and batch.cu (many beams of uneven shape per launch); each
// translation unit instantiates the templates it launches.
//
// Kernel map (one execute):
//   k_ingest_*   Sec. 2.3 data-flow steps 1, 2 and 4: the new block lands
//                channel-major in the beam's circular buffer behind the carried
//                tail (time-major input is transposed on the way); nothing is
//                shifted, the buffer start advances by T instead.
//   k_stage1     stage 1: P[k][s][t] = sum_{c in s} X[c][t + d1[k][c]]
//   k_stage2_*   stage 2: D[d][t] = sum_s P[k(d)][s][t + d2[d][s]], plus exact
//                per-tile sums of D and D^2
//   k_stats      mean / sigma per DM (block or running) and the per-width
//                constants of Eq. 5
//   k_boxcar     prefix sums, window sums for every width, S/N (Eq. 5), best
//                width, and cube / plane / candidates
//
// Every kernel reads what it needs about a beam from a BeamArgs, through an
// argument source (OneBeam: one beam, a kernel parameter; batched sources:
// the kernel walks the concatenated work units of several member beams,
// finds each unit's member from per-member unit offsets, and reads that
// member's arguments from constant memory).
#pragma once

#include <cuda_fp16.h>
#include <type_traits>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "tx_internal.h"

namespace {

using namespace tx;

// ---------------------------------------------------------------------------
// per-beam arguments of one execute
// ---------------------------------------------------------------------------
struct BeamArgs {
  const uint8_t* block;          // this step's input block (plan layout)
  uint8_t* ring;                 // [nchan][R] circular buffer
  void* P;                       // stage-1 sums [nk][nsub][Pp] (uint16 or int32)
  int32_t* D;                    // series [ndm][Dp]
  longlong2* part;               // per-tile (sum D, sum D^2) [ndm][ntile2]
  SnrConst* cst;                 // per (DM, width) S/N constants [ndm][nw]
  double* run;                   // running (mu, var) [ndm][2], then the beam's count of waits its kernels
                                 // gave up (int32; no count when run is null)
  const int32_t* d1;             // [nk][nchan]
  const int32_t* abase;          // [nk][nsub]
  const int32_t* e2;             // [ndm][nsub]
  const int32_t* widths;         // [nw]
  const Stage1Item* items;       // stage-1 work items of the plan
  const int32_t* tab1;           // their precomputed offset tables (window phase tab1_phase)
  const int32_t* tab2;           // pipelined stage 2: offset tables per (coarse group, sub-band chunk)
  float* outf;                   // cube / plane S/N
  uint8_t* outw;                 // plane best-width index
  tx_cand* cands;                // candidate records
  unsigned long long* ncand;     // candidate counter
  uint8_t* tail;                 // compact beams: [nchan][tail_pitch] carried tail
  int32_t* hoff;                 // half intermediates: per-sub-band offsets [nsub], then their sum
  int64_t R, head, start, T, Pp, Dp, Td, max_cands;
  int64_t L, tail_pitch;
  double lam, gamma;
  int32_t nchan, m, nsub, ndm, G, split2, SC, SWW, ntile2, ntile3, nw, wmax;  // split2: part entries per stage-2 tile
  int32_t tail_pad, tab1_phase;
  int32_t box_tile;              // boxcar outputs per unit (a multiple of kBoxTile)
  uint32_t polls;                // polling limit of the first wait for each bulk copy
  int8_t layout, ingest_vec, running, output, compact, half, box_vec;
};
// Two constant-memory slots of kArgSlotBeams of these fit the 64 KB bank.
static_assert(sizeof(BeamArgs) <= 352, "BeamArgs grew");

// Where a kernel finds a beam's arguments (the Src template parameter).
// OneBeam holds them as a kernel parameter (one execute, constant bank); the
// batched source of batch.cu reads member i of a launch from a constant-memory
// slot. Both return the arguments by value so that a kernel loads only the
// fields it uses. Src::kBatch selects the walk over several members' units.
struct OneBeam {
  static constexpr bool kBatch = false;
  BeamArgs a;
  __device__ __forceinline__ BeamArgs get(int) const { return a; }
};

// Member j of a batched launch owns units [off[j], off[j + 1]); returns the
// j with off[j] <= u < off[j + 1] (off has n + 1 entries).
__device__ __forceinline__ int find_member(const int32_t* __restrict__ off, int n, int u) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= u) lo = mid; else hi = mid;
  }
  return lo;
}

// Member lookup for a unit index that only grows (a block's units in turn):
// the member's range stays in registers and is searched only when the unit
// leaves it, walking forward (at most nmem steps over a whole kernel).
struct MemberCursor {
  int j = -1, lo = 0, hi = 0, beam = 0;  // member, its unit range, its argument index
  // returns true when u belongs to another member than the previous call's
  __device__ __forceinline__ bool seek(const int32_t* __restrict__ off, const int32_t* __restrict__ mem, int n,
                                       int u) {
    if (j >= 0 && u >= lo && u < hi) return false;
    if (j < 0 || u < lo) {
      j = find_member(off, n, u);
    } else {
      while (u >= __ldg(off + j + 1)) ++j;
    }
    lo = __ldg(off + j);
    hi = __ldg(off + j + 1);
    beam = __ldg(mem + j);
    return true;
  }
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
// a * one + c with `one` a runtime value (always 1): the add is issued as an
// integer multiply-add on the FMA pipe, leaving the ALU pipe to the byte
// permutes and the other adds.
__device__ __forceinline__ void madd(uint32_t& acc, uint32_t a, uint32_t one) {
  asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(one));
}

// acc += a >> 16 as one integer multiply-add on the FMA pipe: the high 32 bits
// of a * 65536 are a >> 16.
__device__ __forceinline__ void madd_hi16(uint32_t& acc, uint32_t a) {
  asm("mad.hi.u32 %0, %1, 65536, %0;" : "+r"(acc) : "r"(a));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }

// Bulk (TMA) copies into shared memory, completed on an mbarrier: the
// issuing side announces the byte count (expect_tx, one arrival) and each
// copy completes its bytes on the barrier; waiting threads poll the phase.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this CTA's earlier generic-proxy accesses of shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared.b64 st, [%0], %1;\n\t}"
               ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// waits for phase `parity` of bar to complete, giving up after max_iter polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
  for (uint32_t i = 0; i < max_iter; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr uint32_t kMbarPolls = kWaitPolls;   // the full limit

// Waits that gave up (a copy that never completed) in this translation
// unit's kernels; a kernel that saw one returns early and its results are not
// valid. Read by tx_wait_timeouts.
__device__ int g_tx_wait_timeouts = 0;
// Records a wait that gave up: in the counter above and in the beam's own
// count, which marks the beam's state (tail, running statistics) and every
// later result as not valid until the beam is reset or imported.
template <typename A>
__device__ __forceinline__ void record_give_up(const A& a) {
  atomicAdd(&g_tx_wait_timeouts, 1);
  if (a.run) atomicAdd(reinterpret_cast<int32_t*>(a.run + 2 * (size_t)a.ndm), 1);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it in the stream is still
// finishing. Each kernel of the path waits (pdl_wait) before it touches
// memory, so it runs on the completed results of everything before it; and
// lets the next kernel start launching at once (pdl_trigger), so that the
// next kernel's launch and block set-up overlap this one's tail. Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// ingest (Sec. 2.3 data flow)
// ---------------------------------------------------------------------------
// Both ingest kernels also zero *zero (when given): the stage-1 item counter
// of the execute, so that no launch of its own is spent on it.
// Channel-major rows: ring[c][dst_off + i] = src[c][src_off + i], i < n.
__global__ void k_ingest_ft(const uint8_t* __restrict__ src, int64_t src_pitch, int64_t src_off, int64_t n,
                            uint8_t* __restrict__ ring, int64_t R, int64_t dst_off, int vec, int32_t* zero) {
  pdl_wait();
  pdl_trigger();
  if (zero && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *zero = 0;
  const int c = blockIdx.y;
  const uint8_t* s = src + (int64_t)c * src_pitch + src_off;
  uint8_t* d = ring + (int64_t)c * R + dst_off;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (vec) {
    const uint4* s4 = reinterpret_cast<const uint4*>(s);
    uint4* d4 = reinterpret_cast<uint4*>(d);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 16; i += stride) d4[i] = s4[i];
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) d[i] = s[i];
  }
}

constexpr int kIngestTiles = 4;

// This thread's 16 bytes of the 64-time x 64-channel byte tile (times t0..,
// channels c0..) of a time-major block [t][nchan]: time t0 + tid / 4,
// channels c0 + 16 (tid % 4) ..; zero outside the block. 256 threads.
__device__ __forceinline__ uint4 tf_tile_chunk(const uint8_t* __restrict__ src, int64_t t0, int64_t n, int c0,
                                               int nchan, int vec) {
  const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
  const int64_t t = t0 + r;
  const int c = c0 + 16 * q;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (t < n) {
    const uint8_t* sp = src + t * nchan + c;
    if (vec && c + 16 <= nchan) {
      v = __ldg(reinterpret_cast<const uint4*>(sp));
    } else {
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      for (int i = 0; i < 16; ++i)
        if (c + i < nchan) w[i >> 2] |= (uint32_t)sp[i] << (8 * (i & 3));
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  return v;
}

// Loads such a tile into tile[time][channel].
__device__ __forceinline__ void tf_load_tile(uint8_t (*tile)[80], const uint8_t* __restrict__ src, int64_t t0,
                                             int64_t n, int c0, int nchan, int vec) {
  *reinterpret_cast<uint4*>(&tile[threadIdx.x >> 2][16 * (threadIdx.x & 3)]) =
      tf_tile_chunk(src, t0, n, c0, nchan, vec);
}

// Column cc of a tile, times 16 pq .. 16 pq + 15, as four little-endian words.
__device__ __forceinline__ void tf_column(const uint8_t (*tile)[80], int cc, int pq, uint32_t w[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = (uint32_t)tile[16 * pq + 4 * i][cc] | ((uint32_t)tile[16 * pq + 4 * i + 1][cc] << 8) |
           ((uint32_t)tile[16 * pq + 4 * i + 2][cc] << 16) | ((uint32_t)tile[16 * pq + 4 * i + 3][cc] << 24);
}

// Time-major block rows [t][nchan], t in [t_off, t_off + n) -> ring[c][dst_off + t - t_off],
// through 64-time x 64-channel byte tiles, kIngestTiles consecutive ones per
// block (blockIdx.x: times 64 kIngestTiles blockIdx.x ..; blockIdx.y: channels
// 64 blockIdx.y ..). vec: 16-byte loads and stores (nchan, dst_off and the
// source all 16-byte aligned).
__global__ void __launch_bounds__(256) k_ingest_tf(const uint8_t* __restrict__ src, int64_t t_off, int64_t n,
                                                   int nchan, uint8_t* __restrict__ ring, int64_t R,
                                                   int64_t dst_off, int vec, int32_t* zero) {
  __shared__ __align__(16) uint8_t tiles[kIngestTiles][64][80];
  pdl_wait();
  pdl_trigger();
  if (zero && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *zero = 0;
  const int c0 = blockIdx.y * 64;
  uint4 vv[kIngestTiles];   // all of the block's loads in flight at once
#pragma unroll
  for (int i = 0; i < kIngestTiles; ++i)
    vv[i] = tf_tile_chunk(src + t_off * nchan, ((int64_t)blockIdx.x * kIngestTiles + i) * 64, n, c0, nchan, vec);
#pragma unroll
  for (int i = 0; i < kIngestTiles; ++i)
    *reinterpret_cast<uint4*>(&tiles[i][threadIdx.x >> 2][16 * (threadIdx.x & 3)]) = vv[i];
  __syncthreads();
  const int cc = threadIdx.x & 63, pq = threadIdx.x >> 6;
  const int c = c0 + cc;
  if (c >= nchan) return;
#pragma unroll 1
  for (int i = 0; i < kIngestTiles; ++i) {
    const int64_t t0 = ((int64_t)blockIdx.x * kIngestTiles + i) * 64;
    uint32_t w[4];
    tf_column(tiles[i], cc, pq, w);
    const int64_t t = t0 + 16 * pq;
    uint8_t* dp = ring + (int64_t)c * R + dst_off + t;
    if (vec && t + 16 <= n) {
      *reinterpret_cast<uint4*>(dp) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      for (int j = 0; j < 16; ++j)
        if (t + j < n) dp[j] = (uint8_t)(w[j >> 2] >> (8 * (j & 3)));
    }
  }
}

// Batched ingest: persistent blocks walk the tiles of every member beam's
// block and write them into that beam's ring at ring position head + t
// (mod R, R a multiple of 64, so an aligned 16-byte group never straddles the
// wrap). Time-major tiles are 64 times x 64 channels; channel-major tiles are
// 4096 samples of one channel.
template <typename Src>
__global__ void __launch_bounds__(256) k_ingest_batch(const Src src, const int32_t* __restrict__ uoff,
                                                      const int32_t* __restrict__ umem, int nmem, int nunits) {
  __shared__ __align__(16) uint8_t tile[64][80];
  MemberCursor cur, nxt;
  // time-major tiles: this thread's 16 bytes of the block's next tile are loaded
  // while the current tile is transposed and stored
  uint4 pre = make_uint4(0u, 0u, 0u, 0u);
  auto tf_fetch = [&](int u) {
    nxt.seek(uoff, umem, nmem, u);
    const BeamArgs b = src.get(nxt.beam);
    if (b.layout != TX_LAYOUT_TF) return;
    const int lu = u - nxt.lo, nct = (b.nchan + 63) >> 6;
    pre = tf_tile_chunk(b.block, (int64_t)(lu / nct) * 64, b.T, (lu % nct) * 64, b.nchan, b.ingest_vec);
  };
  if ((int)blockIdx.x < nunits) tf_fetch(blockIdx.x);
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    cur.seek(uoff, umem, nmem, u);
    const int lu = u - cur.lo;
    const BeamArgs a = src.get(cur.beam);
    if (a.half && lu == 0)  // k_offsets accumulates into these next
      for (int i = threadIdx.x; i <= a.nsub; i += blockDim.x) a.hoff[i] = 0;
    if (a.layout == TX_LAYOUT_TF) {
      const int nct = (a.nchan + 63) >> 6;
      const int64_t t0 = (int64_t)(lu / nct) * 64;
      const int c0 = (lu % nct) * 64;
      __syncthreads();  // the previous tile's readers are done with `tile`
      *reinterpret_cast<uint4*>(&tile[threadIdx.x >> 2][16 * (threadIdx.x & 3)]) = pre;
      if (u + (int)gridDim.x < nunits) tf_fetch(u + gridDim.x);
      __syncthreads();
      const int cc = threadIdx.x & 63, pq = threadIdx.x >> 6;
      const int c = c0 + cc;
      if (c < a.nchan) {
        uint32_t w[4];
        tf_column(tile, cc, pq, w);
        const int64_t t = t0 + 16 * pq;
        int64_t pos = a.head + t;
        if (pos >= a.R) pos -= a.R;
        uint8_t* row = a.ring + (int64_t)c * a.R;
        if (a.ingest_vec && t + 16 <= a.T) {
          *reinterpret_cast<uint4*>(row + pos) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          for (int i = 0; i < 16; ++i) {
            if (t + i >= a.T) break;
            int64_t pb = pos + i;
            if (pb >= a.R) pb -= a.R;
            row[pb] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
          }
        }
      }
    } else {
      if (u + (int)gridDim.x < nunits) tf_fetch(u + gridDim.x);
      const int nchunk = (int)((a.T + 4095) >> 12);
      const int c = lu / nchunk;
      const int64_t t = (int64_t)(lu - c * nchunk) * 4096 + 16 * threadIdx.x;
      if (t < a.T) {
        const uint8_t* src = a.block + (int64_t)c * a.T;
        uint8_t* row = a.ring + (int64_t)c * a.R;
        int64_t pos = a.head + t;
        if (pos >= a.R) pos -= a.R;
        if (a.ingest_vec && t + 16 <= a.T) {
          *reinterpret_cast<uint4*>(row + pos) = __ldg(reinterpret_cast<const uint4*>(src + t));
        } else {
          for (int i = 0; i < 16 && t + i < a.T; ++i) {
            int64_t pb = pos + i;
            if (pb >= a.R) pb -= a.R;
            row[pb] = src[t + i];
          }
        }
      }
    }
  }
}

// Compact beams: the carried tail moves between the beam's tail store
// [nchan][tail_pitch] (samples at tail_pad + i) and the borrowed ring, where
// it sits just before the block (ring positions head - L .. head - 1, head a
// multiple of 64; the store and the ring share the 16-byte phase).
//   dir 0, in:  ring[c][head - L - pad + j] = store[c][j], j < tail_pitch (the
//               pad bytes land before the window, where nothing reads them
//               into a sum);
//   dir 1, out: store[c][pad + i] = ring[c][head - L + T + i], i < L: the last
//               L samples of the buffer, the next block's tail.
// 16-byte chunks throughout, except dir 1 when T is not a multiple of 16.
// Units: (channel, 4096-byte chunk) of every member in turn; 256 threads.
template <typename Src>
__global__ void __launch_bounds__(256) k_tail(const Src src, int dir, const int32_t* __restrict__ uoff,
                                              const int32_t* __restrict__ umem, int nmem, int nunits) {
  MemberCursor cur;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    int lu = u;
    BeamArgs a;
    if constexpr (Src::kBatch) {
      cur.seek(uoff, umem, nmem, u);
      lu = u - cur.lo;
      a = src.get(cur.beam);
    } else {
      a = src.get(0);
    }
    const int nchunk = (int)((a.tail_pitch + 4095) >> 12);
    const int c = lu / nchunk;
    const int64_t j = (int64_t)(lu - c * nchunk) * 4096 + 16 * threadIdx.x;
    uint8_t* store = a.tail + (int64_t)c * a.tail_pitch;
    uint8_t* ring = a.ring + (int64_t)c * a.R + (a.head - a.L - a.tail_pad);
    if (j >= a.tail_pitch) continue;
    if (dir == 0) {
      *reinterpret_cast<uint4*>(ring + j) = *reinterpret_cast<const uint4*>(store + j);
    } else if (a.T % 16 == 0) {
      *reinterpret_cast<uint4*>(store + j) = *reinterpret_cast<const uint4*>(ring + a.T + j);
    } else {
      for (int64_t i = j; i < j + 16; ++i)
        if (i >= a.tail_pad) store[i] = ring[a.T + i];
    }
  }
}

// Half intermediates: the integer offset of sub-band s is
//   o_s = sum_{c in s} rnd(sum_t X[c][t] / T)
// over the block's T new samples (ring positions head .. head + T - 1 mod R),
// rnd rounding half up. hoff[s] = o_s and hoff[nsub] = sum_s o_s accumulate
// with integer atomics (order-free) from zero (set by the ingest). Units:
// channels of every member in turn; 256 threads read 16-byte aligned chunks
// of the ring and count only the bytes inside the block.
__device__ __forceinline__ uint32_t byte_sum(uint32_t w) { return __dp4a(w, 0x01010101u, 0u); }

template <typename Src>
__global__ void __launch_bounds__(256) k_offsets(const Src src, const int32_t* __restrict__ uoff,
                                                 const int32_t* __restrict__ umem, int nmem, int nunits) {
  __shared__ unsigned long long red[8];
  MemberCursor cur;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    int lu = u;
    BeamArgs a;
    if constexpr (Src::kBatch) {
      cur.seek(uoff, umem, nmem, u);
      lu = u - cur.lo;
      a = src.get(cur.beam);
    } else {
      a = src.get(0);
    }
    const int c = lu;
    const uint8_t* row = a.ring + (int64_t)c * a.R;
    unsigned long long part = 0;
    // the block's samples: [head, head + T) of the ring, in at most two ranges
    const int64_t e0 = a.head + a.T;
    for (int r = 0; r < 2; ++r) {
      const int64_t b = r == 0 ? a.head : 0;
      const int64_t e = r == 0 ? (e0 < a.R ? e0 : a.R) : (e0 > a.R ? e0 - a.R : 0);
      for (int64_t q = (b & ~(int64_t)15) + 16 * (int64_t)threadIdx.x; q < e; q += 16 * (int64_t)blockDim.x) {
        const uint4 w = *reinterpret_cast<const uint4*>(row + q);
        if (q >= b && q + 16 <= e) {
          part += byte_sum(w.x) + byte_sum(w.y) + byte_sum(w.z) + byte_sum(w.w);
        } else {
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
          for (int i = 0; i < 16; ++i)
            if (q + i >= b && q + i < e) part += (ws[i >> 2] >> (8 * (i & 3))) & 0xFFu;
        }
      }
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) part += __shfl_xor_sync(0xffffffffu, part, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      const int mean = (int)((2 * tot + (unsigned long long)a.T) / (2 * (unsigned long long)a.T));
      atomicAdd(a.hoff + c / a.m, mean);
      atomicAdd(a.hoff + a.nsub, mean);
    }
    __syncthreads();
  }
}

// De-dispersion plans (Sec. 2.3, last paragraph): the block averaged over f
// consecutive samples per channel, rounded half up, so it stays uint8:
//   out[t'] = (sum_{i<f} in[f t' + i] + f / 2) / f,  t' < n / f.
// Time-major blocks [t][nchan] are read four channels per 32-bit word when
// nchan is a multiple of four (vec), byte by byte otherwise; channel-major
// blocks [nchan][n] one output per thread.
__global__ void __launch_bounds__(256) k_downsample(const uint8_t* __restrict__ in, int layout, int nchan, int64_t n,
                                                    int f, int vec, uint8_t* __restrict__ out) {
  const int64_t nout = n / f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint32_t half = (uint32_t)(f >> 1);
  if (layout == TX_LAYOUT_TF && vec) {
    const int nw = nchan >> 2;
    const int64_t total = nout * nw;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
      const int64_t t = i / nw;
      const int w = (int)(i - t * nw);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(in + t * f * nchan) + w;
      uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int k = 0; k < f; ++k) {
        const uint32_t v = __ldg(src + (int64_t)k * nw);
        s0 += v & 0xFFu;
        s1 += (v >> 8) & 0xFFu;
        s2 += (v >> 16) & 0xFFu;
        s3 += v >> 24;
      }
      const uint32_t o = ((s0 + half) / f) | (((s1 + half) / f) << 8) | (((s2 + half) / f) << 16) |
                         (((s3 + half) / f) << 24);
      reinterpret_cast<uint32_t*>(out + t * nchan)[w] = o;
    }
  } else if (layout == TX_LAYOUT_TF) {
    const int64_t total = nout * nchan;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
      const int64_t t = i / nchan;
      const int c = (int)(i - t * nchan);
      uint32_t sum = 0;
      for (int k = 0; k < f; ++k) sum += in[(t * f + k) * nchan + c];
      out[t * nchan + c] = (uint8_t)((sum + half) / f);
    }
  } else {
    const int64_t total = nout * nchan;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
      const int c = (int)(i / nout);
      const int64_t t = i - (int64_t)c * nout;
      const uint8_t* src = in + (int64_t)c * n + t * f;
      uint32_t sum = 0;
      for (int k = 0; k < f; ++k) sum += src[k];
      out[(int64_t)c * nout + t] = (uint8_t)((sum + half) / f);
    }
  }
}

// ---------------------------------------------------------------------------
// stage 1 (Sec. 2.3: de-disperse each sub-band on the coarse DM grid)
// ---------------------------------------------------------------------------
// Sums one coarse DM over the sub-band's m channels for VW words per lane,
// starting at word jbase of the tile, and stores the 4 * VW * 32 outputs.
// Stored form of an exact stage-1 sum v: itself (uint16 or int32), or with
// HALF the FP16 bits of v - off (off the sub-band's integer offset), rounded
// to nearest even and saturated at +-65504.
template <typename PT, bool HALF>
__device__ __forceinline__ PT stage1_store(uint32_t v, int off) {
  if constexpr (HALF) {
    const float x = fminf(fmaxf((float)((int)v - off), -65504.f), 65504.f);
    return (PT)__half_as_ushort(__float2half_rn(x));
  } else {
    return (PT)v;
  }
}

template <int Q, int VW, typename PT, bool HALF>
__device__ __forceinline__ void stage1_sum(const uint32_t* __restrict__ S, const uint32_t* __restrict__ t, int m,
                                           uint32_t one, int lane, int jbase, PT* __restrict__ prow, int rel0,
                                           int64_t Pp, int off) {
  uint32_t aw[VW], ah[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) aw[v] = ah[v] = 0u;
  const uint32_t* base = S + jbase + lane;
  int c = 0;
  for (; c + 3 < m; c += 4) {
    const uint4 oo = *reinterpret_cast<const uint4*>(t + c);
    const uint32_t* r0 = base + oo.x;
    const uint32_t* r1 = base + oo.y;
    const uint32_t* r2 = base + oo.z;
    const uint32_t* r3 = base + oo.w;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const uint32_t w0 = r0[32 * v], w1 = r1[32 * v], w2 = r2[32 * v], w3 = r3[32 * v];
      madd(aw[v], w0, one);
      madd(aw[v], w1, one);
      madd(aw[v], w2, one);
      madd(aw[v], w3, one);
      ah[v] += __byte_perm(w0, 0u, 0x4341) + __byte_perm(w1, 0u, 0x4341);
      ah[v] += __byte_perm(w2, 0u, 0x4341) + __byte_perm(w3, 0u, 0x4341);
    }
  }
  for (; c < m; ++c) {
    const uint32_t* r0 = base + t[c];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const uint32_t w0 = r0[32 * v];
      madd(aw[v], w0, one);
      ah[v] += __byte_perm(w0, 0u, 0x4341);
    }
  }
  const int r = rel0 + jbase;
  if (r >= 0 && (int64_t)r + 4 * Q - jbase <= Pp) {
    // every output inside the row: unguarded stores at fixed offsets
    PT* o = prow + r + lane;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const uint32_t lo = aw[v] - (ah[v] << 8);
      const PT v0 = stage1_store<PT, HALF>(lo & 0xFFFFu, off), v1 = stage1_store<PT, HALF>(ah[v] & 0xFFFFu, off);
      const PT v2 = stage1_store<PT, HALF>(lo >> 16, off), v3 = stage1_store<PT, HALF>(ah[v] >> 16, off);
      o[32 * v] = v0;
      o[32 * v + Q] = v1;
      o[32 * v + 2 * Q] = v2;
      o[32 * v + 3 * Q] = v3;
    }
  } else {
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const int j = lane + 32 * v;
      const uint32_t lo = aw[v] - (ah[v] << 8);
      const uint32_t val[4] = {lo & 0xFFFFu, ah[v] & 0xFFFFu, lo >> 16, ah[v] >> 16};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t u = (uint32_t)(r + j + q * Q);
        if (u < (uint64_t)Pp) prow[u] = stage1_store<PT, HALF>(val[q], off);
      }
    }
  }
}

// Persistent blocks walk the work items (sub-band s, coarse DMs [kb, ke),
// absolute times [tau0, tau0 + 4Q)) of the plan, or in a batch the members'
// items in turn (unit u of member j is item u - off[j] of its plan). For each
// item the channels' input windows (from 16-byte aligned ring positions) are
// brought into a raw buffer by bulk (TMA) copies, one per channel (two where
// a window wraps the ring's end), completed on an mbarrier, while the
// previous item is being summed; they are then rearranged so that shared
// word S[c][j] holds channel c's samples at raw offsets j + qQ in byte q
// (q = 0..3). For coarse DM k the output word j is
// sum_c S[c][j + a_c + d1[k][c] - d1[kb][c]] (a_c the window's
// misalignment): four outputs per 32-bit load whatever the delays.
// Sums use the byte-lane identity
//   sum w = sum(lo lanes) + 256 * sum(hi lanes)  (mod 2^32)
// with the hi lanes (bytes 1, 3) accumulated separately as 16-bit lanes,
// exact for up to 257 channels per sub-band. Warps take (coarse DM, part of
// the tile) tasks; a chunk with few coarse DMs splits each tile between 2, 4
// or 8 warps. Shared memory is laid out for mL channels (the largest sub-band
// of the launch), so an item's prefetch never overlaps the previous item's
// staged words or table. Nothing an item needs is fetched by a dependent
// global load between barriers: a block's first item is blockIdx.x and it
// takes each later one from a counter two items ahead (blocks that drew cheap
// items take more); an item's descriptor is copied to shared memory two items ahead and
// its channels' delays d1[kb][c] one item ahead (both with cp.async), so that
// the next item's windows are issued from shared memory; the offset table
// and the P-row bases of the item's coarse DMs come precomputed with the
// plan (copied in during the staging transform) whenever the window phase
// matches, else they are built after the transform.
template <int Q, typename PT, typename Src, bool HALF = false>
__global__ void __launch_bounds__(kStage1Warps * 32, 1)
k_stage1(const Src src, const int32_t* __restrict__ uoff, const int32_t* __restrict__ umem, int nmem, int nitems,
         int mL, uint32_t unit, int32_t* __restrict__ ictr) {
  extern __shared__ __align__(16) uint8_t smem1[];
  pdl_wait();
  pdl_trigger();
  constexpr int SW = kStage1StagedWords(Q);      // staged words per channel
  constexpr int RB = kStage1RawBytes(Q);         // raw bytes per channel
  constexpr int V = Q / 32;
  const int TSL = (mL + 3) & ~3;
  uint32_t* S = reinterpret_cast<uint32_t*>(smem1);
  uint8_t* raw = smem1 + (size_t)mL * SW * 4;
  uint32_t* tab = reinterpret_cast<uint32_t*>(raw + (size_t)mL * RB);   // [kStage1MaxCoarse][TS] offsets
  int32_t* tabase = reinterpret_cast<int32_t*>(tab + (size_t)kStage1MaxCoarse * TSL);  // P-row base per coarse DM
  Stage1Item* iq = reinterpret_cast<Stage1Item*>(tabase + kStage1MaxCoarse);          // items k, k+1, k+2
  int32_t* wrow = reinterpret_cast<int32_t*>(iq + 3);                                  // [2][TSL] d1[kb][c]
  int32_t* hsub = wrow + 2 * TSL;  // [2] the sub-band's offset of items k, k+1 (half intermediates)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ __align__(8) uint64_t barr;   // completion of the bulk copies of the raw windows
  __shared__ int32_t uq[3];                // the item of each descriptor slot
  uint32_t rphase = 0u;

  MemberCursor cur_c, cur_n, cur_f;  // items being summed / next (prefetched and announced) / two ahead
  auto locate = [&](MemberCursor& c, int u, int& lu) -> BeamArgs {
    if constexpr (Src::kBatch) {
      c.seek(uoff, umem, nmem, u);
      lu = u - c.lo;
      return src.get(c.beam);
    } else {
      lu = u;
      return src.get(0);
    }
  };
  // descriptor of item u into slot sl
  auto fetch_item = [&](int u, int sl) {
    if (u >= nitems) return;
    int lu;
    const BeamArgs a = locate(cur_f, u, lu);
    if (threadIdx.x < 2)
      cp_async16(reinterpret_cast<uint8_t*>(iq + sl) + 16 * threadIdx.x,
                 reinterpret_cast<const uint8_t*>(a.items + lu) + 16 * threadIdx.x);
  };
  // delays d1[kb][c] of item u (descriptor in slot sl) into row w (and its sub-band's offset)
  auto fetch_row = [&](int u, int sl, int w) {
    if (u >= nitems) return;
    int lu;
    const BeamArgs a = locate(cur_n, u, lu);
    const Stage1Item& it = iq[sl];
    const int32_t* d1kb = a.d1 + (size_t)it.kb * a.nchan + it.s * a.m;
    for (int c = threadIdx.x; c < a.m; c += blockDim.x) cp_async4(wrow + w * TSL + c, d1kb + c);
    if (HALF && threadIdx.x == 0) cp_async4(hsub + w, a.hoff + it.s);
  };
  // input windows of item u (descriptor in slot sl, delays in row w): bulk copies of RB bytes per
  // channel (split at the ring's end), issued by lane 0 of the warps; the byte count was announced
  // on barr before the barrier that precedes this call
  auto issue = [&](int u, int sl, int w) {
    int lu;
    const BeamArgs a = locate(cur_n, u, lu);
    const Stage1Item& it = iq[sl];
    const int R = (int)a.R;
    if (lane == 0) {
      fence_proxy_async();   // the transform's reads of raw (ordered by the barrier) before the copies
      for (int c = warp; c < a.m; c += kStage1Warps) {
        int64_t p = a.start + it.tau0 + wrow[w * TSL + c];
        while (p >= R) p -= R;
        const int pa = (int)p & ~15;
        const uint8_t* row = a.ring + (size_t)(it.s * a.m + c) * R;
        uint8_t* dst = raw + (size_t)c * RB;
        const int first = min(RB, R - pa);
        bulk_g2s(dst, row + pa, (uint32_t)first, &barr);
        if (first < RB) bulk_g2s(dst + first, row, (uint32_t)(RB - first), &barr);
      }
    }
  };
  auto announce = [&](int u) {  // thread 0: the bytes of item u's windows
    if (threadIdx.x == 0 && u < nitems) {
      int lu;
      const BeamArgs a = locate(cur_n, u, lu);
      mbar_expect_tx(&barr, (uint32_t)(a.m * RB));
    }
  };

  // A block's first item is blockIdx.x; it takes each later one from the
  // launch's counter (zeroed before the launch) two items ahead, so blocks
  // that drew cheap items take more of them. Warp 0 asks (lane 0) and copies
  // the descriptor; the rest of the block reads the index from uq.
  const int G = gridDim.x;
  const int u0 = blockIdx.x;
  if (u0 >= nitems) return;
  auto take = [&](int sl, bool more) {   // warp 0: the next item into slot sl
    int v = nitems;
    if (more) {
      if (lane == 0) v = G + atomicAdd(ictr, 1);
      v = __shfl_sync(0xffffffffu, v, 0);
    }
    if (lane == 0) uq[sl] = v;
    fetch_item(v, sl);
  };
  if (threadIdx.x == 0) {
    mbar_init(&barr, 1);
    fence_mbar_init();
    uq[0] = u0;
  }
  fetch_item(u0, 0);
  if (warp == 0) take(1, true);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  fetch_row(u0, 0, 0);
  cp_async_commit();
  cp_async_wait_all();
  announce(u0);
  __syncthreads();
  issue(u0, 0, 0);
  for (int k = 0, u = u0; u < nitems; ++k, u = uq[k % 3]) {
    const int sl = k % 3, sl1 = (k + 1) % 3, sl2 = (k + 2) % 3;
    const int un = uq[sl1];   // the next item (taken one item earlier)
    int lu;
    const BeamArgs a = locate(cur_c, u, lu);
    cp_async_wait_all();
    const uint32_t ph = rphase;
    const bool landed = mbar_wait(&barr, ph, a.polls);
    rphase ^= 1u;
    if (__syncthreads_or(!landed)) {
      // a copy never completed: record it, give the copies in flight a last wait at the full limit, give up
      if (threadIdx.x == 0) {
        record_give_up(a);
        mbar_wait(&barr, ph, kMbarPolls);
      }
      return;
    }
    const Stage1Item it = iq[sl];
    const int m = a.m;
    const int TS = (m + 3) & ~3;                 // offset-table row stride (16-byte aligned quads)
    const int c0 = it.s * m;
    const int nkk = it.ke - it.kb;
    // one group: this item's precomputed table and row bases, the descriptor
    // two items ahead, the delays of the next item
    const bool pre = a.tab1 != nullptr && (int)(a.start & 15) == a.tab1_phase;
    if (pre) {
      const int nq = nkk * TS / 4;
      const int32_t* src_t = a.tab1 + it.tab;
      for (int q = threadIdx.x; q < nq; q += blockDim.x) cp_async16(tab + 4 * q, src_t + 4 * q);
      const int32_t* src_b = src_t + nkk * TS;
      for (int q = threadIdx.x; q < (nkk + 3) / 4; q += blockDim.x) cp_async16(tabase + 4 * q, src_b + 4 * q);
    }
    if (warp == 0) take(sl2, un < nitems);
    fetch_row(un, sl1, (k + 1) & 1);
    cp_async_commit();
    // raw -> four-quarter words; lane g builds words 4g .. 4g + 3 of a channel
    const int n4 = (Q + it.span + 15 + 3) >> 2;
    for (int c = warp; c < m; c += kStage1Warps) {
      const uint8_t* rw = raw + (size_t)c * RB;
      uint32_t* srow = S + (size_t)c * SW;
      for (int g = lane; g < n4; g += 32) {
        const int j = g << 2;
        uint32_t r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = *reinterpret_cast<const uint32_t*>(rw + j + q * Q);
        // 4 x 4 byte transpose: word j+i collects byte i of each quarter
        const uint32_t t0 = __byte_perm(r[0], r[1], 0x5140), t1 = __byte_perm(r[0], r[1], 0x7362);
        const uint32_t t2 = __byte_perm(r[2], r[3], 0x5140), t3 = __byte_perm(r[2], r[3], 0x7362);
        uint4 w;
        w.x = __byte_perm(t0, t2, 0x5410);
        w.y = __byte_perm(t0, t2, 0x7632);
        w.z = __byte_perm(t1, t3, 0x5410);
        w.w = __byte_perm(t1, t3, 0x7632);
        *reinterpret_cast<uint4*>(srow + j) = w;
      }
    }
    if (!pre) {
      // word offset of S[c][a_c + d1[k][c] - d1[kb][c]] for every (k, c), and the row bases
      const int32_t* d1kb = wrow + (k & 1) * TSL;
      for (int kk = warp; kk < nkk; kk += kStage1Warps) {
        const int32_t* d1k = a.d1 + (size_t)(it.kb + kk) * a.nchan + c0;
        for (int c = lane; c < m; c += 32) {
          const int32_t wa = (int32_t)((a.start + it.tau0 + d1kb[c]) & 15);
          tab[kk * TS + c] = (uint32_t)(c * SW + wa + d1k[c] - d1kb[c]);
        }
      }
      for (int kk = threadIdx.x; kk < nkk; kk += blockDim.x) tabase[kk] = a.abase[(size_t)(it.kb + kk) * a.nsub + it.s];
    }
    cp_async_wait_all();
    announce(un);
    __syncthreads();
    if (un < nitems) issue(un, sl1, (k + 1) & 1);

    const int off = HALF ? hsub[k & 1] : 0;   // the sub-band's offset (half intermediates)
    // tasks: (coarse DM, part of the tile); split the tile when coarse DMs are few
    int split = 1;
    while (split < V && nkk * split * 2 <= kStage1Warps) split *= 2;
    for (int task = warp; task < nkk * split; task += kStage1Warps) {
      const int kk = task / split, part = task - kk * split;
      const int k1 = it.kb + kk;
      const int64_t ab = tabase[kk];
      if ((int64_t)it.tau0 + 4 * Q <= ab || (int64_t)it.tau0 >= ab + a.Pp) continue;
      PT* prow = static_cast<PT*>(a.P) + ((size_t)k1 * a.nsub + it.s) * a.Pp;
      const int rel0 = (int)((int64_t)it.tau0 - ab);  // |rel0| < 2^30
      const uint32_t* t = tab + kk * TS;
      if (split == 1) {
        stage1_sum<Q, V, PT, HALF>(S, t, m, unit, lane, 0, prow, rel0, a.Pp, off);
      } else if (split == 2) {
        if constexpr (V >= 2) stage1_sum<Q, V / 2, PT, HALF>(S, t, m, unit, lane, part * (Q / 2), prow, rel0, a.Pp, off);
      } else if (split == 4) {
        if constexpr (V >= 4) stage1_sum<Q, V / 4, PT, HALF>(S, t, m, unit, lane, part * (Q / 4), prow, rel0, a.Pp, off);
      } else {
        if constexpr (V >= 8) stage1_sum<Q, V / 8, PT, HALF>(S, t, m, unit, lane, part * (Q / 8), prow, rel0, a.Pp, off);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// stage 2 (Sec. 2.3: de-disperse the sub-bands on the fine DM grid)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_sum_stats(long long& s1, unsigned long long& s2) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
}

// Persistent blocks walk units (coarse group k, tile of 2 NW outputs) in
// sub-band chunks; SPLIT warps share fine DM kG + g, each summing NW / SPLIT
// words of the tile. A chunk's uint16 stage-1 rows are copied (bulk TMA
// copies, one per row, issued by lane 0 of the warps in turn and completed on
// the buffer's mbarrier; double-buffered) into shared memory as 32-bit words
// of consecutive pairs (even copy) and re-paired one element later (odd
// copy), so every delay,
// even or odd, is a 32-bit load feeding two outputs. Sums use
//   sum w = sum(lo) + 65536 * sum(hi) (mod 2^32), sum(hi) = sum(w >> 16),
// exact because every stage-2 sum is below 2^32. Shared memory holds two
// buffers of e2w words for the stage-2 delays of a unit's group (rows
// dfirst.. of e2, copied with cp.async one unit ahead so that no delay is a
// dependent global load between barriers), two even-copy slots and one
// odd-copy slot of `slot` words (the largest SC * SWW of the launch) and the
// address table.
template <int NW, int MAXWARPS, int SPLIT, typename Src, bool HALF = false>
__global__ void __launch_bounds__(MAXWARPS * 32, 1)
k_stage2_u16(const Src src, const int32_t* __restrict__ uoff, const int32_t* __restrict__ umem, int nmem, int nunits,
             int slot, int e2w) {
  extern __shared__ __align__(16) uint32_t smem2[];
  pdl_wait();
  pdl_trigger();
  constexpr int VW = NW / 32 / SPLIT;                    // words per lane
  int32_t* E = reinterpret_cast<int32_t*>(smem2);        // [2][e2w] delays of a unit's group
  uint32_t* Se = smem2 + 2 * (size_t)e2w;                // [2][slot]
  uint32_t* So = Se + 2 * (size_t)slot;                  // [slot]
  uint32_t* tab = So + (size_t)slot;                     // [kStage2MaxGroup][SC rounded up to even] word offsets
  __shared__ long long st1[MAXWARPS];
  __shared__ unsigned long long st2[MAXWARPS];
  __shared__ __align__(8) uint64_t bar2[2];  // completion of the bulk copies into even buffer 0 / 1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int g = warp / SPLIT, part_i = warp - g * SPLIT;  // fine DM of the group, part of the tile
  const int jbase = part_i * (NW / SPLIT);
  uint32_t phase[2] = {0u, 0u};

  MemberCursor cur_c, cur_i;  // units being computed / being prefetched
  auto locate = [&](MemberCursor& c, int u, int& lu) -> BeamArgs {
    if constexpr (Src::kBatch) {
      c.seek(uoff, umem, nmem, u);
      lu = u - c.lo;
      return src.get(c.beam);
    } else {
      lu = u;
      return src.get(0);
    }
  };
  // copies the stage-2 delays of unit u's group (rows dfirst .. dfirst + nd - 1) into E buffer eb
  auto fetch_e2 = [&](int u, int eb) {
    int lu;
    const BeamArgs a = locate(cur_i, u, lu);
    const int dfirst = (lu / a.ntile2) * a.G;
    const int n = min(a.G, a.ndm - dfirst) * a.nsub;
    const int32_t* src_e = a.e2 + (size_t)dfirst * a.nsub;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async4(E + (size_t)eb * e2w + i, src_e + i);
  };
  // copies sub-band chunk ch of unit (k, tile) of beam a into even-copy buffer buf (Eu: the group's
  // delays); its byte count was announced on the buffer's mbarrier before the barrier preceding this
  auto issue_chunk = [&](const BeamArgs& a, int k, int64_t t0, int ch, int buf, const int32_t* Eu) {
    const int s0 = ch * a.SC, ns = min(a.SC, a.nsub - s0);
    const uint16_t* P = static_cast<const uint16_t*>(a.P);
    uint32_t* dst = Se + (size_t)buf * slot;
    if (lane == 0) {
      for (int ss = warp; ss < ns; ss += nwarps) {
        const int s = s0 + ss;
        const int64_t b = (t0 + Eu[s]) & ~(int64_t)7;
        fence_proxy_async();
        bulk_g2s(dst + (size_t)ss * a.SWW, P + ((size_t)k * a.nsub + s) * a.Pp + b, (uint32_t)a.SWW * 4u, &bar2[buf]);
      }
    }
  };
  // thread 0: announce the bytes of chunk ch of beam a into buffer buf (before the barrier that precedes the copies)
  auto announce = [&](const BeamArgs& a, int ch, int buf) {
    if (threadIdx.x != 0) return;
    const int ns = min(a.SC, a.nsub - ch * a.SC);
    mbar_expect_tx(&bar2[buf], (uint32_t)ns * (uint32_t)a.SWW * 4u);
  };
  auto announce_unit = [&](int u, int buf) {  // the first chunk of unit u (the unit prefetched next)
    int lu;
    announce(locate(cur_i, u, lu), 0, buf);
  };
  auto issue_unit = [&](int u, int buf, const int32_t* Eu) {  // first chunk of unit u
    int lu;
    const BeamArgs a = locate(cur_i, u, lu);
    const int k = lu / a.ntile2, tile = lu - k * a.ntile2;
    issue_chunk(a, k, (int64_t)tile * 2 * NW, 0, buf, Eu);
  };

  uint32_t aw[VW], ah[VW];   // uint16 pairs: sum of words, sum of high lanes
  float fl[VW], fh[VW];      // half pairs: FP32 sums of the low and high halves
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    aw[v] = ah[v] = 0u;
    fl[v] = fh[v] = 0.f;
  }
  int buf = 0;
  if ((int)blockIdx.x >= nunits) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar2[0], 1);
    mbar_init(&bar2[1], 1);
    fence_mbar_init();
  }
  fetch_e2(blockIdx.x, 0);
  cp_async_commit();
  cp_async_wait_all();
  announce_unit(blockIdx.x, 0);
  __syncthreads();
  issue_unit(blockIdx.x, 0, E);
  for (int u = blockIdx.x, ju = 0; u < nunits; u += gridDim.x, ++ju) {
    int lu;
    const BeamArgs a = locate(cur_c, u, lu);  // once per unit
    const int32_t* Eu = E + (size_t)(ju & 1) * e2w;  // this unit's delays (rows dfirst ..)
    const int SC = a.SC, SWW = a.SWW, nsub = a.nsub;
    const int SCp = (SC + 1) & ~1;  // table row stride: even, so sub-band pairs load as one uint2
    const int nchunk = (nsub + SC - 1) / SC;
    const int k = lu / a.ntile2, tile = lu - k * a.ntile2;
    const int64_t t0 = (int64_t)tile * 2 * NW;
    const int dfirst = k * a.G;
    const int nd = min(a.G, a.ndm - dfirst);
    for (int ch = 0; ch < nchunk; ++ch, buf ^= 1) {
      const int s0 = ch * SC, ns = min(SC, nsub - s0);
      uint32_t* cur = Se + (size_t)buf * slot;
      cp_async_wait_all();
      const uint32_t ph = phase[buf];
      const bool landed = mbar_wait(&bar2[buf], ph, a.polls);
      phase[buf] ^= 1u;
      if (__syncthreads_or(!landed)) {
        // a copy never completed: record it, give the copies in flight a last wait at the full limit, give up
        if (threadIdx.x == 0) {
          record_give_up(a);
          mbar_wait(&bar2[buf], ph, kMbarPolls);
        }
        return;
      }
      // odd copy: So[ss][i] = (P[2i + 1], P[2i + 2]) relative to the staged base
      for (int ss = warp; ss < ns; ss += nwarps) {
        const uint32_t* r = cur + (size_t)ss * SWW;
        uint32_t* o = So + (size_t)ss * SWW;
        for (int j = 4 * lane; j < SWW - 4; j += 128) {
          const uint4 x = *reinterpret_cast<const uint4*>(r + j);
          const uint32_t y = r[j + 4];
          *reinterpret_cast<uint4*>(o + j) =
              make_uint4(__funnelshift_r(x.x, x.y, 16), __funnelshift_r(x.y, x.z, 16), __funnelshift_r(x.z, x.w, 16),
                         __funnelshift_r(x.w, y, 16));
        }
      }
      if (ch == 0) {
        // the next unit's delays, one unit ahead (landed at this unit's next
        // chunk, or waited for below when this is its only chunk)
        if (u + (int)gridDim.x < nunits) fetch_e2(u + gridDim.x, (ju + 1) & 1);
        cp_async_commit();
      }
      for (int gg = warp; gg < nd; gg += nwarps) {
        for (int ss = lane; ss < ns; ss += 32) {
          const int s = s0 + ss;
          const int32_t emin = Eu[s];
          const int off = Eu[gg * nsub + s] - emin + (int)((t0 + emin) & 7);
          const uint32_t* base = (off & 1) ? So : cur;
          tab[gg * SCp + ss] = (uint32_t)(base - smem2) + (uint32_t)(ss * SWW + (off >> 1));
        }
      }
      if (ch + 1 == nchunk) cp_async_wait_all();   // the next unit's delays, for its first chunk
      if (ch + 1 < nchunk) announce(a, ch + 1, buf ^ 1);
      else if (u + (int)gridDim.x < nunits) announce_unit(u + gridDim.x, buf ^ 1);
      __syncthreads();
      // prefetch the next chunk: of this unit, else the first of the block's next unit
      if (ch + 1 < nchunk) {
        issue_chunk(a, k, t0, ch + 1, buf ^ 1, Eu);
      } else if (u + (int)gridDim.x < nunits) {
        issue_unit(u + gridDim.x, buf ^ 1, E + (size_t)((ju + 1) & 1) * e2w);
      }

      if (g < nd) {
        const uint32_t* t = tab + g * SCp;
        const uint32_t* Sl = smem2 + jbase + lane;
        int ss = 0;
#pragma unroll 2
        for (; ss + 1 < ns; ss += 2) {
          const uint2 tt = *reinterpret_cast<const uint2*>(t + ss);
          const uint32_t* r0 = Sl + tt.x;
          const uint32_t* r1 = Sl + tt.y;
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            if constexpr (HALF) {
              const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(r0 + 32 * v));
              const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(r1 + 32 * v));
              fl[v] += f0.x + f1.x;
              fh[v] += f0.y + f1.y;
            } else {
              const uint32_t w0 = r0[32 * v], w1 = r1[32 * v];
              aw[v] += w0 + w1;
              madd_hi16(ah[v], w0);
              madd_hi16(ah[v], w1);
            }
          }
        }
        if (ss < ns) {
          const uint32_t* r0 = Sl + t[ss];
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            if constexpr (HALF) {
              const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(r0 + 32 * v));
              fl[v] += f0.x;
              fh[v] += f0.y;
            } else {
              const uint32_t w0 = r0[32 * v];
              aw[v] += w0;
              madd_hi16(ah[v], w0);
            }
          }
        }
      }
    }
    // the unit's sums are complete: store the series and the tile's exact sums
    long long s1 = 0;
    unsigned long long s2 = 0;
    if (g < nd) {
      const int d = dfirst + g;
      int32_t* drow = a.D + (size_t)d * a.Dp;
      const int O = HALF ? a.hoff[a.nsub] : 0;   // the offsets taken out in stage 1, added back
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const int64_t ta = t0 + 2 * (jbase + lane + 32 * v);
        uint32_t lo, hi;
        if constexpr (HALF) {
          // the halves hold integers and their FP32 sums stay below 2^24: exact
          lo = (uint32_t)((int)fl[v] + O);
          hi = (uint32_t)((int)fh[v] + O);
        } else {
          lo = aw[v] - (ah[v] << 16);
          hi = ah[v];
        }
        if (ta + 1 < a.Td && (a.Dp & 1) == 0) {
          *reinterpret_cast<int2*>(drow + ta) = make_int2((int32_t)lo, (int32_t)hi);
        } else {
          if (ta < a.Td) drow[ta] = (int32_t)lo;
          if (ta + 1 < a.Td) drow[ta + 1] = (int32_t)hi;
        }
        if (ta < a.T) { s1 += lo; s2 += (unsigned long long)lo * lo; }
        if (ta + 1 < a.T) { s1 += hi; s2 += (unsigned long long)hi * hi; }
      }
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      aw[v] = ah[v] = 0u;
      fl[v] = fh[v] = 0.f;
    }
    warp_sum_stats(s1, s2);
    if (SPLIT == 1) {
      if (g < nd && lane == 0) a.part[(size_t)(dfirst + g) * a.ntile2 + tile] = make_longlong2(s1, (long long)s2);
    } else {
      // combine the parts of each fine DM in a fixed order (deterministic sums)
      if (lane == 0) { st1[warp] = s1; st2[warp] = s2; }
      __syncthreads();
      if (part_i == 0 && g < nd && lane == 0) {
        long long x = 0;
        unsigned long long y = 0;
        for (int i = 0; i < SPLIT; ++i) { x += st1[warp + i]; y += st2[warp + i]; }
        a.part[(size_t)(dfirst + g) * a.ntile2 + tile] = make_longlong2(x, (long long)y);
      }
    }
  }
}

// Stage 2 as a pipeline without block-wide barriers (16-bit intermediates,
// groups of up to 16 fine DMs). Warps [0, NC) are consumers: warp w sums
// fine DM kG + w / SPLIT over words (w % SPLIT) * 512 / SPLIT .. of a unit's
// tile of 512 words (1024 outputs), VW words per lane. Then one issuing warp
// and kPipeProc processing warps. A block walks the chunks of its units (unit
// u = blockIdx.x + i * gridDim.x; a chunk = up to SC sub-bands) in order
// through kPipeStages shared-memory stages; for chunk c in stage c % kPipeStages:
//   * the issuing warp waits until every consumer has left the stage
//     (mbarrier `empty`), announces the bytes and bulk-copies (TMA) the
//     chunk's uint16 rows into the stage's even slots, one row per lane, and
//     the chunk's offset table (precomputed with the plan: per fine DM and
//     sub-band the element offset of its pairs from the staged row start,
//     then the rows' start offsets) into the stage's table; both complete the
//     mbarrier `full`. It runs up to kPipeStages chunks ahead;
//   * the processing warps wait for `full`, write the odd copy (pairs re-formed
//     one element later, as in k_stage2_u16) and arrive on `ready`;
//   * consumers wait for `ready`, sum (an odd offset reads the odd copy), and
//     arrive on `empty`.
// The copies, the odd copies and the sums of different chunks thus overlap,
// and no thread waits for the whole block. After a unit's last chunk each
// consumer warp stores its slice of the series and its exact sums to
// part[d][tile * SPLIT + (w % SPLIT)]. Every wait is bounded; a wait that
// gives up raises a block-wide abort flag that every other wait sees, the
// issuing warp waits (at the full limit) for the copies it has in flight, and
// the block returns.
constexpr int kPipeStages = kPipeStages2;
constexpr int kPipeProc = kPipeProd2 - 1;   // processing warps (the other producer warp issues)

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(done)
               : "r"(smem_addr(bar)), "r"(parity)
               : "memory");
  return done != 0u;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait that also gives up as soon as another thread of the block has
// raised the abort flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, uint32_t polls,
                                                   const volatile int* abort) {
  for (uint32_t i = 0; i < polls; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
  }
  return false;
}

// The walk of one role over the block's chunks: unit, chunk within the unit,
// tile, which member's arguments apply, and the few of them every chunk uses
// (read once per unit: a batched launch finds them in constant memory at a
// run-time index, which would put a load in every chunk's path); the rest
// are read from the source when used.
// The fields of a beam's arguments that the pipelined stage 2 reads for
// every chunk.
struct PipeHot {
  int G, SWW, ndm, SC, nsub;
  uint32_t polls;
  int64_t Pp;
  const void* P;
  const int32_t* tab2;
  double* run;   // where a wait that gives up is recorded
};

template <typename Src>
struct PipeCursor {
  MemberCursor mc;
  int u, ch, nchunk, k, tile, ns, s0, SC, nsub, beam;
  int64_t t0;
  struct NoHot {};
  // batched sources: the member's fields every chunk uses, read once per unit
  std::conditional_t<Src::kBatch, PipeHot, NoHot> hc;
  // the fields every chunk uses: the kernel parameters for one beam, the
  // per-unit copy in a batch
  __device__ __forceinline__ auto hot(const Src& src) const {
    if constexpr (Src::kBatch) return hc; else return src.get(0);
  }
  __device__ __forceinline__ BeamArgs args(const Src& src) const { return src.get(beam); }
  __device__ __forceinline__ void load(const Src& src, const int32_t* __restrict__ uoff,
                                       const int32_t* __restrict__ umem, int nmem) {
    int lu;
    if constexpr (Src::kBatch) {
      mc.seek(uoff, umem, nmem, u);
      lu = u - mc.lo;
      beam = mc.beam;
    } else {
      lu = u;
      beam = 0;
    }
    const BeamArgs a = src.get(beam);
    SC = a.SC;
    nsub = a.nsub;
    if constexpr (Src::kBatch) hc = PipeHot{a.G, a.SWW, a.ndm, a.SC, a.nsub, a.polls, a.Pp, a.P, a.tab2, a.run};
    nchunk = (nsub + SC - 1) / SC;
    k = lu / a.ntile2;
    tile = lu - k * a.ntile2;
    t0 = (int64_t)tile * 1024;
    ch = 0;
    s0 = 0;
    ns = min(SC, nsub);
  }
  // first chunk of unit u0; false when the block has no unit
  __device__ __forceinline__ bool start(const Src& src, const int32_t* uoff, const int32_t* umem, int nmem,
                                        int nunits) {
    u = blockIdx.x;
    if (u >= nunits) return false;
    load(src, uoff, umem, nmem);
    return true;
  }
  // the next chunk; false past the block's last one
  __device__ __forceinline__ bool next(const Src& src, const int32_t* uoff, const int32_t* umem, int nmem,
                                       int nunits) {
    if (++ch < nchunk) {
      s0 = ch * SC;
      ns = min(SC, nsub - s0);
      return true;
    }
    u += gridDim.x;
    if (u >= nunits) return false;
    load(src, uoff, umem, nmem);
    return true;
  }
};

template <int VW, typename Src, bool HALF = false>
__global__ void __launch_bounds__(VW == 16 ? 704 : 1024, 1)
k_stage2_pipe(const Src src, const int32_t* __restrict__ uoff, const int32_t* __restrict__ umem, int nmem,
              int nunits, int slot, int tabw) {
  extern __shared__ __align__(16) uint32_t smp[];
  pdl_wait();
  pdl_trigger();
  constexpr int SPLIT = 16 / VW;                         // consumer warps per fine DM
  __shared__ __align__(8) uint64_t full[kPipeStages], ready[kPipeStages], empty[kPipeStages];
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NC = (int)(blockDim.x >> 5) - 1 - kPipeProc;   // consumer warps
  const int stage_words = 2 * slot + tabw;                 // even slots, odd slots, offset table
  if ((int)blockIdx.x >= nunits) return;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kPipeStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&ready[i], kPipeProc * 32);
      mbar_init(&empty[i], NC * 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();   // barriers initialised: the only block-wide barrier
  volatile int* abort = &abort_flag;
  // a wait that gave up: the first thread to see it raises the flag and records it
  auto give_up = [&](const auto& a) {
    if (atomicExch(&abort_flag, 1) == 0) record_give_up(a);
  };

  if (warp == NC) {
    // --------------------------------------------------------- the issuing warp
    PipeCursor<Src> ic;
    bool more = ic.start(src, uoff, umem, nmem, nunits);
    int64_t q = 0;   // chunks issued
    while (more) {
      const auto a = ic.hot(src);
      const int bq = (int)(q % kPipeStages);
      // the stage's previous chunk: every consumer has left it
      if (q >= kPipeStages &&
          !mbar_wait_or_abort(&empty[bq], (uint32_t)((q / kPipeStages - 1) & 1), a.polls, abort)) {
        give_up(a);
        break;
      }
      const int SCq = (a.SC + 3) & ~3;
      const int32_t* tabk = a.tab2 + ((size_t)ic.k * ic.nchunk + ic.ch) * (size_t)(a.G + 1) * SCq;
      uint32_t* ev = smp + (size_t)bq * stage_words;
      if (lane == 0) mbar_expect_tx(&full[bq], ((uint32_t)ic.ns * (uint32_t)a.SWW + (uint32_t)(a.G + 1) * SCq) * 4u);
      __syncwarp();
      fence_proxy_async();
      const uint16_t* P = static_cast<const uint16_t*>(a.P);
      for (int ss = lane; ss < ic.ns; ss += 32) {   // one row per lane: its start from the table's last row
        const int s = ic.s0 + ss;
        const int64_t b = ic.t0 + __ldg(tabk + (size_t)a.G * SCq + ss);
        bulk_g2s(ev + (size_t)ss * a.SWW, P + ((size_t)ic.k * a.nsub + s) * a.Pp + b, (uint32_t)a.SWW * 4u,
                 &full[bq]);
      }
      if (lane == 0) bulk_g2s(ev + 2 * (size_t)slot, tabk, (uint32_t)(a.G + 1) * SCq * 4u, &full[bq]);
      ++q;
      more = ic.next(src, uoff, umem, nmem, nunits);
    }
    if (lane == 0) {
      // copies still in flight complete before the block's shared memory is released
      for (int64_t r = q > kPipeStages ? q - kPipeStages : 0; r < q; ++r)
        mbar_wait(&full[(int)(r % kPipeStages)], (uint32_t)((r / kPipeStages) & 1), kMbarPolls);
    }
    return;
  }

  if (warp > NC) {
    // ---------------------------------------------------- the processing warps
    const int pw = warp - NC - 1;
    PipeCursor<Src> pc;
    bool more = pc.start(src, uoff, umem, nmem, nunits);
    for (int64_t p = 0; more; ++p) {
      const auto a = pc.hot(src);
      const int bp = (int)(p % kPipeStages);
      if (!mbar_wait_or_abort(&full[bp], (uint32_t)((p / kPipeStages) & 1), a.polls, abort)) {
        give_up(a);
        return;
      }
      // odd copy: od[ss][i] = (P[2i + 1], P[2i + 2]) relative to the staged row start
      const uint32_t* ev = smp + (size_t)bp * stage_words;
      uint32_t* od = smp + (size_t)bp * stage_words + slot;
      // (four 16-byte groups per lane at a time, their loads issued before their stores)
      for (int ss = pw; ss < pc.ns; ss += kPipeProc) {
        const uint32_t* r = ev + (size_t)ss * a.SWW;
        uint32_t* o = od + (size_t)ss * a.SWW;
        for (int j0 = 4 * lane; j0 < a.SWW - 4; j0 += 512) {
          uint4 x[4];
          uint32_t y[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int j = j0 + 128 * i;
            if (j < a.SWW - 4) {
              x[i] = *reinterpret_cast<const uint4*>(r + j);
              y[i] = r[j + 4];
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int j = j0 + 128 * i;
            if (j < a.SWW - 4)
              *reinterpret_cast<uint4*>(o + j) =
                  make_uint4(__funnelshift_r(x[i].x, x[i].y, 16), __funnelshift_r(x[i].y, x[i].z, 16),
                             __funnelshift_r(x[i].z, x[i].w, 16), __funnelshift_r(x[i].w, y[i], 16));
          }
        }
      }
      mbar_arrive(&ready[bp]);
      more = pc.next(src, uoff, umem, nmem, nunits);
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int g = warp / SPLIT, part_i = warp - g * SPLIT;   // fine DM of the group, part of the tile
  const int jbase = part_i * (512 / SPLIT);
  uint32_t aw[VW], ah[VW];   // uint16 pairs: sum of words, sum of high lanes
  float fl[VW], fh[VW];      // half pairs: FP32 sums of the low and high halves
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    aw[v] = ah[v] = 0u;
    fl[v] = fh[v] = 0.f;
  }
  PipeCursor<Src> cc;
  cc.start(src, uoff, umem, nmem, nunits);
  for (int64_t p = 0;; ++p) {
    const auto a = cc.hot(src);
    const int bp = (int)(p % kPipeStages);
    if (!mbar_wait_or_abort(&ready[bp], (uint32_t)((p / kPipeStages) & 1), a.polls, abort)) {
      give_up(a);
      return;
    }
    const int dfirst = cc.k * a.G;
    const int nd = min(a.G, a.ndm - dfirst);
    if (g < nd) {
      const int SCq = (a.SC + 3) & ~3;
      const uint32_t* ev = smp + (size_t)bp * stage_words + jbase + lane;   // this lane's first word, even slots
      const uint32_t* od = ev + slot;                                         // ... odd slots
      const int32_t* t = reinterpret_cast<const int32_t*>(smp + (size_t)bp * stage_words + 2 * (size_t)slot) + g * SCq;
      const int ns = cc.ns, sww = a.SWW;
      int ss = 0;
#pragma unroll 2
      for (; ss + 1 < ns; ss += 2) {
        const int2 tt = *reinterpret_cast<const int2*>(t + ss);
        const uint32_t* r0 = ((tt.x & 1) ? od : ev) + ss * sww + (tt.x >> 1);
        const uint32_t* r1 = ((tt.y & 1) ? od : ev) + (ss + 1) * sww + (tt.y >> 1);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          if constexpr (HALF) {
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(r0 + 32 * v));
            const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(r1 + 32 * v));
            fl[v] += f0.x + f1.x;
            fh[v] += f0.y + f1.y;
          } else {
            const uint32_t w0 = r0[32 * v], w1 = r1[32 * v];
            aw[v] += w0 + w1;
            madd_hi16(ah[v], w0);
            madd_hi16(ah[v], w1);
          }
        }
      }
      if (ss < ns) {
        const int o = t[ss];
        const uint32_t* r0 = ((o & 1) ? od : ev) + ss * sww + (o >> 1);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          if constexpr (HALF) {
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(r0 + 32 * v));
            fl[v] += f0.x;
            fh[v] += f0.y;
          } else {
            const uint32_t w0 = r0[32 * v];
            aw[v] += w0;
            madd_hi16(ah[v], w0);
          }
        }
      }
    }
    mbar_arrive(&empty[bp]);   // this thread is done with the stage
    if (cc.ch + 1 == cc.nchunk) {
      // the unit's sums are complete: this warp's slice of the series and its
      // exact sums (a beam's arguments: the chunk's own for one beam, the
      // member's in a batch)
      auto finish = [&](const BeamArgs& e) {
        long long s1 = 0;
        unsigned long long s2 = 0;
        if (g < nd) {
          const int d = dfirst + g;
          int32_t* drow = e.D + (size_t)d * e.Dp;
          const int O = HALF ? e.hoff[e.nsub] : 0;   // the offsets taken out in stage 1, added back
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const int64_t ta = cc.t0 + 2 * (jbase + lane + 32 * v);
            uint32_t lo, hi;
            if constexpr (HALF) {
              // the halves hold integers and their FP32 sums stay below 2^24: exact
              lo = (uint32_t)((int)fl[v] + O);
              hi = (uint32_t)((int)fh[v] + O);
            } else {
              lo = aw[v] - (ah[v] << 16);
              hi = ah[v];
            }
            if (ta + 1 < e.Td && (e.Dp & 1) == 0) {
              *reinterpret_cast<int2*>(drow + ta) = make_int2((int32_t)lo, (int32_t)hi);
            } else {
              if (ta < e.Td) drow[ta] = (int32_t)lo;
              if (ta + 1 < e.Td) drow[ta + 1] = (int32_t)hi;
            }
            if (ta < e.T) { s1 += lo; s2 += (unsigned long long)lo * lo; }
            if (ta + 1 < e.T) { s1 += hi; s2 += (unsigned long long)hi * hi; }
          }
        }
        warp_sum_stats(s1, s2);
        if (g < nd && lane == 0)
          e.part[((size_t)(dfirst + g) * e.ntile2 + cc.tile) * SPLIT + part_i] = make_longlong2(s1, (long long)s2);
      };
      if constexpr (Src::kBatch) finish(cc.args(src)); else finish(a);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        aw[v] = ah[v] = 0u;
        fl[v] = fh[v] = 0.f;
      }
    }
    if (!cc.next(src, uoff, umem, nmem, nunits)) break;
  }
}

// Stage 2 from int32 intermediates (plain layout, one output per load); one
// block per (tile of 2 NW outputs, coarse group), sub-band chunks in turn.
template <int NW>
__global__ void __launch_bounds__(kStage2MaxGroup * 32)
k_stage2_i32(const int32_t* __restrict__ P, int64_t Pp, const int32_t* __restrict__ e2, int ndm, int nsub,
             int G, int SC, int SW, int32_t* __restrict__ D, int64_t Dp, int64_t Td, int64_t T,
             longlong2* __restrict__ part, int ntile) {
  extern __shared__ __align__(16) uint32_t smem3[];
  pdl_wait();
  pdl_trigger();
  constexpr int V = 2 * NW / 32;
  const int tile = blockIdx.x, k = blockIdx.y;
  const int64_t t0 = (int64_t)tile * 2 * NW;
  const int dfirst = k * G;
  const int nd = min(G, ndm - dfirst);
  int32_t* S = reinterpret_cast<int32_t*>(smem3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0;
  for (int sb = 0; sb < nsub; sb += SC) {
    const int ns = min(SC, nsub - sb);
    for (int i = threadIdx.x; i < ns * SW; i += blockDim.x) {
      const int ss = i / SW, j = i - ss * SW;
      const int s = sb + ss;
      S[(size_t)ss * SW + j] = __ldg(P + ((size_t)k * nsub + s) * Pp + t0 + e2[(size_t)dfirst * nsub + s] + j);
    }
    __syncthreads();
    if (warp < nd) {
      for (int ss = 0; ss < ns; ++ss) {
        const int s = sb + ss;
        const int o = e2[(size_t)(dfirst + warp) * nsub + s] - e2[(size_t)dfirst * nsub + s];
        const int32_t* rw = S + (size_t)ss * SW + o + lane;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += rw[32 * v];
      }
    }
    __syncthreads();
  }
  if (warp < nd) {
    const int d = dfirst + warp;
    int32_t* drow = D + (size_t)d * Dp;
    long long s1 = 0;
    unsigned long long s2 = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int64_t t = t0 + lane + 32 * v;
      if (t < Td) drow[t] = acc[v];
      if (t < T) { s1 += acc[v]; s2 += (unsigned long long)((long long)acc[v] * acc[v]); }
    }
    warp_sum_stats(s1, s2);
    if (lane == 0) part[(size_t)d * ntile + tile] = make_longlong2(s1, (long long)s2);
  }
}

// ---------------------------------------------------------------------------
// statistics (Eq. 5's sigma: the spread of the series' noise, per DM)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double u128_to_double(unsigned __int128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __dadd_rn(__dmul_rn((double)hi, 18446744073709551616.0), (double)lo);
}

// One warp per fine DM (its lanes sum the tiles' exact sums). mu = S1 / T,
// var = (T S2 - S1^2) / T^2 with an exact 128-bit numerator; the running mode
// updates (mu, var) <- (1 - l) prev + l new. Then, per width W (one lane
// each): hi + lo = W mu (hi integer) and inv = 1 / (sigma sqrt W). The warp of
// a candidate-mode beam's first DM also zeroes the beam's candidate counter
// (the boxcar launch comes after this one).
template <typename Src>
__global__ void k_stats(const Src src, const int32_t* __restrict__ uoff, const int32_t* __restrict__ umem, int nmem,
                        int nunits) {
  pdl_wait();
  pdl_trigger();
  const int gd = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);   // one warp per DM
  const int lane = threadIdx.x & 31;
  if (gd >= nunits) return;
  int d;
  BeamArgs a;
  if constexpr (Src::kBatch) {
    const int j = find_member(uoff, nmem, gd);
    d = gd - uoff[j];
    a = src.get(umem[j]);
  } else {
    d = gd;
    a = src.get(0);
  }
  if (d == 0 && lane == 0 && a.output == TX_OUT_CANDS) *a.ncand = 0ull;   // the boxcar launch comes after this one
  const int64_t T = a.T;
  unsigned long long s1 = 0, s2 = 0;
  const int np = a.ntile2 * a.split2;   // the stage-2 tiles' exact sums (per warp of a fine DM in a pipeline plan)
  for (int i = lane; i < np; i += 32) {
    const longlong2 v = a.part[(size_t)d * np + i];
    s1 += (unsigned long long)v.x;
    s2 += (unsigned long long)v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {   // integer sums: exact in any order
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  double mu = __ddiv_rn((double)s1, (double)T);
  const unsigned __int128 num = (unsigned __int128)(unsigned long long)T * s2 - (unsigned __int128)s1 * s1;
  double var = __ddiv_rn(u128_to_double(num), __dmul_rn((double)T, (double)T));
  if (a.running) {
    if (lane == 0) {
      double* r = a.run + (size_t)d * 2;
      const double lam = a.lam;
      if (r[1] < 0.0) {  // never initialised (reset writes -1)
        r[0] = mu;
        r[1] = var;
      } else {
        mu = __dadd_rn(__dmul_rn(1.0 - lam, r[0]), __dmul_rn(lam, mu));
        var = __dadd_rn(__dmul_rn(1.0 - lam, r[1]), __dmul_rn(lam, var));
        r[0] = mu;
        r[1] = var;
      }
    }
    mu = __shfl_sync(0xffffffffu, mu, 0);
    var = __shfl_sync(0xffffffffu, var, 0);
  }
  const double sigma = sqrt(var);
  const double gamma = a.gamma;
  for (int w = lane; w < a.nw; w += 32) {   // the widths' constants, one lane each
    const double W = (double)a.widths[w];
    const double cw = __dmul_rn(W, mu);
    const double hi = rint(cw);
    SnrConst c;
    c.hi = (int32_t)hi;
    c.lo = (float)__dsub_rn(cw, hi);
    c.inv = sigma > 0.0 ? (float)__ddiv_rn(1.0, __dmul_rn(sigma, sqrt(W))) : 0.f;
    if (sigma > 0.0) {
      // smallest integer window sum whose S/N reaches gamma
      const double t = ceil(__dadd_rn(cw, __dmul_rn(gamma, __dmul_rn(sigma, sqrt(W)))));
      c.thr = t > 2147483647.0 ? INT32_MAX : t < -2147483647.0 ? -INT32_MAX : (int32_t)t;
    } else {
      c.thr = gamma <= 0.0 ? -INT32_MAX : INT32_MAX;  // S/N is 0 everywhere
    }
    a.cst[(size_t)d * a.nw + w] = c;
  }
}

// ---------------------------------------------------------------------------
// boxcar matched filter (Eq. 5 via prefix sums, Sec. 2.4) and outputs (Sec. 2.5)
// ---------------------------------------------------------------------------
// Persistent blocks walk contiguous runs of units (fine DM d, tile of
// box_tile outputs, a multiple of kBoxTile chosen by the plan; in a batch, the
// units of all member beams in turn); each
// unit's series (with its W_max - 1 look-ahead) is copied into shared memory
// by one bulk (TMA) copy while the previous unit is being filtered, then turned in
// place into the prefix sum P (P[0] = 0), and each output t takes
// B_W = P[t + W] - P[t] for every width.
//   CUBE / PLANE: S/N for every width (float), best width for the plane.
//   CANDS: a point is a candidate when B_W >= thr_W for some width, an exact
//   integer form of S/N >= gamma; float S/N and the best width are computed
//   for those points only.
// NWT > 0: exactly NWT widths, per-width constants in registers.
// NWT = 0: any count up to kMaxWidths, constants in shared memory.
// The two shared buffers are sized for tileL and wmaxL (the largest box_tile and
// W_max of the launch). A batched launch keeps three blocks per SM (up to 80
// registers a thread; its arguments are loaded from constant memory at a run-
// time index): measured faster there, while the single-beam kernel at 64
// registers was faster on blocks with many candidates.
template <int NWT, int MODE, typename Src>
__global__ void __launch_bounds__(kBoxThreads, Src::kBatch || NWT > 12 ? 3 : 4)
k_boxcar(const Src src, const int32_t* __restrict__ uoff, const int32_t* __restrict__ umem, int nmem, int nunits,
         int tileL, int wmaxL) {
  constexpr int NR = NWT > 0 ? NWT : 1;
  extern __shared__ __align__(16) uint32_t smb[];
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t wsum[kBoxThreads / 32];
  __shared__ int32_t sW[kMaxWidths];
  __shared__ SnrConst sC[kMaxWidths];
  __shared__ __align__(8) uint64_t barb[2];  // completion of the bulk copy into series buffer 0 / 1
  uint32_t bph = 0u;   // bit b: the phase to wait for on barb[b]
  const int bufw = (tileL + wmaxL + 8 + 3) & ~3;  // words per buffer: 4 pad + series + chunk rounding
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int u_begin = (int)((int64_t)nunits * blockIdx.x / gridDim.x);
  const int u_end = (int)((int64_t)nunits * (blockIdx.x + 1) / gridDim.x);

  // In a batch, the unit in buffer b belongs to the member whose arguments
  // sit at index ubx[b] and whose first unit is ubx[2 + b]; thread 0 finds it
  // when it issues the unit's copy, walking a cursor (ubx[4..6]: member, its
  // first and end unit) forward. No member state stays in registers.
  __shared__ int32_t ubx[Src::kBatch ? 7 : 1];
  // thread 0: one bulk copy of unit u's series window into buffer buf (16-byte aligned both sides)
  auto issue = [&](int u, int buf) {
    if (threadIdx.x != 0) return;
    int b = 0, lu = u;
    if constexpr (Src::kBatch) {
      int j = ubx[4], lo = ubx[5], hi = ubx[6];
      if (j < 0 || u >= hi) {
        j = j < 0 ? find_member(uoff, nmem, u) : j;
        while (u >= __ldg(uoff + j + 1)) ++j;
        lo = __ldg(uoff + j);
        hi = __ldg(uoff + j + 1);
        ubx[4] = j;
        ubx[5] = lo;
        ubx[6] = hi;
      }
      b = __ldg(umem + j);
      lu = u - lo;
      ubx[buf] = b;
      ubx[2 + buf] = lo;
    }
    const BeamArgs a = src.get(b);
    const int d = lu / a.ntile3, tile = lu - d * a.ntile3;
    const int64_t t0 = (int64_t)tile * a.box_tile;
    const int n = (int)min((int64_t)a.box_tile, a.T - t0);
    const int nq = (n + a.wmax - 1 + 3) >> 2;  // 16-byte chunks of the series window
    fence_proxy_async();
    mbar_expect_tx(&barb[buf], (uint32_t)nq * 16u);
    bulk_g2s(smb + (size_t)buf * bufw + 4, a.D + (size_t)d * a.Dp + t0, (uint32_t)nq * 16u, &barb[buf]);
  };

  int32_t Wr[NR], thr[NR];
  int cur_d = -1, cur_j = -1;
  if (u_begin >= u_end) return;
  if (threadIdx.x == 0) {
    mbar_init(&barb[0], 1);
    mbar_init(&barb[1], 1);
    fence_mbar_init();
    if constexpr (Src::kBatch) ubx[4] = -1;
  }
  __syncthreads();
  issue(u_begin, 0);
  if constexpr (Src::kBatch) __syncthreads();   // the first unit's member
  for (int u = u_begin, it = 0; u < u_end; ++u, ++it) {
    const int buf = it & 1;
    int lu, j;
    BeamArgs a;
    if constexpr (Src::kBatch) {
      j = ubx[buf];
      lu = u - ubx[2 + buf];
      a = src.get(j);
    } else {
      j = 0;
      lu = u;
      a = src.get(0);
    }
    const int nw = NWT > 0 ? NWT : a.nw;
    const int d = lu / a.ntile3, tile = lu - d * a.ntile3;
    const int64_t T = a.T;
    const int64_t t0 = (int64_t)tile * a.box_tile;
    const int n = (int)min((int64_t)a.box_tile, T - t0);
    const int N = n + a.wmax - 1;
    const SnrConst* cst = a.cst + (size_t)d * nw;
    // series D[j] at C[j] (16-byte aligned); the scan leaves C[k] = D[0] + ... + D[k - 1]
    uint32_t* C = smb + (size_t)buf * bufw + 4;
    const bool fresh = d != cur_d || j != cur_j;
    if (NWT > 0 && fresh) {
#pragma unroll
      for (int w = 0; w < NR; ++w) {
        Wr[w] = __ldg(a.widths + w);
        thr[w] = cst[w].thr;
      }
    }
    const uint32_t ph = (bph >> buf) & 1u;
    const bool landed = mbar_wait(&barb[buf], ph, a.polls);
    bph ^= 1u << buf;
    // this unit's series landed; the previous unit is done with sW/sC and the other buffer
    if (__syncthreads_or(!landed)) {
      // a copy never completed: record it, give the copy in flight a last wait at the full limit, give up
      if (threadIdx.x == 0) {
        record_give_up(a);
        mbar_wait(&barb[buf], ph, kMbarPolls);
      }
      return;
    }
    if (NWT == 0 && fresh && threadIdx.x < nw) {
      sW[threadIdx.x] = a.widths[threadIdx.x];
      sC[threadIdx.x] = cst[threadIdx.x];
    }
    cur_d = d;
    cur_j = j;
    if (u + 1 < u_end) issue(u + 1, buf ^ 1);
    // exclusive scan of C[0..N] in place (uint32, wrap-around is harmless:
    // window sums < 2^31); D[N] (possibly not loaded) only enters sums past C[N]
    const int E = (N + 1 + blockDim.x - 1) / blockDim.x;
    const int beg = threadIdx.x * E, end = min(beg + E, N + 1);
    uint32_t local = 0;
    for (int i = beg; i < end; ++i) local += C[i];
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t pre = x - local;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    for (int i = beg; i < end; ++i) {
      const uint32_t v = C[i];
      C[i] = pre;
      pre += v;
    }
    __syncthreads();

    // candidates of a full run of quads, widths 1, 2 and multiples of 4: each
    // thread tests the four outputs 4q .. 4q + 3 of quads q = tid + 256 r
    // (r < QR) from aligned 16-byte loads of Cs (its own quad and the next for
    // widths 1, 2 and 4, one more per wider width); hits go to a bit mask and
    // the rare hits are written after, once per warp that has any
    auto vec_cands = [&](const uint32_t* Cs, int64_t ts, auto qr) {
      constexpr int QR = decltype(qr)::value;
      const uint4* C4 = reinterpret_cast<const uint4*>(Cs);
      uint32_t mask = 0;
#pragma unroll
      for (int r = 0; r < QR; ++r) {
        const int q = threadIdx.x + r * kBoxThreads;
        const uint4 cl = C4[q], nx = C4[q + 1];
        int32_t m0 = (int32_t)(cl.y - cl.x) - thr[0], m1 = (int32_t)(cl.z - cl.y) - thr[0];
        int32_t m2 = (int32_t)(cl.w - cl.z) - thr[0], m3 = (int32_t)(nx.x - cl.w) - thr[0];
        m0 = max(m0, (int32_t)(cl.z - cl.x) - thr[1]);
        m1 = max(m1, (int32_t)(cl.w - cl.y) - thr[1]);
        m2 = max(m2, (int32_t)(nx.x - cl.z) - thr[1]);
        m3 = max(m3, (int32_t)(nx.y - cl.w) - thr[1]);
#pragma unroll
        for (int w = 2; w < NR; ++w) {
          // width 4 (the usual third) is the next quad, already loaded
          const uint4 cw = (w == 2 && Wr[2] == 4) ? nx : C4[q + (Wr[w] >> 2)];
          m0 = max(m0, (int32_t)(cw.x - cl.x) - thr[w]);
          m1 = max(m1, (int32_t)(cw.y - cl.y) - thr[w]);
          m2 = max(m2, (int32_t)(cw.z - cl.z) - thr[w]);
          m3 = max(m3, (int32_t)(cw.w - cl.w) - thr[w]);
        }
        mask |= ((uint32_t)(m0 >= 0) | ((uint32_t)(m1 >= 0) << 1) | ((uint32_t)(m2 >= 0) << 2) |
                 ((uint32_t)(m3 >= 0) << 3)) << (4 * r);
      }
      // only the bit positions where some lane of the warp has a hit
      for (uint32_t rows = __reduce_or_sync(0xffffffffu, mask); rows != 0u; rows &= rows - 1u) {
        {
          const int r = __ffs(rows) - 1;
          const int i = 4 * (threadIdx.x + (r >> 2) * kBoxThreads) + (r & 3);
          const bool hit = (mask >> r) & 1u;
          const unsigned hits = __ballot_sync(0xffffffffu, hit);
          if (!hits) continue;
          float best = -INFINITY;
          int bw = 0;
          if (hit) {
            const uint32_t* Ci = Cs + i;
            const uint32_t cl = Ci[0];
            #pragma unroll   // static indices keep Wr in registers
            for (int w = 0; w < NR; ++w) {
              const SnrConst c = cst[w];
              const float sv = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
              if (sv > best) { best = sv; bw = w; }
            }
          }
          const int leader = __ffs(hits) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(a.ncand, (unsigned long long)__popc(hits));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (hit) {
            const unsigned long long idx = base + __popc(hits & ((1u << lane) - 1u));
            if (idx < (unsigned long long)a.max_cands) {
              tx_cand rec;
              rec.dm_index = d;
              rec.t = (int32_t)(ts + i);
              rec.w_index = bw;
              rec.snr = best;
              a.cands[idx] = rec;
            }
          }
        }
      }
    };
    if constexpr (NWT > 0 && MODE == TX_OUT_CANDS) {
      if (n == a.box_tile && a.box_vec) {   // a full unit in one pass
        if (n == 4 * kBoxTile) vec_cands(C, t0, std::integral_constant<int, 4 * kBoxTile / 4 / kBoxThreads>{});
        else if (n == 2 * kBoxTile) vec_cands(C, t0, std::integral_constant<int, 2 * kBoxTile / 4 / kBoxThreads>{});
        else vec_cands(C, t0, std::integral_constant<int, kBoxTile / 4 / kBoxThreads>{});
        continue;
      }
    }
    // the unit in sub-tiles of kBoxTile outputs: full ones take the unrolled tests
    for (int s0 = 0; s0 < n; s0 += kBoxTile) {
      const int ns = min(kBoxTile, n - s0);
      const uint32_t* Cs = C + s0;
      const int64_t ts = t0 + s0;
      if constexpr (NWT > 0 && MODE == TX_OUT_CANDS) {
        if (ns == kBoxTile && a.box_vec) {
          vec_cands(Cs, ts, std::integral_constant<int, kBoxTile / 4 / kBoxThreads>{});
          continue;
        }
        if (ns == kBoxTile) {
          // full tile, candidates: each thread tests outputs tid + 256 r (r < 8)
          // and keeps its hits in a bit mask; the rare hits are written after,
          // once per warp that has any
          constexpr int RR = kBoxTile / kBoxThreads;
          uint32_t mask = 0;
#pragma unroll
          for (int r = 0; r < RR; ++r) {
            const uint32_t* Ci = Cs + threadIdx.x + r * kBoxThreads;
            const uint32_t cl = Ci[0];
            int32_t mx = INT32_MIN;
#pragma unroll
            for (int w = 0; w < NR; ++w) mx = max(mx, (int32_t)(Ci[Wr[w]] - cl) - thr[w]);
            mask |= (uint32_t)(mx >= 0) << r;
          }
          for (uint32_t rows = __reduce_or_sync(0xffffffffu, mask); rows != 0u; rows &= rows - 1u) {
            {
              const int r = __ffs(rows) - 1;
              const int i = threadIdx.x + r * kBoxThreads;
              const bool hit = (mask >> r) & 1u;
              const unsigned hits = __ballot_sync(0xffffffffu, hit);
              if (!hits) continue;
              float best = -INFINITY;
              int bw = 0;
              if (hit) {
                const uint32_t* Ci = Cs + i;
                const uint32_t cl = Ci[0];
                #pragma unroll   // static indices keep Wr in registers
                for (int w = 0; w < NR; ++w) {
                  const SnrConst c = cst[w];
                  const float sv = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
                  if (sv > best) { best = sv; bw = w; }
                }
              }
              const int leader = __ffs(hits) - 1;
              unsigned long long base = 0;
              if (lane == leader) base = atomicAdd(a.ncand, (unsigned long long)__popc(hits));
              base = __shfl_sync(0xffffffffu, base, leader);
              if (hit) {
                const unsigned long long idx = base + __popc(hits & ((1u << lane) - 1u));
                if (idx < (unsigned long long)a.max_cands) {
                  tx_cand rec;
                  rec.dm_index = d;
                  rec.t = (int32_t)(ts + i);
                  rec.w_index = bw;
                  rec.snr = best;
                  a.cands[idx] = rec;
                }
              }
            }
          }
          continue;
        }
      }

      for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const uint32_t* Ci = Cs + i;
        const uint32_t cl = Ci[0];
        float best = -INFINITY;
        int bw = 0;
        bool hit = false;
        if (NWT > 0) {
          if (MODE == TX_OUT_CANDS) {
            int32_t mx = INT32_MIN;
#pragma unroll
            for (int w = 0; w < NR; ++w) mx = max(mx, (int32_t)(Ci[Wr[w]] - cl) - thr[w]);
            hit = mx >= 0;
            if (hit) {  // rare: float S/N and the best width of a candidate
              #pragma unroll   // static indices keep Wr in registers
              for (int w = 0; w < NR; ++w) {
                const SnrConst c = cst[w];
                const float sv = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
                if (sv > best) { best = sv; bw = w; }
              }
            }
          } else {
            float sv[NR];
#pragma unroll
            for (int w = 0; w < NR; ++w) {
              const SnrConst c = cst[w];
              sv[w] = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
            }
            if (MODE == TX_OUT_CUBE) {
#pragma unroll
              for (int w = 0; w < NR; ++w) a.outf[((size_t)d * nw + w) * T + ts + i] = sv[w];
            } else {
#pragma unroll
              for (int w = 0; w < NR; ++w) best = fmaxf(best, sv[w]);
              bw = NR - 1;
#pragma unroll
              for (int w = NR - 1; w >= 0; --w)
                if (sv[w] == best) bw = w;
            }
          }
        } else {
          for (int w = 0; w < nw; ++w) {
            const int32_t B = (int32_t)(Ci[sW[w]] - cl);
            const float snr = ((float)(B - sC[w].hi) - sC[w].lo) * sC[w].inv;
            if (MODE == TX_OUT_CUBE) a.outf[((size_t)d * nw + w) * T + ts + i] = snr;
            if (snr > best) { best = snr; bw = w; }
            hit = hit || B >= sC[w].thr;
          }
        }
        if (MODE == TX_OUT_PLANE) {
          a.outf[(size_t)d * T + ts + i] = best;
          a.outw[(size_t)d * T + ts + i] = (uint8_t)bw;
        } else if (MODE == TX_OUT_CANDS) {
          const unsigned act = __activemask();
          const unsigned hits = __ballot_sync(act, hit);
          if (hits) {
            const int leader = __ffs(hits) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.ncand, (unsigned long long)__popc(hits));
            base = __shfl_sync(act, base, leader);
            if (hit) {
              const unsigned long long idx = base + __popc(hits & ((1u << lane) - 1u));
              if (idx < (unsigned long long)a.max_cands) {
                tx_cand r;
                r.dm_index = d;
                r.t = (int32_t)(ts + i);
                r.w_index = bw;
                r.snr = best;
                a.cands[idx] = r;
              }
            }
          }
        }
      }
    }
  }
}

template <typename Src>
using BoxKernel = void (*)(const Src, const int32_t*, const int32_t*, int, int, int, int);

// Exact width counts 1..12 and 16 get their own instantiation; others use
// the generic one (NWT = 0).
template <int MODE, typename Src>
BoxKernel<Src> box_kernel_m(int nw) {
  switch (nw) {
#define TX_BOX(N) \
  case N: return k_boxcar<N, MODE, Src>;
    TX_BOX(1) TX_BOX(2) TX_BOX(3) TX_BOX(4) TX_BOX(5) TX_BOX(6) TX_BOX(7) TX_BOX(8) TX_BOX(9) TX_BOX(10)
    TX_BOX(11) TX_BOX(12) TX_BOX(16)
#undef TX_BOX
    default: return k_boxcar<0, MODE, Src>;
  }
}

template <typename Src>
BoxKernel<Src> box_kernel(int nw, int mode) {
  return mode == TX_OUT_CANDS ? box_kernel_m<TX_OUT_CANDS, Src>(nw)
         : mode == TX_OUT_PLANE ? box_kernel_m<TX_OUT_PLANE, Src>(nw) : box_kernel_m<TX_OUT_CUBE, Src>(nw);
}

// Instantiation class of a width count: the exact-count kernels, or 0 (generic).
inline int box_class(int nw) { return (nw >= 1 && nw <= 12) || nw == 16 ? nw : 0; }

__global__ void k_fill_run(double* run, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) run[2 * i + 1] = -1.0;  // marks "not initialised"
}

// ---------------------------------------------------------------------------
// host helpers shared by the single-beam and batched launchers
// ---------------------------------------------------------------------------
// Launches kernel k with programmatic stream serialization (see pdl_wait):
// the launch and block set-up overlap the tail of the kernel before it.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Raises kernel k's dynamic shared memory limit on the current device to at
// least `bytes`, never lowering it: plans of different shapes share kernels,
// and the limit one plan needs must survive another plan's set-up.
inline cudaError_t raise_smem_limit(const void* k, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> lim;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(dev, k);
  const auto it = lim.find(key);
  const int cur = it == lim.end() ? 48 * 1024 : it->second;  // the default limit
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) lim[key] = bytes;
  return e;
}

// two buffers of (4 pad words + tile + look-ahead, rounded to 16-byte chunks)
inline int box_smem_for(int tile, int wmax) { return 2 * ((tile + wmax + 8 + 3) & ~3) * 4; }

// uint16 stage 2: two even-copy slots, one odd-copy slot, address table
inline int stage2_u16_smem_for(int slot, int sc, int e2w) {
  return (2 * e2w + 3 * slot + kStage2MaxGroup * ((sc + 1) & ~1)) * 4;
}

// Warps per fine DM of the uint16 stage 2 (the plan's tile choice).
inline int stage2_split(const tx_plan* p) { return p->split2; }

inline int stage2_threads(const tx_plan* p) {
  if (p->pipe2) return (p->group * p->split2 + kPipeProd2) * 32;   // consumer warps, then the issuing and processing warps
  return std::min(p->group, kStage2MaxGroup) * 32 * stage2_split(p);
}

// The pipelined stage 2 for `split` consumer warps per fine DM (4, 2 or 1: 4, 8
// or 16 words per lane), half or uint16 intermediates.
template <typename Src>
const void* stage2_pipe_kernel(int split, bool half) {
  switch (split) {
    case 4: return half ? (const void*)k_stage2_pipe<4, Src, true> : (const void*)k_stage2_pipe<4, Src, false>;
    case 2: return half ? (const void*)k_stage2_pipe<8, Src, true> : (const void*)k_stage2_pipe<8, Src, false>;
    default: return half ? (const void*)k_stage2_pipe<16, Src, true> : (const void*)k_stage2_pipe<16, Src, false>;
  }
}

// Launches it over `nunits` (coarse group, tile) units; slot = the largest
// chunk's staged words (sub-bands x words), smem from stage2_pipe_smem.
template <typename Src>
void launch_stage2_pipe(int split, bool half, int grid, int threads, int smem, cudaStream_t st, const Src& src,
                        const int32_t* uoff, const int32_t* umem, int nmem, int nunits, int sc, int slot,
                        bool pdl = false) {
  const int tabw = (kPipeMaxGroup2 + 1) * ((sc + 3) & ~3);
#define TX_P2(VW)                                                                                               \
  do {                                                                                                          \
    auto k = half ? k_stage2_pipe<VW, Src, true> : k_stage2_pipe<VW, Src, false>;                              \
    if (pdl)                                                                                                    \
      launch_pdl(k, grid, threads, smem, st, src, uoff, umem, nmem, nunits, slot, tabw);                        \
    else                                                                                                        \
      k<<<grid, threads, smem, st>>>(src, uoff, umem, nmem, nunits, slot, tabw);                                \
  } while (0)
  switch (split) {
    case 4: TX_P2(4); break;
    case 2: TX_P2(8); break;
    default: TX_P2(16); break;
  }
#undef TX_P2
}

// The arguments of one execute of plan p on beam b: the block lands at ring
// position `head`, buffer time 0 sits at `start` (a compact beam uses its
// borrowed ring instead: head0 and head0 - L); ws is the execute's
// workspace; out / ncand as tx_execute.
inline BeamArgs make_args(const tx_plan* p, const tx_beam* b, const uint8_t* block, void* out, int64_t* ncand,
                          void* ws_ptr, int64_t head, int64_t start) {
  uint8_t* ws = static_cast<uint8_t*>(ws_ptr);
  const bool series = p->output == TX_OUT_SERIES;
  BeamArgs a{};
  a.block = block;
  a.ring = b->ring;
  if (b->compact) {  // a fresh linear window in the workspace: tail, then the block at head0
    a.ring = ws + p->ws_ring;
    head = p->head0;
    start = p->head0 - p->L;
    a.tail = b->tail;
    a.compact = 1;
  }
  a.L = p->L;
  a.tail_pitch = p->tail_pitch;
  a.tail_pad = (int32_t)p->tail_pad;
  a.P = ws + p->ws_P;
  a.D = series ? static_cast<int32_t*>(out) : reinterpret_cast<int32_t*>(ws + p->ws_D);
  a.part = reinterpret_cast<longlong2*>(ws + p->ws_part);
  a.cst = reinterpret_cast<SnrConst*>(ws + p->ws_const);
  a.hoff = reinterpret_cast<int32_t*>(ws + p->ws_hoff);
  a.half = p->interm == TX_INTERM_F16;
  a.box_vec = (int8_t)p->box_vec;
  a.box_tile = p->box_tile;
  a.tab1 = p->dev.tab1;
  a.tab2 = p->dev.tab2;
  a.tab1_phase = p->tab1_phase;
  a.run = b->run;
  a.d1 = p->dev.d1;
  a.abase = p->dev.abase;
  a.e2 = p->dev.e2;
  a.widths = p->dev.widths;
  a.items = p->dev.items1;
  a.outf = static_cast<float*>(out);
  a.outw = p->output == TX_OUT_PLANE ? static_cast<uint8_t*>(out) + (size_t)p->ndm * p->T * 4 : nullptr;
  a.cands = static_cast<tx_cand*>(out);
  a.ncand = reinterpret_cast<unsigned long long*>(ncand);
  a.R = p->R;
  a.head = head;
  a.start = start;
  a.T = p->T;
  a.Pp = p->Pp;
  a.Dp = series ? p->Td : p->Dp;
  a.Td = p->Td;
  a.max_cands = p->max_cands;
  a.lam = p->lambda;
  a.gamma = (double)p->gamma;
  a.nchan = p->nchan;
  a.m = p->m;
  a.nsub = p->nsub;
  a.ndm = p->ndm;
  a.G = p->group;
  a.split2 = p->pipe2 ? p->split2 : 1;
  a.SC = p->nsub_chunk2;
  a.SWW = p->sww2;
  a.ntile2 = p->ntile2;
  a.ntile3 = p->ntile3;
  a.nw = p->nw;
  a.wmax = p->wmax;
  a.layout = p->layout;
  const bool al = ((uintptr_t)block & 15) == 0 && head % 16 == 0;
  a.ingest_vec = p->layout == TX_LAYOUT_TF ? (al && p->nchan % 16 == 0) : (al && p->T % 16 == 0);
  a.running = p->stats == TX_STATS_RUNNING;
  a.output = p->output;
  a.polls = first_wait_polls();
  return a;
}

}  // namespace
