// CUDA side (sm_103a) of the library: ingest, two-stage sub-band
// de-dispersion (Sec. 2.3), block statistics, and the boxcar matched filter
// with its outputs (Sec. 2.4, 2.5); plus the C-ABI entry points that launch
// them.
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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------------------
// ingest (Sec. 2.3 data flow)
// ---------------------------------------------------------------------------
// Channel-major rows: ring[c][dst_off + i] = src[c][src_off + i], i < n.
__global__ void k_ingest_ft(const uint8_t* __restrict__ src, int64_t src_pitch, int64_t src_off, int64_t n,
                            uint8_t* __restrict__ ring, int64_t R, int64_t dst_off, int vec) {
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

// Time-major block rows [t][nchan], t in [t_off, t_off + n) -> ring[c][dst_off + t - t_off],
// through a 64-time x 64-channel byte tile. vec: 16-byte loads and stores
// (nchan, dst_off and the source all 16-byte aligned).
__global__ void __launch_bounds__(256) k_ingest_tf(const uint8_t* __restrict__ src, int64_t t_off, int64_t n,
                                                   int nchan, uint8_t* __restrict__ ring, int64_t R,
                                                   int64_t dst_off, int vec) {
  __shared__ __align__(16) uint8_t tile[64][80];
  const int64_t t0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  {
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    const int64_t t = t0 + r;
    const int c = c0 + 16 * q;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (t < n) {
      const uint8_t* sp = src + (t_off + t) * nchan + c;
      if (vec && c + 16 <= nchan) {
        v = __ldg(reinterpret_cast<const uint4*>(sp));
      } else {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (int i = 0; i < 16; ++i)
          if (c + i < nchan) w[i >> 2] |= (uint32_t)sp[i] << (8 * (i & 3));
        v = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    *reinterpret_cast<uint4*>(&tile[r][16 * q]) = v;
  }
  __syncthreads();
  {
    const int cc = threadIdx.x & 63, pq = threadIdx.x >> 6;
    const int c = c0 + cc;
    if (c < nchan) {
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        w[i] = (uint32_t)tile[16 * pq + 4 * i][cc] | ((uint32_t)tile[16 * pq + 4 * i + 1][cc] << 8) |
               ((uint32_t)tile[16 * pq + 4 * i + 2][cc] << 16) | ((uint32_t)tile[16 * pq + 4 * i + 3][cc] << 24);
      const int64_t t = t0 + 16 * pq;
      uint8_t* dp = ring + (int64_t)c * R + dst_off + t;
      if (vec && t + 16 <= n) {
        *reinterpret_cast<uint4*>(dp) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        for (int i = 0; i < 16; ++i)
          if (t + i < n) dp[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// stage 1 (Sec. 2.3: de-disperse each sub-band on the coarse DM grid)
// ---------------------------------------------------------------------------
// Sums one coarse DM over the sub-band's m channels for VW words per lane,
// starting at word jbase of the tile, and stores the 4 * VW * 32 outputs.
template <int Q, int VW, typename PT>
__device__ __forceinline__ void stage1_sum(const uint32_t* __restrict__ S, const uint32_t* __restrict__ t, int m,
                                           uint32_t one, int lane, int jbase, PT* __restrict__ prow, int rel0,
                                           int64_t Pp) {
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
      const PT v0 = (PT)(lo & 0xFFFFu), v1 = (PT)(ah[v] & 0xFFFFu), v2 = (PT)(lo >> 16), v3 = (PT)(ah[v] >> 16);
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
        if (u < (uint64_t)Pp) prow[u] = (PT)val[q];
      }
    }
  }
}

// Persistent blocks walk the work items (sub-band s, coarse DMs [kb, ke),
// absolute times [tau0, tau0 + 4Q)). For each item the channels' input
// windows (from 16-byte aligned ring positions) are copied with cp.async into
// a raw buffer while the previous item is being summed, then rearranged so
// that shared word S[c][j] holds channel c's samples at raw offsets j + qQ in
// byte q (q = 0..3). For coarse DM k the output word j is
// sum_c S[c][j + a_c + d1[k][c] - d1[kb][c]] (a_c the window's misalignment):
// four outputs per 32-bit load whatever the delays. Sums use the byte-lane
// identity  sum w = sum(lo lanes) + 256 * sum(hi lanes)  (mod 2^32)  with the hi
// lanes (bytes 1, 3) accumulated separately as 16-bit lanes, exact for up to
// 257 channels per sub-band. Warps take (coarse DM, part of the tile) tasks;
// a chunk with few coarse DMs splits each tile between 2, 4 or 8 warps.
template <int Q, typename PT>
__global__ void __launch_bounds__(kStage1Warps * 32, 1)
k_stage1(const uint8_t* __restrict__ ring, int R, int start, const Stage1Item* __restrict__ items,
         int nitems, const int32_t* __restrict__ d1, int nchan, int m, int nsub, const int32_t* __restrict__ abase,
         PT* __restrict__ P, int64_t Pp, uint32_t one) {
  extern __shared__ __align__(16) uint8_t smem1[];
  constexpr int SW = kStage1StagedWords(Q);      // staged words per channel
  constexpr int RB = kStage1RawBytes(Q);         // raw bytes per channel
  constexpr int NCH = RB / 16;
  constexpr int V = Q / 32;
  const int TS = (m + 3) & ~3;                   // offset-table row stride (16-byte aligned quads)
  uint32_t* S = reinterpret_cast<uint32_t*>(smem1);
  uint8_t* raw = smem1 + (size_t)m * SW * 4;
  uint32_t* tab = reinterpret_cast<uint32_t*>(raw + (size_t)m * RB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // physical ring position of channel c's first wanted sample for an item
  auto wstart = [&](const Stage1Item& it, int c) -> int {
    int64_t p = (int64_t)start + it.tau0 + d1[(size_t)it.kb * nchan + it.s * m + c];
    while (p >= R) p -= R;
    return (int)p;
  };
  auto issue = [&](int idx) {
    const Stage1Item it = items[idx];
    for (int c = warp; c < m; c += kStage1Warps) {
      const int pa = wstart(it, c) & ~15;
      const uint8_t* row = ring + (size_t)(it.s * m + c) * R;
      uint8_t* dst = raw + (size_t)c * RB;
      for (int ch = lane; ch < NCH; ch += 32) {
        int q = pa + 16 * ch;  // R is a multiple of 64: a chunk never straddles the wrap
        while (q >= R) q -= R;
        cp_async16(dst + 16 * ch, row + q);
      }
    }
    cp_async_commit();
  };

  int idx = blockIdx.x;
  if (idx < nitems) issue(idx);
  while (idx < nitems) {
    const Stage1Item it = items[idx];
    const int c0 = it.s * m;
    const int nkk = it.ke - it.kb;
    const int32_t* d1kb = d1 + (size_t)it.kb * nchan + c0;
    cp_async_wait_all();
    __syncthreads();
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
    // word offset of S[c][a_c + d1[k][c] - d1[kb][c]] for every (k, c)
    for (int kk = warp; kk < nkk; kk += kStage1Warps) {
      const int32_t* d1k = d1 + (size_t)(it.kb + kk) * nchan + c0;
      for (int c = lane; c < m; c += 32)
        tab[kk * TS + c] = (uint32_t)(c * SW + (wstart(it, c) & 15) + d1k[c] - d1kb[c]);
    }
    __syncthreads();
    const int next = idx + gridDim.x;
    if (next < nitems) issue(next);

    // tasks: (coarse DM, part of the tile); split the tile when coarse DMs are few
    int split = 1;
    while (split < V && nkk * split * 2 <= kStage1Warps) split *= 2;
    for (int task = warp; task < nkk * split; task += kStage1Warps) {
      const int kk = task / split, part = task - kk * split;
      const int k = it.kb + kk;
      const int64_t ab = abase[(size_t)k * nsub + it.s];
      if ((int64_t)it.tau0 + 4 * Q <= ab || (int64_t)it.tau0 >= ab + Pp) continue;
      PT* prow = P + ((size_t)k * nsub + it.s) * Pp;
      const int rel0 = (int)((int64_t)it.tau0 - ab);  // |rel0| < 2^30
      const uint32_t* t = tab + kk * TS;
      if (split == 1) {
        stage1_sum<Q, V, PT>(S, t, m, one, lane, 0, prow, rel0, Pp);
      } else if (split == 2) {
        if constexpr (V >= 2) stage1_sum<Q, V / 2, PT>(S, t, m, one, lane, part * (Q / 2), prow, rel0, Pp);
      } else if (split == 4) {
        if constexpr (V >= 4) stage1_sum<Q, V / 4, PT>(S, t, m, one, lane, part * (Q / 4), prow, rel0, Pp);
      } else {
        if constexpr (V >= 8) stage1_sum<Q, V / 8, PT>(S, t, m, one, lane, part * (Q / 8), prow, rel0, Pp);
      }
    }
    __syncthreads();
    idx = next;
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
// words of the tile. A chunk's uint16 stage-1 rows are copied (cp.async,
// double-buffered) into shared memory as 32-bit words of consecutive pairs
// (even copy) and re-paired one element later (odd copy), so every delay,
// even or odd, is a 32-bit load feeding two outputs. Sums use
//   sum w = sum(lo) + 65536 * sum(hi) (mod 2^32), sum(hi) = sum(w >> 16),
// exact because every stage-2 sum is below 2^32.
template <int NW, int MAXWARPS, int SPLIT>
__global__ void __launch_bounds__(MAXWARPS * 32, 1)
k_stage2_u16(const uint16_t* __restrict__ P, int64_t Pp, const int32_t* __restrict__ e2, int ndm, int nsub,
             int G, int nk, int SC, int SWW, int ntile, int32_t* __restrict__ D, int64_t Dp, int64_t Td, int64_t T,
             longlong2* __restrict__ part, int64_t* __restrict__ part_tmp) {
  extern __shared__ __align__(16) uint32_t smem2[];
  constexpr int VW = NW / 32 / SPLIT;                    // words per lane
  uint32_t* Se = smem2;                                  // [2][SC][SWW]
  uint32_t* So = Se + 2 * (size_t)SC * SWW;              // [SC][SWW]
  uint32_t* tab = So + (size_t)SC * SWW;                 // [kStage2MaxGroup][SC] word offsets from smem2
  __shared__ long long st1[MAXWARPS];
  __shared__ unsigned long long st2[MAXWARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int g = warp / SPLIT, part_i = warp - g * SPLIT;  // fine DM of the group, part of the tile
  const int jbase = part_i * (NW / SPLIT);
  const int nchunk = (nsub + SC - 1) / SC;
  const int nunits = nk * ntile;
  // steps (unit, chunk) of this block: unit = blockIdx.x + r * gridDim.x
  const int my_units = (int)blockIdx.x < nunits ? (nunits - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nsteps = my_units * nchunk;
  const int nq = SWW >> 2;

  auto issue = [&](int step, int buf) {
    const int unit = blockIdx.x + (step / nchunk) * gridDim.x;
    const int ch = step % nchunk;
    const int k = unit / ntile, tile = unit - k * ntile;
    const int64_t t0 = (int64_t)tile * 2 * NW;
    const int s0 = ch * SC, ns = min(SC, nsub - s0);
    uint32_t* dst = Se + (size_t)buf * SC * SWW;
    for (int ss = warp; ss < ns; ss += nwarps) {
      const int s = s0 + ss;
      const int64_t b = (t0 + e2[(size_t)k * G * nsub + s]) & ~(int64_t)7;
      const uint16_t* src = P + ((size_t)k * nsub + s) * Pp + b;
      uint32_t* d = dst + (size_t)ss * SWW;
      for (int q = lane; q < nq; q += 32) cp_async16(d + 4 * q, src + 8 * q);
    }
    cp_async_commit();
  };

  uint32_t aw[VW], ah[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) aw[v] = ah[v] = 0u;
  if (nsteps > 0) issue(0, 0);
  for (int step = 0; step < nsteps; ++step) {
    const int buf = step & 1;
    const int unit = blockIdx.x + (step / nchunk) * gridDim.x;
    const int ch = step % nchunk;
    const int k = unit / ntile, tile = unit - k * ntile;
    const int64_t t0 = (int64_t)tile * 2 * NW;
    const int dfirst = k * G;
    const int nd = min(G, ndm - dfirst);
    const int s0 = ch * SC, ns = min(SC, nsub - s0);
    uint32_t* cur = Se + (size_t)buf * SC * SWW;
    cp_async_wait_all();
    __syncthreads();
    // odd copy: So[ss][i] = (P[2i + 1], P[2i + 2]) relative to the staged base
    for (int ss = warp; ss < ns; ss += nwarps) {
      const uint32_t* r = cur + (size_t)ss * SWW;
      uint32_t* o = So + (size_t)ss * SWW;
      for (int j = 4 * lane; j < SWW - 4; j += 128) {
        const uint4 a = *reinterpret_cast<const uint4*>(r + j);
        const uint32_t b = r[j + 4];
        *reinterpret_cast<uint4*>(o + j) =
            make_uint4(__funnelshift_r(a.x, a.y, 16), __funnelshift_r(a.y, a.z, 16), __funnelshift_r(a.z, a.w, 16),
                       __funnelshift_r(a.w, b, 16));
      }
    }
    for (int gg = warp; gg < nd; gg += nwarps) {
      for (int ss = lane; ss < ns; ss += 32) {
        const int s = s0 + ss;
        const int32_t emin = e2[(size_t)dfirst * nsub + s];
        const int off = e2[(size_t)(dfirst + gg) * nsub + s] - emin + (int)((t0 + emin) & 7);
        const uint32_t* base = (off & 1) ? So : cur;
        tab[gg * SC + ss] = (uint32_t)(base - smem2) + (uint32_t)(ss * SWW + (off >> 1));
      }
    }
    __syncthreads();
    if (step + 1 < nsteps) issue(step + 1, buf ^ 1);

    if (g < nd) {
      const uint32_t* t = tab + g * SC;
      const uint32_t* Sl = smem2 + jbase + lane;
      int ss = 0;
#pragma unroll 2
      for (; ss + 1 < ns; ss += 2) {
        const uint32_t* r0 = Sl + t[ss];
        const uint32_t* r1 = Sl + t[ss + 1];
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const uint32_t w0 = r0[32 * v], w1 = r1[32 * v];
          aw[v] += w0 + w1;
          madd_hi16(ah[v], w0);
          madd_hi16(ah[v], w1);
        }
      }
      if (ss < ns) {
        const uint32_t* r0 = Sl + t[ss];
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const uint32_t w0 = r0[32 * v];
          aw[v] += w0;
          madd_hi16(ah[v], w0);
        }
      }
    }
    if (ch == nchunk - 1) {
      long long s1 = 0;
      unsigned long long s2 = 0;
      if (g < nd) {
        const int d = dfirst + g;
        int32_t* drow = D + (size_t)d * Dp;
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const int64_t ta = t0 + 2 * (jbase + lane + 32 * v);
          const uint32_t lo = aw[v] - (ah[v] << 16), hi = ah[v];
          if (ta + 1 < Td && (Dp & 1) == 0) {
            *reinterpret_cast<int2*>(drow + ta) = make_int2((int32_t)lo, (int32_t)hi);
          } else {
            if (ta < Td) drow[ta] = (int32_t)lo;
            if (ta + 1 < Td) drow[ta + 1] = (int32_t)hi;
          }
          if (ta < T) { s1 += lo; s2 += (unsigned long long)lo * lo; }
          if (ta + 1 < T) { s1 += hi; s2 += (unsigned long long)hi * hi; }
        }
      }
#pragma unroll
      for (int v = 0; v < VW; ++v) aw[v] = ah[v] = 0u;
      warp_sum_stats(s1, s2);
      if (SPLIT == 1) {
        if (g < nd && lane == 0) part[(size_t)(dfirst + g) * ntile + tile] = make_longlong2(s1, (long long)s2);
      } else {
        // combine the parts of each fine DM in a fixed order (deterministic sums)
        if (lane == 0) { st1[warp] = s1; st2[warp] = s2; }
        __syncthreads();
        if (part_i == 0 && g < nd && lane == 0) {
          long long a = 0;
          unsigned long long b = 0;
          for (int i = 0; i < SPLIT; ++i) { a += st1[warp + i]; b += st2[warp + i]; }
          part[(size_t)(dfirst + g) * ntile + tile] = make_longlong2(a, (long long)b);
        }
      }
    }
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
// statistics (Eq. 5's sigma: the standard deviation of the noise)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double u128_to_double(unsigned __int128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __dadd_rn(__dmul_rn((double)hi, 18446744073709551616.0), (double)lo);
}

// One thread per fine DM. mu = S1 / T, var = (T S2 - S1^2) / T^2 with an exact
// 128-bit numerator; the running mode updates (mu, var) <- (1 - l) prev + l new.
// Then, per width W: hi + lo = W mu (hi integer) and inv = 1 / (sigma sqrt W).
__global__ void k_stats(const longlong2* __restrict__ part, int ntile, int ndm, int64_t T, int nw,
                        const int32_t* __restrict__ widths, int running, double lam, double* __restrict__ run,
                        SnrConst* __restrict__ cst, double gamma) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndm) return;
  unsigned long long s1 = 0, s2 = 0;
  for (int i = 0; i < ntile; ++i) {
    const longlong2 v = part[(size_t)d * ntile + i];
    s1 += (unsigned long long)v.x;
    s2 += (unsigned long long)v.y;
  }
  double mu = __ddiv_rn((double)s1, (double)T);
  const unsigned __int128 num = (unsigned __int128)(unsigned long long)T * s2 - (unsigned __int128)s1 * s1;
  double var = __ddiv_rn(u128_to_double(num), __dmul_rn((double)T, (double)T));
  if (running) {
    double* r = run + (size_t)d * 2;
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
  const double sigma = sqrt(var);
  for (int w = 0; w < nw; ++w) {
    const double W = (double)widths[w];
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
    cst[(size_t)d * nw + w] = c;
  }
}

// ---------------------------------------------------------------------------
// boxcar matched filter (Eq. 5 via prefix sums, Sec. 2.4) and outputs (Sec. 2.5)
// ---------------------------------------------------------------------------
// Persistent blocks walk contiguous runs of units (fine DM d, tile of
// kBoxTile outputs); each unit's series (with its W_max - 1 look-ahead) is
// copied into shared memory with cp.async while the previous unit is being
// filtered, then turned in place into the prefix sum P (P[0] = 0), and each
// output t takes B_W = P[t + W] - P[t] for every width.
//   CUBE / PLANE: S/N for every width (float), best width for the plane.
//   CANDS: a point is a candidate when B_W >= thr_W for some width, an exact
//   integer form of S/N >= gamma; float S/N and the best width are computed
//   for those points only.
// NWT > 0: exactly NWT widths, per-width constants in registers.
// NWT = 0: any count up to kMaxWidths, constants in shared memory.
template <int NWT, int MODE>
__global__ void __launch_bounds__(kBoxThreads)
k_boxcar(const int32_t* __restrict__ D, int64_t Dp, int64_t T, int nw_rt, const int32_t* __restrict__ widths,
         int wmax, const SnrConst* __restrict__ cst, float* __restrict__ outf, uint8_t* __restrict__ outw,
         tx_cand* __restrict__ cands, unsigned long long* __restrict__ ncand, long long max_cands, int ndm,
         int ntile) {
  constexpr int NR = NWT > 0 ? NWT : 1;
  extern __shared__ __align__(16) uint32_t smb[];
  __shared__ uint32_t wsum[kBoxThreads / 32];
  __shared__ int32_t sW[kMaxWidths];
  __shared__ SnrConst sC[kMaxWidths];
  const int nw = NWT > 0 ? NWT : nw_rt;
  const int bufw = (kBoxTile + wmax + 8 + 3) & ~3;  // words per buffer: 4 pad + series + chunk rounding
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nunits = (int64_t)ndm * ntile;
  const int u_begin = (int)(nunits * blockIdx.x / gridDim.x), u_end = (int)(nunits * (blockIdx.x + 1) / gridDim.x);

  auto issue = [&](int unit, int buf) {
    const int d = unit / ntile, tile = unit - d * ntile;
    const int64_t t0 = (int64_t)tile * kBoxTile;
    const int n = (int)min((int64_t)kBoxTile, T - t0);
    const int nq = (n + wmax - 1 + 3) >> 2;  // 16-byte chunks of the series window
    const int32_t* src = D + (size_t)d * Dp + t0;
    uint32_t* dst = smb + (size_t)buf * bufw + 4;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) cp_async16(dst + 4 * q, src + 4 * q);
    cp_async_commit();
  };

  int32_t Wr[NR], thr[NR];
  int cur_d = -1;
  if (u_begin < u_end) issue(u_begin, 0);
  for (int unit = u_begin, it = 0; unit < u_end; ++unit, ++it) {
    const int buf = it & 1;
    const int d = unit / ntile, tile = unit - d * ntile;
    const int64_t t0 = (int64_t)tile * kBoxTile;
    const int n = (int)min((int64_t)kBoxTile, T - t0);
    const int N = n + wmax - 1;
    uint32_t* C = smb + (size_t)buf * bufw + 3;  // C[0] = P[0] = 0, C[1 + j] = D[j] -> P[1 + j]
    if (NWT > 0 && d != cur_d) {
#pragma unroll
      for (int w = 0; w < NR; ++w) {
        Wr[w] = __ldg(widths + w);
        thr[w] = cst[(size_t)d * nw + w].thr;
      }
    }
    cp_async_wait_all();
    __syncthreads();  // this unit's series landed; the previous unit is done with sW/sC and the other buffer
    if (NWT == 0 && d != cur_d && threadIdx.x < nw) {
      sW[threadIdx.x] = widths[threadIdx.x];
      sC[threadIdx.x] = cst[(size_t)d * nw + threadIdx.x];
    }
    cur_d = d;
    if (threadIdx.x == 0) C[0] = 0u;
    if (unit + 1 < u_end) issue(unit + 1, buf ^ 1);
    // inclusive scan of C[1..N] (uint32, wrap-around is harmless: window sums < 2^31)
    const int E = (N + blockDim.x - 1) / blockDim.x;
    const int beg = 1 + threadIdx.x * E, end = min(beg + E, N + 1);
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
      pre += C[i];
      C[i] = pre;
    }
    __syncthreads();

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t* Ci = C + i;
      const uint32_t cl = Ci[0];
      float best = -INFINITY;
      int bw = 0;
      bool hit = false;
      if (NWT > 0) {
        if (MODE == TX_OUT_CANDS) {
          int32_t m = INT32_MIN;
#pragma unroll
          for (int w = 0; w < NR; ++w) m = max(m, (int32_t)(Ci[Wr[w]] - cl) - thr[w]);
          hit = m >= 0;
          if (hit) {  // rare: float S/N and the best width of a candidate
            for (int w = 0; w < NR; ++w) {
              const SnrConst c = cst[(size_t)d * nw + w];
              const float sv = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
              if (sv > best) { best = sv; bw = w; }
            }
          }
        } else {
          float sv[NR];
#pragma unroll
          for (int w = 0; w < NR; ++w) {
            const SnrConst c = cst[(size_t)d * nw + w];
            sv[w] = ((float)((int32_t)(Ci[Wr[w]] - cl) - c.hi) - c.lo) * c.inv;
          }
          if (MODE == TX_OUT_CUBE) {
#pragma unroll
            for (int w = 0; w < NR; ++w) outf[((size_t)d * nw + w) * T + t0 + i] = sv[w];
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
          if (MODE == TX_OUT_CUBE) outf[((size_t)d * nw + w) * T + t0 + i] = snr;
          if (snr > best) { best = snr; bw = w; }
          hit = hit || B >= sC[w].thr;
        }
      }
      if (MODE == TX_OUT_PLANE) {
        outf[(size_t)d * T + t0 + i] = best;
        outw[(size_t)d * T + t0 + i] = (uint8_t)bw;
      } else if (MODE == TX_OUT_CANDS) {
        const unsigned act = __activemask();
        const unsigned hits = __ballot_sync(act, hit);
        if (hits) {
          const int leader = __ffs(hits) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(ncand, (unsigned long long)__popc(hits));
          base = __shfl_sync(act, base, leader);
          if (hit) {
            const unsigned long long idx = base + __popc(hits & ((1u << lane) - 1u));
            if (idx < (unsigned long long)max_cands) {
              tx_cand r;
              r.dm_index = d;
              r.t = (int32_t)(t0 + i);
              r.w_index = bw;
              r.snr = best;
              cands[idx] = r;
            }
          }
        }
      }
    }
  }
}

// Launch helper: exact width counts 1..12 and 16 get their own instantiation.
template <int NWT, int MODE>
void launch_boxcar_t(dim3 grid, int smem, cudaStream_t st, const int32_t* D, int64_t Dp, int64_t T, int nw,
                     const int32_t* widths, int wmax, const SnrConst* cst, float* outf, uint8_t* outw,
                     tx_cand* cands, unsigned long long* nc, long long max_cands, int ndm, int ntile) {
  k_boxcar<NWT, MODE><<<grid, kBoxThreads, smem, st>>>(D, Dp, T, nw, widths, wmax, cst, outf, outw, cands, nc,
                                                       max_cands, ndm, ntile);
}

using BoxLaunch = void (*)(dim3, int, cudaStream_t, const int32_t*, int64_t, int64_t, int, const int32_t*, int,
                           const SnrConst*, float*, uint8_t*, tx_cand*, unsigned long long*, long long, int, int);
using BoxKernel = void (*)(const int32_t*, int64_t, int64_t, int, const int32_t*, int, const SnrConst*, float*,
                           uint8_t*, tx_cand*, unsigned long long*, long long, int, int);

struct BoxEntry {
  BoxLaunch launch;
  BoxKernel kernel;
};

template <int MODE>
BoxEntry box_entry_m(int nw) {
  switch (nw) {
#define TX_BOX(N) \
  case N: return {launch_boxcar_t<N, MODE>, k_boxcar<N, MODE>};
    TX_BOX(1) TX_BOX(2) TX_BOX(3) TX_BOX(4) TX_BOX(5) TX_BOX(6) TX_BOX(7) TX_BOX(8) TX_BOX(9) TX_BOX(10)
    TX_BOX(11) TX_BOX(12) TX_BOX(16)
#undef TX_BOX
    default: return {launch_boxcar_t<0, MODE>, k_boxcar<0, MODE>};
  }
}

BoxEntry box_entry(int nw, int mode) {
  return mode == TX_OUT_CANDS ? box_entry_m<TX_OUT_CANDS>(nw)
         : mode == TX_OUT_PLANE ? box_entry_m<TX_OUT_PLANE>(nw) : box_entry_m<TX_OUT_CUBE>(nw);
}

__global__ void k_fill_run(double* run, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) run[2 * i + 1] = -1.0;  // marks "not initialised"
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <typename T>
int upload(T** dst, const std::vector<T>& v) {
  TX_CUDA(cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(T)));
  if (!v.empty()) TX_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TX_OK;
}

int stage2_smem(const tx_plan* p) {
  if (p->interm == TX_INTERM_U16)
    return (3 * p->nsub_chunk2 * p->sww2 + kStage2MaxGroup * p->nsub_chunk2) * 4;
  return p->nsub_chunk2 * p->sw2_i32 * 4;
}

// two buffers of (4 pad words + tile + look-ahead, rounded to 16-byte chunks)
int box_smem(const tx_plan* p) { return 2 * ((kBoxTile + p->wmax + 8 + 3) & ~3) * 4; }

template <int Q, typename PT>
int set_stage1_attr(int bytes) {
  TX_CUDA(cudaFuncSetAttribute(k_stage1<Q, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return TX_OK;
}

template <int NW, int MAXWARPS, int SPLIT>
int set_stage2_attr(int bytes) {
  TX_CUDA(cudaFuncSetAttribute(k_stage2_u16<NW, MAXWARPS, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return TX_OK;
}

// Warps per fine DM for the uint16 stage 2: enough to fill 32 warps.
int stage2_split(const tx_plan* p) {
  if (p->nw2 != 512) return 1;
  return p->group <= 4 ? 8 : p->group <= 8 ? 4 : p->group <= 16 ? 2 : 1;
}

int do_upload(tx_plan* p) {
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  p->dev.device = dev;
  TX_CUDA(cudaDeviceGetAttribute(&p->dev.num_sms, cudaDevAttrMultiProcessorCount, dev));
  int rc;
  if ((rc = upload(&p->dev.d1, p->d1))) return rc;
  if ((rc = upload(&p->dev.abase, p->abase))) return rc;
  if ((rc = upload(&p->dev.e2, p->e2))) return rc;
  if ((rc = upload(&p->dev.widths, p->widths))) return rc;
  if ((rc = upload(&p->dev.items1, p->items1))) return rc;
  const int s1 = (int)stage1_smem_bytes(p->m, p->q1);
  const bool u16 = p->interm == TX_INTERM_U16;
  switch (p->q1) {
    case 256: rc = u16 ? set_stage1_attr<256, uint16_t>(s1) : set_stage1_attr<256, int32_t>(s1); break;
    case 128: rc = u16 ? set_stage1_attr<128, uint16_t>(s1) : set_stage1_attr<128, int32_t>(s1); break;
    case 64: rc = u16 ? set_stage1_attr<64, uint16_t>(s1) : set_stage1_attr<64, int32_t>(s1); break;
    default: rc = u16 ? set_stage1_attr<32, uint16_t>(s1) : set_stage1_attr<32, int32_t>(s1); break;
  }
  if (rc) return rc;
  const int s2 = stage2_smem(p);
  if (u16) {
    switch (stage2_split(p)) {
      case 8: rc = set_stage2_attr<512, 32, 8>(s2); break;
      case 4: rc = set_stage2_attr<512, 32, 4>(s2); break;
      case 2: rc = set_stage2_attr<512, 32, 2>(s2); break;
      default: rc = set_stage2_attr<256, 32, 1>(s2); break;
    }
    if (rc) return rc;
  } else if (p->nw2 == 512) {
    TX_CUDA(cudaFuncSetAttribute(k_stage2_i32<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2));
  } else {
    TX_CUDA(cudaFuncSetAttribute(k_stage2_i32<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2));
  }
  if (p->output != TX_OUT_SERIES) {
    const BoxEntry be = box_entry(p->nw, p->output);
    TX_CUDA(cudaFuncSetAttribute(be.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, box_smem(p)));
    TX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->dev.box_blocks_per_sm, be.kernel, kBoxThreads,
                                                          box_smem(p)));
  }
  p->dev.box_blocks_per_sm = std::max(p->dev.box_blocks_per_sm, 1);
  return TX_OK;
}

template <int Q, typename PT>
void launch_stage1(const tx_plan* p, const uint8_t* ring, int64_t start, void* P, cudaStream_t st) {
  const int nitems = (int)p->items1.size();
  const int grid = std::min(nitems, std::max(p->dev.num_sms, 1));
  k_stage1<Q, PT><<<grid, kStage1Warps * 32, (int)stage1_smem_bytes(p->m, Q), st>>>(
      ring, (int)p->R, (int)start, p->dev.items1, nitems, p->dev.d1, p->nchan, p->m, p->nsub, p->dev.abase,
      reinterpret_cast<PT*>(P), p->Pp, 1u);
}

int check_beam(const tx_plan* p, const tx_beam* b) {
  if (!p || !b) { set_error("null plan or beam"); return TX_ERR_INVALID_ARG; }
  if (b->plan != p) { set_error("beam was created for another plan"); return TX_ERR_INVALID_ARG; }
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) { set_error("beam lives on device %d, current device is %d", b->device, dev); return TX_ERR_INVALID_ARG; }
  return TX_OK;
}

int64_t mod(int64_t a, int64_t r) { return ((a % r) + r) % r; }

// Writes n samples (plan layout, rows of n samples for FT) into the ring at
// physical positions [pos, pos + n) mod R, splitting at the wrap.
int ingest(const tx_plan* p, const uint8_t* src, int64_t n, uint8_t* ring, int64_t pos, cudaStream_t st) {
  if (n <= 0) return TX_OK;
  const int64_t R = p->R;
  int64_t done = 0;
  pos = mod(pos, R);
  while (done < n) {
    const int64_t len = std::min(n - done, R - pos);
    if (p->layout == TX_LAYOUT_TF) {
      const int vec = (p->nchan % 16 == 0) && (pos % 16 == 0) && (((uintptr_t)src & 15) == 0);
      dim3 grid((unsigned)((len + 63) / 64), (unsigned)((p->nchan + 63) / 64));
      k_ingest_tf<<<grid, 256, 0, st>>>(src, done, len, p->nchan, ring, R, pos, vec);
    } else {
      const int vec = (n % 16 == 0) && (done % 16 == 0) && (len % 16 == 0) && (pos % 16 == 0) &&
                      (((uintptr_t)src & 15) == 0);
      dim3 grid((unsigned)std::min<int64_t>((len + 4095) / 4096, 64), (unsigned)p->nchan);
      k_ingest_ft<<<grid, 256, 0, st>>>(src, n, done, len, ring, R, pos, vec);
    }
    TX_CUDA(cudaGetLastError());
    done += len;
    pos = 0;
  }
  return TX_OK;
}

// Copies the carried tail (the L samples before `head`, per channel) between
// the ring and a host buffer [nchan][L].
int copy_tail(const tx_plan* p, const tx_beam* b, uint8_t* host, bool to_host) {
  const int64_t L = p->L, R = p->R;
  if (L <= 0) return TX_OK;
  const int64_t a = mod(b->head - L, R);
  const int64_t first = std::min(L, R - a);
  if (to_host) {
    TX_CUDA(cudaMemcpy2D(host, (size_t)L, b->ring + a, (size_t)R, (size_t)first, (size_t)p->nchan, cudaMemcpyDeviceToHost));
    if (first < L)
      TX_CUDA(cudaMemcpy2D(host + first, (size_t)L, b->ring, (size_t)R, (size_t)(L - first), (size_t)p->nchan,
                           cudaMemcpyDeviceToHost));
  } else {
    TX_CUDA(cudaMemcpy2D(b->ring + a, (size_t)R, host, (size_t)L, (size_t)first, (size_t)p->nchan, cudaMemcpyHostToDevice));
    if (first < L)
      TX_CUDA(cudaMemcpy2D(b->ring, (size_t)R, host + first, (size_t)L, (size_t)(L - first), (size_t)p->nchan,
                           cudaMemcpyHostToDevice));
  }
  return TX_OK;
}

}  // namespace

int tx_upload_plan(const tx_plan* cp) {
  tx_plan* p = const_cast<tx_plan*>(cp);
  std::call_once(p->dev_once, [p] { p->dev_status = do_upload(p); });
  if (p->dev_status) return p->dev_status;
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev != p->dev.device) { set_error("plan tables live on device %d, current device is %d", p->dev.device, dev); return TX_ERR_INVALID_ARG; }
  return TX_OK;
}

extern "C" {

void tx_plan_destroy(tx_plan* p) {
  if (!p) return;
  if (p->dev.device >= 0) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->dev.device);
    cudaFree(p->dev.d1);
    cudaFree(p->dev.abase);
    cudaFree(p->dev.e2);
    cudaFree(p->dev.widths);
    cudaFree(p->dev.items1);
    cudaSetDevice(prev);
  }
  delete p;
}

int32_t tx_beam_create(const tx_plan* p, tx_beam** out) {
  if (!p || !out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  int rc = tx_upload_plan(p);
  if (rc) return rc;
  tx_beam* b = new (std::nothrow) tx_beam();
  if (!b) { set_error("out of host memory"); return TX_ERR_OOM; }
  b->plan = p;
  cudaGetDevice(&b->device);
  cudaError_t e = cudaMalloc((void**)&b->ring, (size_t)p->nchan * p->R);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->run, (size_t)p->ndm * 2 * sizeof(double));
  if (e != cudaSuccess) {
    set_error("beam allocation failed: %s", cudaGetErrorString(e));
    tx_beam_destroy(b);
    return e == cudaErrorMemoryAllocation ? TX_ERR_OOM : TX_ERR_CUDA;
  }
  rc = tx_beam_reset(p, b, nullptr);
  if (rc == TX_OK && cudaDeviceSynchronize() != cudaSuccess) {
    set_error("beam initialisation failed");
    rc = TX_ERR_CUDA;
  }
  if (rc) { tx_beam_destroy(b); return rc; }
  *out = b;
  return TX_OK;
}

int32_t tx_beam_reset(const tx_plan* p, tx_beam* b, void* stream) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  TX_CUDA(cudaMemsetAsync(b->ring, 0, (size_t)p->nchan * p->R, st));
  TX_CUDA(cudaMemsetAsync(b->run, 0, (size_t)p->ndm * 2 * sizeof(double), st));
  k_fill_run<<<(p->ndm + 255) / 256, 256, 0, st>>>(b->run, p->ndm);
  TX_CUDA(cudaGetLastError());
  b->head = p->head0;
  b->nblocks = 0;
  return TX_OK;
}

int32_t tx_beam_prime(const tx_plan* p, tx_beam* b, const uint8_t* d_tail, void* stream) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!d_tail && p->L > 0) { set_error("null tail"); return TX_ERR_INVALID_ARG; }
  // the tail sits in the L positions before the next block
  return ingest(p, d_tail, p->L, b->ring, b->head - p->L, (cudaStream_t)stream);
}

int32_t tx_beam_blocks(const tx_beam* b, int64_t* n) {
  if (!b || !n) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  *n = b->nblocks;
  return TX_OK;
}

int32_t tx_beam_export(const tx_plan* p, const tx_beam* b, void* h_dst, int64_t bytes) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!h_dst || bytes < p->export_bytes) { set_error("export buffer needs %lld bytes", (long long)p->export_bytes); return TX_ERR_INVALID_ARG; }
  uint8_t* h = static_cast<uint8_t*>(h_dst);
  std::memset(h, 0, 64);
  const int64_t hdr[4] = {0x54584245414d32LL, p->nchan, p->L, b->nblocks};
  std::memcpy(h, hdr, sizeof(hdr));
  TX_CUDA(cudaDeviceSynchronize());
  if ((rc = copy_tail(p, b, h + 64, true))) return rc;
  TX_CUDA(cudaMemcpy(h + 64 + (size_t)p->nchan * p->L, b->run, (size_t)p->ndm * 16, cudaMemcpyDeviceToHost));
  return TX_OK;
}

int32_t tx_beam_import(const tx_plan* p, tx_beam* b, const void* h_src, int64_t bytes) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!h_src || bytes < p->export_bytes) { set_error("import buffer needs %lld bytes", (long long)p->export_bytes); return TX_ERR_INVALID_ARG; }
  const uint8_t* h = static_cast<const uint8_t*>(h_src);
  int64_t hdr[4];
  std::memcpy(hdr, h, sizeof(hdr));
  if (hdr[0] != 0x54584245414d32LL || hdr[1] != p->nchan || hdr[2] != p->L) { set_error("export does not match this plan"); return TX_ERR_INVALID_ARG; }
  TX_CUDA(cudaDeviceSynchronize());
  if ((rc = copy_tail(p, b, const_cast<uint8_t*>(h + 64), false))) return rc;
  TX_CUDA(cudaMemcpy(b->run, h + 64 + (size_t)p->nchan * p->L, (size_t)p->ndm * 16, cudaMemcpyHostToDevice));
  b->nblocks = hdr[3];
  return TX_OK;
}

void tx_beam_destroy(tx_beam* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (b->device >= 0) cudaSetDevice(b->device);
  cudaFree(b->ring);
  cudaFree(b->run);
  cudaSetDevice(prev);
  delete b;
}

}  // extern "C"

struct tx_timer {
  int device = -1;
  int32_t max_steps = 0, nsteps = 0;
  std::vector<cudaEvent_t> ev;  // [max_steps][TX_NPHASES + 1]
};

namespace {

#define TX_MARK(i)                                                     \
  do {                                                                 \
    if (ev) TX_CUDA(cudaEventRecord(ev[(i)], st));                     \
  } while (0)

int execute_impl(const tx_plan* p, tx_beam* b, const uint8_t* d_block, void* d_out, int64_t* d_ncand,
                 void* d_workspace, void* stream, cudaEvent_t* ev) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!d_block || !d_out || !d_workspace) { set_error("null device buffer"); return TX_ERR_INVALID_ARG; }
  if (p->output == TX_OUT_CANDS && !d_ncand) { set_error("candidate mode needs d_ncand"); return TX_ERR_INVALID_ARG; }
  if ((rc = tx_upload_plan(p))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = static_cast<uint8_t*>(d_workspace);
  TX_MARK(0);

  // Sec. 2.3 data flow: the block lands behind the carried tail (steps 1, 2, 4)
  if ((rc = ingest(p, d_block, p->T, b->ring, b->head, st))) return rc;
  const int64_t start = mod(b->head - p->L, p->R);
  b->head = mod(b->head + p->T, p->R);
  TX_MARK(1);

  // stage 1
  void* P = ws + p->ws_P;
  const bool u16 = p->interm == TX_INTERM_U16;
  switch (p->q1) {
    case 256: u16 ? launch_stage1<256, uint16_t>(p, b->ring, start, P, st) : launch_stage1<256, int32_t>(p, b->ring, start, P, st); break;
    case 128: u16 ? launch_stage1<128, uint16_t>(p, b->ring, start, P, st) : launch_stage1<128, int32_t>(p, b->ring, start, P, st); break;
    case 64: u16 ? launch_stage1<64, uint16_t>(p, b->ring, start, P, st) : launch_stage1<64, int32_t>(p, b->ring, start, P, st); break;
    default: u16 ? launch_stage1<32, uint16_t>(p, b->ring, start, P, st) : launch_stage1<32, int32_t>(p, b->ring, start, P, st); break;
  }
  TX_CUDA(cudaGetLastError());
  TX_MARK(2);

  // stage 2 (+ exact per-tile sums)
  const bool series = p->output == TX_OUT_SERIES;
  int32_t* D = series ? static_cast<int32_t*>(d_out) : reinterpret_cast<int32_t*>(ws + p->ws_D);
  const int64_t Dp = series ? p->Td : p->Dp;
  longlong2* part = reinterpret_cast<longlong2*>(ws + p->ws_part);
  {
    const int threads = std::min(p->group, kStage2MaxGroup) * 32;
    if (u16) {
      const int nunits = p->nk * p->ntile2;
      const int grid = std::min(nunits, std::max(p->dev.num_sms, 1));
      const int split = stage2_split(p);
      const int nthreads = std::min(p->group, kStage2MaxGroup) * 32 * split;
#define TX_S2(NW, SP)                                                                                          \
  k_stage2_u16<NW, 32, SP><<<grid, nthreads, stage2_smem(p), st>>>(                                            \
      static_cast<const uint16_t*>(P), p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nk, p->nsub_chunk2,     \
      p->sww2, p->ntile2, D, Dp, p->Td, p->T, part, nullptr)
      switch (split) {
        case 8: TX_S2(512, 8); break;
        case 4: TX_S2(512, 4); break;
        case 2: TX_S2(512, 2); break;
        default: TX_S2(256, 1); break;
      }
#undef TX_S2
    } else {
      dim3 grid((unsigned)p->ntile2, (unsigned)p->nk);
      if (p->nw2 == 512)
        k_stage2_i32<512><<<grid, threads, stage2_smem(p), st>>>(
            static_cast<const int32_t*>(P), p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nsub_chunk2, p->sw2_i32,
            D, Dp, p->Td, p->T, part, p->ntile2);
      else
        k_stage2_i32<256><<<grid, threads, stage2_smem(p), st>>>(
            static_cast<const int32_t*>(P), p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nsub_chunk2, p->sw2_i32,
            D, Dp, p->Td, p->T, part, p->ntile2);
    }
    TX_CUDA(cudaGetLastError());
  }
  TX_MARK(3);

  if (!series) {
    SnrConst* cst = reinterpret_cast<SnrConst*>(ws + p->ws_const);
    k_stats<<<(p->ndm + 127) / 128, 128, 0, st>>>(part, p->ntile2, p->ndm, p->T, p->nw, p->dev.widths,
                                                  p->stats == TX_STATS_RUNNING, p->lambda, b->run, cst,
                                                  (double)p->gamma);
    TX_CUDA(cudaGetLastError());
    TX_MARK(4);
    if (p->output == TX_OUT_CANDS) TX_CUDA(cudaMemsetAsync(d_ncand, 0, sizeof(int64_t), st));
    float* outf = static_cast<float*>(d_out);
    uint8_t* outw = p->output == TX_OUT_PLANE ? static_cast<uint8_t*>(d_out) + (size_t)p->ndm * p->T * 4 : nullptr;
    auto* cands = static_cast<tx_cand*>(d_out);
    auto* nc = reinterpret_cast<unsigned long long*>(d_ncand);
    const int nunits = p->ndm * p->ntile3;
    const dim3 grid((unsigned)std::min(nunits, std::max(p->dev.num_sms, 1) * p->dev.box_blocks_per_sm));
    box_entry(p->nw, p->output).launch(grid, box_smem(p), st, D, p->Dp, p->T, p->nw, p->dev.widths, p->wmax, cst,
                                       outf, outw, cands, nc, (long long)p->max_cands, p->ndm, p->ntile3);
    TX_CUDA(cudaGetLastError());
  } else {
    TX_MARK(4);
  }
  TX_MARK(5);
  ++b->nblocks;
  return TX_OK;
}

}  // namespace

extern "C" {

int32_t tx_execute(const tx_plan* p, tx_beam* b, const uint8_t* d_block, void* d_out, int64_t* d_ncand,
                   void* d_workspace, void* stream) {
  return execute_impl(p, b, d_block, d_out, d_ncand, d_workspace, stream, nullptr);
}

int32_t tx_timer_create(int32_t max_steps, tx_timer** out) {
  if (!out || max_steps < 1) { set_error("need max_steps >= 1"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  tx_timer* t = new (std::nothrow) tx_timer();
  if (!t) { set_error("out of host memory"); return TX_ERR_OOM; }
  cudaGetDevice(&t->device);
  t->max_steps = max_steps;
  t->ev.assign((size_t)max_steps * (TX_NPHASES + 1), nullptr);
  for (auto& e : t->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      set_error("cudaEventCreate failed");
      tx_timer_destroy(t);
      return TX_ERR_CUDA;
    }
  }
  *out = t;
  return TX_OK;
}

int32_t tx_timer_clear(tx_timer* t) {
  if (!t) { set_error("null timer"); return TX_ERR_INVALID_ARG; }
  t->nsteps = 0;
  return TX_OK;
}

int32_t tx_execute_timed(const tx_plan* p, tx_beam* b, const uint8_t* d_block, void* d_out, int64_t* d_ncand,
                         void* d_workspace, void* stream, tx_timer* t) {
  if (!t) { set_error("null timer"); return TX_ERR_INVALID_ARG; }
  if (t->nsteps >= t->max_steps) { set_error("timer is full (%d steps)", t->max_steps); return TX_ERR_INVALID_ARG; }
  const int rc = execute_impl(p, b, d_block, d_out, d_ncand, d_workspace, stream,
                              t->ev.data() + (size_t)t->nsteps * (TX_NPHASES + 1));
  if (rc == TX_OK) ++t->nsteps;
  return rc;
}

int32_t tx_timer_read(tx_timer* t, double* h_ms, int32_t* nsteps, double* h_step_ms) {
  if (!t || !h_ms) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < TX_NPHASES; ++i) h_ms[i] = 0.0;
  if (nsteps) *nsteps = t->nsteps;
  if (!t->nsteps) return TX_OK;
  TX_CUDA(cudaEventSynchronize(t->ev[(size_t)t->nsteps * (TX_NPHASES + 1) - 1]));
  for (int s = 0; s < t->nsteps; ++s) {
    const cudaEvent_t* e = t->ev.data() + (size_t)s * (TX_NPHASES + 1);
    for (int i = 0; i < TX_NPHASES; ++i) {
      float ms = 0.f;
      TX_CUDA(cudaEventElapsedTime(&ms, e[i], e[i + 1]));
      h_ms[i] += ms;
    }
    if (h_step_ms) {
      float ms = 0.f;
      TX_CUDA(cudaEventElapsedTime(&ms, e[0], e[TX_NPHASES]));
      h_step_ms[s] = ms;
    }
  }
  return TX_OK;
}

void tx_timer_destroy(tx_timer* t) {
  if (!t) return;
  for (auto e : t->ev)
    if (e) cudaEventDestroy(e);
  delete t;
}

int32_t tx_execute_host(const tx_plan* p, tx_beam* b, const uint8_t* h_block, void* h_out, int64_t* h_ncand,
                        uint8_t* d_block_staging, void* d_out, int64_t* d_ncand, void* d_workspace, void* stream) {
  if (!p || !h_block || !h_out || !d_block_staging) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (p->output == TX_OUT_CANDS && !h_ncand) { set_error("candidate mode needs h_ncand"); return TX_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  TX_CUDA(cudaMemcpyAsync(d_block_staging, h_block, (size_t)p->nchan * p->T, cudaMemcpyHostToDevice, st));
  int rc = tx_execute(p, b, d_block_staging, d_out, d_ncand, d_workspace, stream);
  if (rc) return rc;
  if (p->output == TX_OUT_CANDS) {
    TX_CUDA(cudaMemcpyAsync(h_ncand, d_ncand, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TX_CUDA(cudaStreamSynchronize(st));
    const int64_t n = std::min<int64_t>(*h_ncand, p->max_cands);
    if (n > 0) TX_CUDA(cudaMemcpyAsync(h_out, d_out, (size_t)n * sizeof(tx_cand), cudaMemcpyDeviceToHost, st));
    TX_CUDA(cudaStreamSynchronize(st));
    if (*h_ncand > p->max_cands) { set_error("%lld candidates, capacity %lld", (long long)*h_ncand, (long long)p->max_cands); return TX_ERR_CAND_OVERFLOW; }
    return TX_OK;
  }
  TX_CUDA(cudaMemcpyAsync(h_out, d_out, (size_t)p->out_bytes, cudaMemcpyDeviceToHost, st));
  TX_CUDA(cudaStreamSynchronize(st));
  return TX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free de-dispersion
// ---------------------------------------------------------------------------
// Some callers cannot call cudaMalloc: a real-time acquisition loop that must
// not take the allocator's locks or risk the implicit device synchronisation an
// allocation can cause, a host that embeds this library under a fixed
// device-memory budget owned by another framework, or code that must never
// fail for lack of memory once running. tx_dedisperse_noalloc serves them: the
// caller passes the input window and the output series; the stage-1 sums, the
// per-tile sums and copies of the plan's tables live in the file-scope array
// below, which every GPU that loads this library holds until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
int noalloc_scratch(void** out) {
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) { set_error("device %d out of range", dev); return TX_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return TX_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return TX_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

int32_t tx_dedisperse_noalloc(const tx_plan* p, const uint8_t* d_x, int64_t ld, int32_t* d_series, void* stream) {
  if (!p || !d_x || !d_series) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (p->interm != TX_INTERM_U16) { set_error("tx_dedisperse_noalloc needs a plan with uint16 intermediates"); return TX_ERR_UNSUPPORTED; }
  if (ld < p->L + p->T || ld % 64 != 0 || ld >= (int64_t)1 << 30 || ((uintptr_t)d_x & 15) != 0) {
    set_error("d_x needs a 16-byte aligned start and a row pitch ld that is a multiple of 64 and >= L + T (%lld)",
              (long long)(p->L + p->T));
    return TX_ERR_INVALID_ARG;
  }
  // scratch layout: stage-1 work items, d1, abase, e2, stage-1 sums, per-tile sums
  const size_t b_items = align256(p->items1.size() * sizeof(Stage1Item));
  const size_t b_d1 = align256(p->d1.size() * 4);
  const size_t b_abase = align256(p->abase.size() * 4);
  const size_t b_e2 = align256(p->e2.size() * 4);
  const size_t b_P = align256((size_t)p->nk * p->nsub * p->Pp * 2);
  const size_t b_part = align256((size_t)p->ndm * p->ntile2 * 16);
  const size_t need = b_items + b_d1 + b_abase + b_e2 + b_P + b_part;
  if (need > kNoAllocScratchBytes) {
    set_error("this plan needs %zu bytes of scratch; the static scratch of tx_dedisperse_noalloc holds %zu",
              need, kNoAllocScratchBytes);
    return TX_ERR_BUDGET;
  }
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  int dev = 0, nsm = 0;
  TX_CUDA(cudaGetDevice(&dev));
  TX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  uint8_t* base = static_cast<uint8_t*>(scratch);
  Stage1Item* items = reinterpret_cast<Stage1Item*>(base);
  int32_t* d1 = reinterpret_cast<int32_t*>(base + b_items);
  int32_t* abase = reinterpret_cast<int32_t*>(base + b_items + b_d1);
  int32_t* e2 = reinterpret_cast<int32_t*>(base + b_items + b_d1 + b_abase);
  uint16_t* P = reinterpret_cast<uint16_t*>(base + b_items + b_d1 + b_abase + b_e2);
  longlong2* part = reinterpret_cast<longlong2*>(base + b_items + b_d1 + b_abase + b_e2 + b_P);
  cudaStream_t st = (cudaStream_t)stream;
  TX_CUDA(cudaMemcpyAsync(items, p->items1.data(), p->items1.size() * sizeof(Stage1Item), cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(d1, p->d1.data(), p->d1.size() * 4, cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(abase, p->abase.data(), p->abase.size() * 4, cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(e2, p->e2.data(), p->e2.size() * 4, cudaMemcpyHostToDevice, st));
  // Nothing in the scratch must start at zero: stage 1 writes every stage-1
  // sum that stage 2 reads, and stage 2 writes every per-tile sum.

  // stage 1 on the caller's window (a linear buffer read as a ring of length ld)
  const int nitems = (int)p->items1.size();
  const int smem1 = (int)stage1_smem_bytes(p->m, p->q1);
  const int grid1 = std::min(nitems, std::max(nsm, 1));
#define TX_NA_S1(Q)                                                                                      \
  do {                                                                                                   \
    TX_CUDA(cudaFuncSetAttribute(k_stage1<Q, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1)); \
    k_stage1<Q, uint16_t><<<grid1, kStage1Warps * 32, smem1, st>>>(d_x, (int)ld, 0, items, nitems, d1, p->nchan, \
                                                                   p->m, p->nsub, abase, P, p->Pp, 1u);   \
  } while (0)
  switch (p->q1) {
    case 256: TX_NA_S1(256); break;
    case 128: TX_NA_S1(128); break;
    case 64: TX_NA_S1(64); break;
    default: TX_NA_S1(32); break;
  }
#undef TX_NA_S1
  TX_CUDA(cudaGetLastError());

  // stage 2 into the caller's series [ndm][T + W_max - 1]
  const int smem2 = (3 * p->nsub_chunk2 * p->sww2 + kStage2MaxGroup * p->nsub_chunk2) * 4;
  const int nunits = p->nk * p->ntile2;
  const int grid2 = std::min(nunits, std::max(nsm, 1));
  const int split = p->nw2 != 512 ? 1 : p->group <= 4 ? 8 : p->group <= 8 ? 4 : p->group <= 16 ? 2 : 1;
  const int nthreads = std::min(p->group, kStage2MaxGroup) * 32 * split;
#define TX_NA_S2(NW, SP)                                                                                        \
  do {                                                                                                          \
    TX_CUDA(cudaFuncSetAttribute(k_stage2_u16<NW, 32, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2)); \
    k_stage2_u16<NW, 32, SP><<<grid2, nthreads, smem2, st>>>(P, p->Pp, e2, p->ndm, p->nsub, p->group, p->nk,      \
                                                             p->nsub_chunk2, p->sww2, p->ntile2, d_series, p->Td, \
                                                             p->Td, p->T, part, nullptr);                         \
  } while (0)
  switch (split) {
    case 8: TX_NA_S2(512, 8); break;
    case 4: TX_NA_S2(512, 4); break;
    case 2: TX_NA_S2(512, 2); break;
    default: TX_NA_S2(256, 1); break;
  }
#undef TX_NA_S2
  TX_CUDA(cudaGetLastError());
  return TX_OK;
}

}  // extern "C"
