// CUDA side (sm_103a) of the library: ingest, two-stage sub-band
// de-dispersion (Sec. 2.3), block statistics, and the boxcar matched filter
// with its outputs (Sec. 2.4, 2.5); plus the C-ABI entry points that launch
// them.
//
// Kernel map (one execute):
//   k_tail / k_ingest_*   Sec. 2.3 data-flow steps 1, 2 and 4: the carried
//                         tail and the new block land channel-major in the
//                         beam's next ring buffer (time-major input is
//                         transposed on the way).
//   k_stage1              stage 1: P[k][s][t] = sum_{c in s} X[c][t + d1[k][c]]
//   k_stage2_*            stage 2: D[d][t] = sum_s P[k(d)][s][t + d2[d][s]],
//                         plus exact per-tile sums of D and D^2
//   k_stats               mean / sigma per DM (block or running), and the
//                         per-width constants of Eq. 5
//   k_boxcar              prefix sums, window sums for every width, S/N
//                         (Eq. 5), best width, and cube / plane / candidates
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
// ingest (Sec. 2.3 data flow)
// ---------------------------------------------------------------------------
// Channel-major block [nchan][n] -> ring rows at byte offset `off`.
__global__ void k_ingest_ft(const uint8_t* __restrict__ src, int64_t n, uint8_t* __restrict__ ring,
                            int64_t Rp, int64_t off) {
  const int c = blockIdx.y;
  const uint8_t* s = src + (int64_t)c * n;
  uint8_t* d = ring + (int64_t)c * Rp + off;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// Same with 16-byte vectors (n, off, the source rows and the ring rows all 16-byte aligned).
__global__ void k_ingest_ft16(const uint4* __restrict__ src, int64_t n16, uint8_t* __restrict__ ring,
                              int64_t Rp, int64_t off) {
  const int c = blockIdx.y;
  const uint4* s = src + (int64_t)c * n16;
  uint4* d = reinterpret_cast<uint4*>(ring + (int64_t)c * Rp + off);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// Time-major block [n][nchan] -> ring[c][off + t], through a 64 x 64 byte tile.
__global__ void __launch_bounds__(256) k_ingest_tf(const uint8_t* __restrict__ src, int64_t n, int nchan,
                                                   uint8_t* __restrict__ ring, int64_t Rp, int64_t off) {
  __shared__ uint8_t tile[64][68];
  const int64_t t0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int tt = i >> 6, cc = i & 63;
    if (t0 + tt < n && c0 + cc < nchan) tile[tt][cc] = src[(t0 + tt) * nchan + c0 + cc];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int cc = i >> 6, tt = i & 63;
    if (t0 + tt < n && c0 + cc < nchan) ring[(int64_t)(c0 + cc) * Rp + off + t0 + tt] = tile[tt][cc];
  }
}

// Carried tail: next[c][pad + i] = cur[c][pad + T + i], i in [0, L).
__global__ void k_tail(const uint8_t* __restrict__ cur, uint8_t* __restrict__ nxt, int64_t Rp, int64_t src_off,
                       int64_t dst_off, int64_t L) {
  const int c = blockIdx.y;
  const uint8_t* s = cur + (int64_t)c * Rp + src_off;
  uint8_t* d = nxt + (int64_t)c * Rp + dst_off;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// ---------------------------------------------------------------------------
// stage 1 (Sec. 2.3: de-disperse each sub-band on the coarse DM grid)
// ---------------------------------------------------------------------------
// One block = one work item: sub-band s, coarse DMs [kb, ke), absolute times
// [tau0, tau0 + 4Q). Shared word S[c][j] holds channel c's samples at times
// tau0 + d1[kb][c] + j + qQ in byte q (q = 0..3). For coarse DM k the output
// word j is sum_c S[c][j + d1[k][c] - d1[kb][c]], four outputs per 32-bit
// load whatever the delays. Sums use the byte-lane identity
//   sum w = sum(lo lanes) + 256 * sum(hi lanes)  (mod 2^32)
// with the hi lanes (bytes 1, 3) accumulated separately as 16-bit lanes,
// exact for up to 257 channels per sub-band.
template <int Q, typename PT>
__global__ void __launch_bounds__(kStage1Warps * 32)
k_stage1(const uint8_t* __restrict__ ring, int64_t Rp, int64_t pad, const Stage1Item* __restrict__ items,
         const int32_t* __restrict__ spans, const int32_t* __restrict__ d1, int nchan, int m, int nsub,
         const int32_t* __restrict__ abase, PT* __restrict__ P, int64_t Pp) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int SW = 2 * Q + 4;  // words per staged channel: Q + span (span <= Q), 16-byte rows
  constexpr int V = Q / 32;
  uint32_t* S = smem;
  int32_t* off = reinterpret_cast<int32_t*>(smem + (size_t)m * SW);
  const Stage1Item it = items[blockIdx.x];
  const int span = spans[blockIdx.x];
  const int nkk = it.ke - it.kb;
  const int c0 = it.s * m;
  const int32_t* d1kb = d1 + (size_t)it.kb * nchan + c0;

  for (int i = threadIdx.x; i < nkk * m; i += blockDim.x) {
    const int kk = i / m, c = i - kk * m;
    off[i] = d1[(size_t)(it.kb + kk) * nchan + c0 + c] - d1kb[c];
  }
  const int nw4 = (Q + span + 3) >> 2;
  for (int i = threadIdx.x; i < m * nw4; i += blockDim.x) {
    const int c = i / nw4, j = (i - c * nw4) << 2;
    const uint8_t* row = ring + (size_t)(c0 + c) * Rp;
    const int64_t b = pad + (int64_t)it.tau0 + d1kb[c] + j;
    uint32_t r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t p = b + (int64_t)q * Q;
      const uint32_t* wp = reinterpret_cast<const uint32_t*>(row + (p & ~(int64_t)3));
      r[q] = __funnelshift_r(__ldg(wp), __ldg(wp + 1), (unsigned)(p & 3) * 8u);
    }
    // 4 x 4 byte transpose: word j+i collects byte i of each quarter
    const uint32_t t0 = __byte_perm(r[0], r[1], 0x5140), t1 = __byte_perm(r[0], r[1], 0x7362);
    const uint32_t t2 = __byte_perm(r[2], r[3], 0x5140), t3 = __byte_perm(r[2], r[3], 0x7362);
    uint4 w;
    w.x = __byte_perm(t0, t2, 0x5410);
    w.y = __byte_perm(t0, t2, 0x7632);
    w.z = __byte_perm(t1, t3, 0x5410);
    w.w = __byte_perm(t1, t3, 0x7632);
    *reinterpret_cast<uint4*>(S + (size_t)c * SW + j) = w;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int kk = warp; kk < nkk; kk += kStage1Warps) {
    const int k = it.kb + kk;
    const int64_t ab = abase[(size_t)k * nsub + it.s];
    if ((int64_t)it.tau0 + 4 * Q <= ab || (int64_t)it.tau0 >= ab + Pp) continue;
    uint32_t aw[V], ah[V];
#pragma unroll
    for (int v = 0; v < V; ++v) aw[v] = ah[v] = 0u;
    const int32_t* o = off + kk * m;
    const uint32_t* base = S + lane;
#pragma unroll 4
    for (int c = 0; c < m; ++c) {
      const uint32_t* rw = base + (size_t)c * SW + o[c];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const uint32_t w = rw[32 * v];
        aw[v] += w;
        ah[v] += __byte_perm(w, 0u, 0x4341);
      }
    }
    PT* prow = P + ((size_t)k * nsub + it.s) * Pp;
    const int64_t rel0 = (int64_t)it.tau0 - ab;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int j = lane + 32 * v;
      const uint32_t lo = aw[v] - (ah[v] << 8);
      const uint32_t val[4] = {lo & 0xFFFFu, ah[v] & 0xFFFFu, lo >> 16, ah[v] >> 16};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t u = rel0 + j + (int64_t)q * Q;
        if (u >= 0 && u < Pp) prow[u] = (PT)val[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// stage 2 (Sec. 2.3: de-disperse the sub-bands on the fine DM grid)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load4_u16(const uint16_t* __restrict__ row, int64_t a, uint32_t& x0, uint32_t& x1) {
  const uint32_t* wp = reinterpret_cast<const uint32_t*>(row + (a & ~(int64_t)1));
  const uint32_t w0 = __ldg(wp), w1 = __ldg(wp + 1), w2 = __ldg(wp + 2);
  if (a & 1) {
    x0 = __funnelshift_r(w0, w1, 16);
    x1 = __funnelshift_r(w1, w2, 16);
  } else {
    x0 = w0;
    x1 = w1;
  }
}

__device__ __forceinline__ void warp_sum_stats(long long& s1, unsigned long long& s2) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
}

// One block = (time tile, coarse group k); warp g handles fine DM kG + g.
// Shared word S[s][j] pairs the uint16 sums P[k][s] at times t0 + emin_s + j
// and t0 + emin_s + j + Q, so a 32-bit load feeds two outputs. Sums use
//   sum w = sum(lo) + 65536 * sum(hi) (mod 2^32), sum(hi) = sum(w >> 16),
// exact because every stage-2 sum is below 2^32.
template <int Q>
__global__ void __launch_bounds__(kStage2MaxGroup * 32)
k_stage2_u16(const uint16_t* __restrict__ P, int64_t Pp, const int32_t* __restrict__ e2, int ndm, int nsub,
             int G, int sc, int SW, int32_t* __restrict__ D, int64_t Dp, int64_t Td, int64_t T,
             longlong2* __restrict__ part, int ntile) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int V = Q / 32;
  const int tile = blockIdx.x, k = blockIdx.y;
  const int64_t t0 = (int64_t)tile * 2 * Q;
  const int dfirst = k * G;
  const int nd = min(G, ndm - dfirst);
  int32_t* emin = reinterpret_cast<int32_t*>(smem);
  int32_t* off = emin + nsub;
  uint32_t* S = smem + (((size_t)nsub * (1 + kStage2MaxGroup) + 3) & ~(size_t)3);
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) emin[s] = e2[(size_t)dfirst * nsub + s];
  for (int i = threadIdx.x; i < nd * nsub; i += blockDim.x) {
    const int g = i / nsub, s = i - g * nsub;
    off[i] = e2[(size_t)(dfirst + g) * nsub + s] - e2[(size_t)dfirst * nsub + s];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t aw[V], ah[V];
#pragma unroll
  for (int v = 0; v < V; ++v) aw[v] = ah[v] = 0u;
  const int nwq = (SW - 4) >> 2;  // staged words / 4
  for (int sb = 0; sb < nsub; sb += sc) {
    const int ns = min(sc, nsub - sb);
    for (int i = threadIdx.x; i < ns * nwq; i += blockDim.x) {
      const int ss = i / nwq, j = (i - ss * nwq) << 2;
      const int s = sb + ss;
      const uint16_t* prow = P + ((size_t)k * nsub + s) * Pp;
      const int64_t a = t0 + emin[s] + j;
      uint32_t x0, x1, y0, y1;
      load4_u16(prow, a, x0, x1);
      load4_u16(prow, a + Q, y0, y1);
      uint4 w;
      w.x = __byte_perm(x0, y0, 0x5410);
      w.y = __byte_perm(x0, y0, 0x7632);
      w.z = __byte_perm(x1, y1, 0x5410);
      w.w = __byte_perm(x1, y1, 0x7632);
      *reinterpret_cast<uint4*>(S + (size_t)ss * SW + j) = w;
    }
    __syncthreads();
    if (warp < nd) {
      const int32_t* o = off + warp * nsub + sb;
      const uint32_t* base = S + lane;
#pragma unroll 4
      for (int ss = 0; ss < ns; ++ss) {
        const uint32_t* rw = base + (size_t)ss * SW + o[ss];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const uint32_t w = rw[32 * v];
          aw[v] += w;
          ah[v] += w >> 16;
        }
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
      const int j = lane + 32 * v;
      const uint32_t lo = aw[v] - (ah[v] << 16);
      const int64_t ta = t0 + j, tb = t0 + Q + j;
      if (ta < Td) drow[ta] = (int32_t)lo;
      if (tb < Td) drow[tb] = (int32_t)ah[v];
      if (ta < T) { s1 += lo; s2 += (unsigned long long)lo * lo; }
      if (tb < T) { s1 += ah[v]; s2 += (unsigned long long)ah[v] * ah[v]; }
    }
    warp_sum_stats(s1, s2);
    if (lane == 0) part[(size_t)d * ntile + tile] = make_longlong2(s1, (long long)s2);
  }
}

// Stage 2 from int32 intermediates (plain layout, one output per load).
template <int Q>
__global__ void __launch_bounds__(kStage2MaxGroup * 32)
k_stage2_i32(const int32_t* __restrict__ P, int64_t Pp, const int32_t* __restrict__ e2, int ndm, int nsub,
             int G, int sc, int SW, int32_t* __restrict__ D, int64_t Dp, int64_t Td, int64_t T,
             longlong2* __restrict__ part, int ntile) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int V = 2 * Q / 32;
  const int tile = blockIdx.x, k = blockIdx.y;
  const int64_t t0 = (int64_t)tile * 2 * Q;
  const int dfirst = k * G;
  const int nd = min(G, ndm - dfirst);
  int32_t* emin = reinterpret_cast<int32_t*>(smem);
  int32_t* off = emin + nsub;
  int32_t* S = reinterpret_cast<int32_t*>(smem + (((size_t)nsub * (1 + kStage2MaxGroup) + 3) & ~(size_t)3));
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) emin[s] = e2[(size_t)dfirst * nsub + s];
  for (int i = threadIdx.x; i < nd * nsub; i += blockDim.x) {
    const int g = i / nsub, s = i - g * nsub;
    off[i] = e2[(size_t)(dfirst + g) * nsub + s] - e2[(size_t)dfirst * nsub + s];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0;
  for (int sb = 0; sb < nsub; sb += sc) {
    const int ns = min(sc, nsub - sb);
    for (int i = threadIdx.x; i < ns * SW; i += blockDim.x) {
      const int ss = i / SW, j = i - ss * SW;
      const int s = sb + ss;
      S[(size_t)ss * SW + j] = __ldg(P + ((size_t)k * nsub + s) * Pp + t0 + emin[s] + j);
    }
    __syncthreads();
    if (warp < nd) {
      const int32_t* o = off + warp * nsub + sb;
#pragma unroll 4
      for (int ss = 0; ss < ns; ++ss) {
        const int32_t* rw = S + (size_t)ss * SW + o[ss] + lane;
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
                        SnrConst* __restrict__ cst) {
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
    c.pad = 0.f;
    cst[(size_t)d * nw + w] = c;
  }
}

// ---------------------------------------------------------------------------
// boxcar matched filter (Eq. 5 via prefix sums, Sec. 2.4) and outputs (Sec. 2.5)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBoxThreads)
k_boxcar(const int32_t* __restrict__ D, int64_t Dp, int64_t T, int nw, const int32_t* __restrict__ widths,
         int wmax, const SnrConst* __restrict__ cst, int mode, float gamma, float* __restrict__ outf,
         uint8_t* __restrict__ outw, tx_cand* __restrict__ cands, unsigned long long* __restrict__ ncand,
         long long max_cands) {
  extern __shared__ __align__(16) uint32_t C[];
  __shared__ int32_t sw[kMaxWidths];
  __shared__ SnrConst sc[kMaxWidths];
  __shared__ uint32_t wsum[kBoxThreads / 32];
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kBoxTile;
  const int n = (int)min((int64_t)kBoxTile, T - t0);
  const int N = n + wmax - 1;
  if (threadIdx.x < nw) {
    sw[threadIdx.x] = widths[threadIdx.x];
    sc[threadIdx.x] = cst[(size_t)d * nw + threadIdx.x];
  }
  const int32_t* drow = D + (size_t)d * Dp + t0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) C[i + 1] = (uint32_t)__ldg(drow + i);
  if (threadIdx.x == 0) C[0] = 0u;
  __syncthreads();
  // inclusive scan of C[1..N] (uint32, wrap-around is harmless: window sums < 2^31)
  const int E = (N + blockDim.x - 1) / blockDim.x;
  const int beg = 1 + threadIdx.x * E, end = min(beg + E, N + 1);
  uint32_t local = 0;
  for (int i = beg; i < end; ++i) local += C[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    const uint32_t cl = C[i];
    float best = -INFINITY;
    int bw = 0;
    for (int w = 0; w < nw; ++w) {
      const uint32_t B = C[i + sw[w]] - cl;
      const float snr = ((float)((int32_t)B - sc[w].hi) - sc[w].lo) * sc[w].inv;
      if (mode == TX_OUT_CUBE) outf[((size_t)d * nw + w) * T + t0 + i] = snr;
      if (snr > best) {
        best = snr;
        bw = w;
      }
    }
    if (mode == TX_OUT_PLANE) {
      outf[(size_t)d * T + t0 + i] = best;
      outw[(size_t)d * T + t0 + i] = (uint8_t)bw;
    } else if (mode == TX_OUT_CANDS) {
      const bool hit = best >= gamma;
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

int stage1_smem(const tx_plan* p) { return p->m * (2 * p->q1 + 4) * 4 + kStage1MaxCoarse * p->m * 4; }

int stage2_smem(const tx_plan* p) {
  const int hdr = (int)(((size_t)p->nsub * (1 + kStage2MaxGroup) + 3) & ~(size_t)3) * 4;
  const int sw = p->interm == TX_INTERM_U16 ? ((kStage2Q + p->span2_max + 3) / 4 * 4 + 4)
                                            : (2 * kStage2Q + p->span2_max + 4);
  return hdr + p->nsub_chunk2 * sw * 4;
}

int stage2_sw(const tx_plan* p) {
  return p->interm == TX_INTERM_U16 ? ((kStage2Q + p->span2_max + 3) / 4 * 4 + 4) : (2 * kStage2Q + p->span2_max + 4);
}

int box_smem(const tx_plan* p) { return (kBoxTile + p->wmax + 4) * 4; }

template <int Q, typename PT>
int set_stage1_attr(int bytes) {
  TX_CUDA(cudaFuncSetAttribute(k_stage1<Q, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return TX_OK;
}

int do_upload(tx_plan* p) {
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  p->dev.device = dev;
  int rc;
  if ((rc = upload(&p->dev.d1, p->d1))) return rc;
  if ((rc = upload(&p->dev.abase, p->abase))) return rc;
  if ((rc = upload(&p->dev.e2, p->e2))) return rc;
  if ((rc = upload(&p->dev.widths, p->widths))) return rc;
  if ((rc = upload(&p->dev.items1, p->items1))) return rc;
  if ((rc = upload(&p->dev.span1, p->span1))) return rc;
  const int s1 = stage1_smem(p);
  const bool u16 = p->interm == TX_INTERM_U16;
  switch (p->q1) {
    case 256: rc = u16 ? set_stage1_attr<256, uint16_t>(s1) : set_stage1_attr<256, int32_t>(s1); break;
    case 128: rc = u16 ? set_stage1_attr<128, uint16_t>(s1) : set_stage1_attr<128, int32_t>(s1); break;
    case 64: rc = u16 ? set_stage1_attr<64, uint16_t>(s1) : set_stage1_attr<64, int32_t>(s1); break;
    default: rc = u16 ? set_stage1_attr<32, uint16_t>(s1) : set_stage1_attr<32, int32_t>(s1); break;
  }
  if (rc) return rc;
  const int s2 = stage2_smem(p);
  if (u16) TX_CUDA(cudaFuncSetAttribute(k_stage2_u16<kStage2Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2));
  else TX_CUDA(cudaFuncSetAttribute(k_stage2_i32<kStage2Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2));
  TX_CUDA(cudaFuncSetAttribute(k_boxcar, cudaFuncAttributeMaxDynamicSharedMemorySize, box_smem(p)));
  return TX_OK;
}

template <int Q, typename PT>
void launch_stage1(const tx_plan* p, const uint8_t* ring, void* P, cudaStream_t st) {
  k_stage1<Q, PT><<<(unsigned)p->items1.size(), kStage1Warps * 32, stage1_smem(p), st>>>(
      ring, p->Rp, p->ring_pad, p->dev.items1, p->dev.span1, p->dev.d1, p->nchan, p->m, p->nsub, p->dev.abase,
      reinterpret_cast<PT*>(P), p->Pp);
}

int check_beam(const tx_plan* p, const tx_beam* b) {
  if (!p || !b) { set_error("null plan or beam"); return TX_ERR_INVALID_ARG; }
  if (b->plan != p) { set_error("beam was created for another plan"); return TX_ERR_INVALID_ARG; }
  int dev = 0;
  TX_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) { set_error("beam lives on device %d, current device is %d", b->device, dev); return TX_ERR_INVALID_ARG; }
  return TX_OK;
}

// Writes a block (plan layout) of n samples into ring rows at byte offset off.
int ingest(const tx_plan* p, const uint8_t* src, int64_t n, uint8_t* ring, int64_t off, cudaStream_t st) {
  if (n <= 0) return TX_OK;
  if (p->layout == TX_LAYOUT_TF) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((p->nchan + 63) / 64));
    k_ingest_tf<<<grid, 256, 0, st>>>(src, n, p->nchan, ring, p->Rp, off);
  } else if (n % 16 == 0 && off % 16 == 0 && ((uintptr_t)src & 15) == 0) {
    const int64_t n16 = n / 16;
    dim3 grid((unsigned)std::min<int64_t>((n16 + 255) / 256, 64), (unsigned)p->nchan);
    k_ingest_ft16<<<grid, 256, 0, st>>>(reinterpret_cast<const uint4*>(src), n16, ring, p->Rp, off);
  } else {
    dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 256), (unsigned)p->nchan);
    k_ingest_ft<<<grid, 256, 0, st>>>(src, n, ring, p->Rp, off);
  }
  TX_CUDA(cudaGetLastError());
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
    cudaFree(p->dev.span1);
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
  const size_t rbytes = (size_t)p->nchan * p->Rp;
  cudaError_t e = cudaMalloc((void**)&b->ring[0], rbytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ring[1], rbytes);
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
  const size_t rbytes = (size_t)p->nchan * p->Rp;
  TX_CUDA(cudaMemsetAsync(b->ring[0], 0, rbytes, st));
  TX_CUDA(cudaMemsetAsync(b->ring[1], 0, rbytes, st));
  TX_CUDA(cudaMemsetAsync(b->run, 0, (size_t)p->ndm * 2 * sizeof(double), st));
  k_fill_run<<<(p->ndm + 255) / 256, 256, 0, st>>>(b->run, p->ndm);
  TX_CUDA(cudaGetLastError());
  b->cur = 0;
  b->nblocks = 0;
  return TX_OK;
}

int32_t tx_beam_prime(const tx_plan* p, tx_beam* b, const uint8_t* d_tail, void* stream) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!d_tail && p->L > 0) { set_error("null tail"); return TX_ERR_INVALID_ARG; }
  // the next execute copies logical [T, T + L) of the current ring
  return ingest(p, d_tail, p->L, b->ring[b->cur], p->ring_pad + p->T, (cudaStream_t)stream);
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
  const int64_t hdr[4] = {0x54584245414d31LL, p->nchan, p->L, b->nblocks};
  std::memcpy(h, hdr, sizeof(hdr));
  TX_CUDA(cudaDeviceSynchronize());
  if (p->L > 0)
    TX_CUDA(cudaMemcpy2D(h + 64, (size_t)p->L, b->ring[b->cur] + p->ring_pad + p->T, (size_t)p->Rp, (size_t)p->L,
                         (size_t)p->nchan, cudaMemcpyDeviceToHost));
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
  if (hdr[0] != 0x54584245414d31LL || hdr[1] != p->nchan || hdr[2] != p->L) { set_error("export does not match this plan"); return TX_ERR_INVALID_ARG; }
  TX_CUDA(cudaDeviceSynchronize());
  if (p->L > 0)
    TX_CUDA(cudaMemcpy2D(b->ring[b->cur] + p->ring_pad + p->T, (size_t)p->Rp, h + 64, (size_t)p->L, (size_t)p->L,
                         (size_t)p->nchan, cudaMemcpyHostToDevice));
  TX_CUDA(cudaMemcpy(b->run, h + 64 + (size_t)p->nchan * p->L, (size_t)p->ndm * 16, cudaMemcpyHostToDevice));
  b->nblocks = hdr[3];
  return TX_OK;
}

void tx_beam_destroy(tx_beam* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (b->device >= 0) cudaSetDevice(b->device);
  cudaFree(b->ring[0]);
  cudaFree(b->ring[1]);
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

  // Sec. 2.3 data flow: carried tail + new block -> next ring (steps 1, 2, 4)
  uint8_t* cur = b->ring[b->cur];
  uint8_t* nxt = b->ring[b->cur ^ 1];
  if (p->L > 0) {
    dim3 grid((unsigned)std::min<int64_t>((p->L + 255) / 256, 128), (unsigned)p->nchan);
    k_tail<<<grid, 256, 0, st>>>(cur, nxt, p->Rp, p->ring_pad + p->T, p->ring_pad, p->L);
    TX_CUDA(cudaGetLastError());
  }
  if ((rc = ingest(p, d_block, p->T, nxt, p->ring_pad + p->L, st))) return rc;
  b->cur ^= 1;
  TX_MARK(1);

  // stage 1
  void* P = ws + p->ws_P;
  const bool u16 = p->interm == TX_INTERM_U16;
  switch (p->q1) {
    case 256: u16 ? launch_stage1<256, uint16_t>(p, nxt, P, st) : launch_stage1<256, int32_t>(p, nxt, P, st); break;
    case 128: u16 ? launch_stage1<128, uint16_t>(p, nxt, P, st) : launch_stage1<128, int32_t>(p, nxt, P, st); break;
    case 64: u16 ? launch_stage1<64, uint16_t>(p, nxt, P, st) : launch_stage1<64, int32_t>(p, nxt, P, st); break;
    default: u16 ? launch_stage1<32, uint16_t>(p, nxt, P, st) : launch_stage1<32, int32_t>(p, nxt, P, st); break;
  }
  TX_CUDA(cudaGetLastError());
  TX_MARK(2);

  // stage 2 (+ exact per-tile sums)
  const bool series = p->output == TX_OUT_SERIES;
  int32_t* D = series ? static_cast<int32_t*>(d_out) : reinterpret_cast<int32_t*>(ws + p->ws_D);
  const int64_t Dp = series ? p->Td : p->Dp;
  longlong2* part = reinterpret_cast<longlong2*>(ws + p->ws_part);
  {
    dim3 grid((unsigned)p->ntile2, (unsigned)p->nk);
    const int threads = std::min(p->group, kStage2MaxGroup) * 32;
    if (u16)
      k_stage2_u16<kStage2Q><<<grid, threads, stage2_smem(p), st>>>(
          static_cast<const uint16_t*>(P), p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nsub_chunk2, stage2_sw(p),
          D, Dp, p->Td, p->T, part, p->ntile2);
    else
      k_stage2_i32<kStage2Q><<<grid, threads, stage2_smem(p), st>>>(
          static_cast<const int32_t*>(P), p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nsub_chunk2, stage2_sw(p),
          D, Dp, p->Td, p->T, part, p->ntile2);
    TX_CUDA(cudaGetLastError());
  }
  TX_MARK(3);

  if (!series) {
    SnrConst* cst = reinterpret_cast<SnrConst*>(ws + p->ws_const);
    k_stats<<<(p->ndm + 127) / 128, 128, 0, st>>>(part, p->ntile2, p->ndm, p->T, p->nw, p->dev.widths,
                                                  p->stats == TX_STATS_RUNNING, p->lambda, b->run, cst);
    TX_CUDA(cudaGetLastError());
    TX_MARK(4);
    if (p->output == TX_OUT_CANDS) TX_CUDA(cudaMemsetAsync(d_ncand, 0, sizeof(int64_t), st));
    float* outf = static_cast<float*>(d_out);
    uint8_t* outw = p->output == TX_OUT_PLANE ? static_cast<uint8_t*>(d_out) + (size_t)p->ndm * p->T * 4 : nullptr;
    dim3 grid((unsigned)p->ntile3, (unsigned)p->ndm);
    k_boxcar<<<grid, kBoxThreads, box_smem(p), st>>>(
        D, p->Dp, p->T, p->nw, p->dev.widths, p->wmax, cst, p->output, p->gamma, outf, outw,
        static_cast<tx_cand*>(d_out), reinterpret_cast<unsigned long long*>(d_ncand), (long long)p->max_cands);
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
