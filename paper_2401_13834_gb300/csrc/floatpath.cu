// The float path (sm_103a): per-channel normalisation (Sec. 2.1) before the
// sub-band de-dispersion (Sec. 2.3) and the boxcar matched filter (Sec. 2.4,
// Eq. 5), for plans with a tx_norm mode.
//
// Per block of a beam:
//   k_chan_sums     exact sums of x and x^2 per channel over the block's T new samples
//   k_chan_weights  mu_c, sigma_c (population), weight w_c = 1/sigma_c or 1/sigma_c^2
//   k_norm_ingest   x' = (float(x) - mu_c) * w_c into the beam's float32 circular buffer
//                   behind the carried tail (which keeps its own block's normalisation)
//   k_stage1_f32    P[k][s][t] = sum_{c in s} x'[c][t + d1[k][c]]  (FP32, channels in order)
//   k_stage2_f32    D[d][t]    = sum_s P[k(d)][s][t + d2[d][s]]     (FP32, sub-bands in order),
//                   with per-tile sums of D and D^2 in double
//   k_stats_f32     mu_d, sigma_d of D over [0, T) in double (block or running)
//   k_boxcar_f32    compensated (TwoSum) prefix sums of D per tile as float (hi, lo) pairs,
//                   window sums B_W = C[t + W] - C[t], S/N = (B_W - W mu_d) / (sigma_d sqrt W)
// Every thread of the de-dispersion stages computes one output by reading its
// operands through the L1/L2 caches; the float path trades the integer path's
// packed sums for arithmetic on normalised data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

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

constexpr int kThreads = 256;
constexpr int kSumChunk = 4096;   // samples per block of the channel sums

// ---- channel statistics -----------------------------------------------------
// S[c] = (sum x, sum x^2) over samples t < n of channel c; block in the plan's
// layout (FT rows of `pitch` bytes, or TF rows of nchan bytes). Atomic integer
// adds: exact and order-free.
__global__ void __launch_bounds__(kThreads) k_chan_sums(const uint8_t* __restrict__ blk, int layout, int nchan,
                                                         int64_t n, int64_t pitch, unsigned long long* __restrict__ S) {
  const int64_t t0 = (int64_t)blockIdx.x * kSumChunk;
  const int64_t t1 = min(n, t0 + kSumChunk);
  unsigned long long s1 = 0, s2 = 0;
  if (layout == TX_LAYOUT_FT) {
    const int c = blockIdx.y;
    const uint8_t* row = blk + (int64_t)c * pitch;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += kThreads) {
      const unsigned x = row[t];
      s1 += x;
      s2 += x * x;
    }
    __shared__ unsigned long long r1[kThreads / 32], r2[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = s1; r2[threadIdx.x >> 5] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long a = 0, b = 0;
      for (int w = 0; w < kThreads / 32; ++w) { a += r1[w]; b += r2[w]; }
      atomicAdd(S + 2 * c, a);
      atomicAdd(S + 2 * c + 1, b);
    }
  } else {
    // one channel per thread, consecutive threads on consecutive channels
    const int c = blockIdx.y * kThreads + threadIdx.x;
    if (c >= nchan) return;
    for (int64_t t = t0; t < t1; ++t) {
      const unsigned x = blk[t * nchan + c];
      s1 += x;
      s2 += x * x;
    }
    atomicAdd(S + 2 * c, s1);
    atomicAdd(S + 2 * c + 1, s2);
  }
}

// (mu_c, w_c) as floats from the exact sums over n samples: mu = S1 / n,
// var = (n S2 - S1^2) / n^2 with an exact 128-bit numerator, sigma = sqrt(var),
// w = 1 / sigma (unit variance) or 1 / var (weights by the reciprocal of the
// variance), 0 when sigma = 0.
__global__ void k_chan_weights(const unsigned long long* __restrict__ S, int nchan, int64_t n, int norm,
                               float2* __restrict__ muw) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchan) return;
  const unsigned long long s1 = S[2 * c], s2 = S[2 * c + 1];
  const double mu = __ddiv_rn((double)s1, (double)n);
  const unsigned __int128 num = (unsigned __int128)(unsigned long long)n * s2 - (unsigned __int128)s1 * s1;
  const double hi = (double)(unsigned long long)(num >> 64), lo = (double)(unsigned long long)num;
  const double var = __ddiv_rn(__dadd_rn(__dmul_rn(hi, 18446744073709551616.0), lo), __dmul_rn((double)n, (double)n));
  double w = 0.0;
  if (var > 0.0) w = norm == TX_NORM_UNIT ? __ddiv_rn(1.0, sqrt(var)) : __ddiv_rn(1.0, var);
  muw[c] = make_float2(__double2float_rn(mu), __double2float_rn(w));
}

__device__ __forceinline__ float norm_sample(unsigned x, float2 mw) {
  return __fmul_rn(__fsub_rn((float)x, mw.x), mw.y);
}

// x' of samples t < n into ring[c][(pos0 + t) mod R]. FT: one channel row per
// blockIdx.y; TF: 64-time x 64-channel byte tiles transposed through shared memory.
__global__ void __launch_bounds__(kThreads) k_norm_ingest(const uint8_t* __restrict__ src, int layout, int nchan,
                                                           int64_t n, int64_t pitch, float* __restrict__ ring, int64_t R,
                                                           int64_t pos0, const float2* __restrict__ muw) {
  if (layout == TX_LAYOUT_FT) {
    const int c = blockIdx.y;
    const float2 mw = muw[c];
    const uint8_t* row = src + (int64_t)c * pitch;
    float* out = ring + (int64_t)c * R;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
      int64_t p = pos0 + t;
      if (p >= R) p -= R;
      out[p] = norm_sample(row[t], mw);
    }
    return;
  }
  __shared__ uint8_t tile[64][65];
  const int64_t t0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  for (int i = threadIdx.x; i < 64 * 64; i += kThreads) {
    const int tt = i >> 6, cc = i & 63;
    const int64_t t = t0 + tt;
    tile[tt][cc] = (t < n && c0 + cc < nchan) ? src[t * nchan + c0 + cc] : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 64; i += kThreads) {
    const int cc = i >> 6, tt = i & 63;          // consecutive threads: consecutive times of one channel
    const int c = c0 + cc;
    const int64_t t = t0 + tt;
    if (c >= nchan || t >= n) continue;
    int64_t p = pos0 + t;
    if (p >= R) p -= R;
    ring[(int64_t)c * R + p] = norm_sample(tile[tt][cc], muw[c]);
  }
}

// ---- de-dispersion ----------------------------------------------------------------
// One block per item (sub-band s, coarse DMs [kb, ke), absolute times
// [tau0, tau0 + tile)): every channel's window of x' (tile + spread samples
// from buffer position start + tau0 + d1[kb][c], mod R) is staged in shared
// memory once, then each warp sums coarse DMs of the item over the
// sub-band's channels in order, P[k][s][tau0 + j - abase[k][s]] = sum_c
// S[c][j + d1[k][c] - d1[kb][c]], VW = tile / 32 outputs per lane.
constexpr int kThreads1 = 1024;   // stage 1: a warp per coarse DM of an item (up to 32)

template <int VW>
__global__ void __launch_bounds__(kThreads1) k_stage1_f32(const float* __restrict__ ring, int64_t R, int64_t start,
                                                          const Stage1Item* __restrict__ items,
                                                          const int32_t* __restrict__ d1,
                                                          const int32_t* __restrict__ abase, int nchan, int m, int nsub,
                                                          int64_t Pp, int sw, float* __restrict__ P) {
  extern __shared__ float S[];   // [m][sw]
  const Stage1Item it = items[blockIdx.x];
  constexpr int tile = 32 * VW;
  const int n = tile + it.span;
  const int c0 = it.s * m;
  const int32_t* d1b = d1 + (size_t)it.kb * nchan + c0;
  // the windows: channel c from buffer position p0_c = (start + tau0 + d1[kb][c]) mod R on
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < m; c += kThreads1 / 32) {
    const int64_t p0 = (start + it.tau0 + d1b[c]) % R;
    const float* src = ring + (int64_t)(c0 + c) * R;
    for (int j = lane; j < n; j += 32) {
      int64_t p = p0 + j;
      if (p >= R) p -= R;
      S[c * sw + j] = __ldg(src + p);
    }
  }
  __syncthreads();
  for (int kk = warp; kk < it.ke - it.kb; kk += kThreads1 / 32) {
    const int k = it.kb + kk;
    const int32_t* d1k = d1 + (size_t)k * nchan + c0;
    float acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = 0.f;
    if (m <= 64) {
      // the DM's channel offsets held two per lane and broadcast by shuffles:
      // no global load between a channel's shared-memory loads
      const int oa = lane < m ? __ldg(d1k + lane) - __ldg(d1b + lane) : 0;
      const int ob = lane + 32 < m ? __ldg(d1k + lane + 32) - __ldg(d1b + lane + 32) : 0;
      for (int c = 0; c < m; ++c) {
        const int o = __shfl_sync(0xffffffffu, c < 32 ? oa : ob, c & 31);
        const float* row = S + c * sw + o + lane;
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] = __fadd_rn(acc[v], row[32 * v]);
      }
    } else {
      for (int c = 0; c < m; ++c) {
        const float* row = S + c * sw + (__ldg(d1k + c) - __ldg(d1b + c)) + lane;
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] = __fadd_rn(acc[v], row[32 * v]);
      }
    }
    const int64_t rel = (int64_t)it.tau0 - abase[(size_t)k * nsub + it.s];
    float* prow = P + ((size_t)k * nsub + it.s) * Pp;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const int64_t j = rel + lane + 32 * v;
      if (j >= 0 && j < Pp) prow[j] = acc[v];
    }
  }
}

// 4-byte global -> shared copy that completes asynchronously (cp.async)
__device__ __forceinline__ void cp_async4f(float* smem, const float* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem) : "memory");
}

// One block per (tile of 2 NW outputs, coarse group k), one warp per fine DM
// of the group: sub-band chunks of SC rows of P (the tile plus the group's
// delay spread) are staged in shared memory, two buffers deep (chunk c + 1's
// copies are in flight while chunk c is summed), and each warp sums its DM's
// shifted rows in sub-band order, V = 2 NW / 32 outputs per lane; then the
// tile's sums of D and D^2 over t < T in double to part[d][tile].
template <int NW>
__global__ void __launch_bounds__(kStage2MaxGroup * 32) k_stage2_f32(const float* __restrict__ P, int64_t Pp,
                                                                      const int32_t* __restrict__ e2, int ndm, int nsub,
                                                                      int G, int SC, int SW, float* __restrict__ D,
                                                                      int64_t Dp, int64_t Td, int64_t T,
                                                                      double2* __restrict__ part, int ntile) {
  extern __shared__ float Sf[];   // [2][SC][SW]
  constexpr int V = 2 * NW / 32;
  const int tile = blockIdx.x, k = blockIdx.y;
  const int64_t t0 = (int64_t)tile * 2 * NW;
  const int dfirst = k * G;
  const int nd = min(G, ndm - dfirst);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (nsub + SC - 1) / SC;
  // chunk c into buffer c & 1 (the group's first DM's delay is each row's start)
  auto stage = [&](int c) {
    const int sb = c * SC, ns = min(SC, nsub - sb);
    float* dst = Sf + (size_t)(c & 1) * SC * SW;
    for (int ss = 0; ss < ns; ++ss) {
      const int s = sb + ss;
      const float* src = P + ((size_t)k * nsub + s) * Pp + t0 + __ldg(e2 + (size_t)dfirst * nsub + s);
      for (int j = threadIdx.x; j < SW; j += blockDim.x) cp_async4f(dst + (size_t)ss * SW + j, src + j);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.f;
  stage(0);
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) {
      stage(c + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");   // chunk c has landed
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const int sb = c * SC, ns = min(SC, nsub - sb);
    const float* buf = Sf + (size_t)(c & 1) * SC * SW;
    if (warp < nd) {
      for (int ss = 0; ss < ns; ++ss) {
        const int s = sb + ss;
        const int o = __ldg(e2 + (size_t)(dfirst + warp) * nsub + s) - __ldg(e2 + (size_t)dfirst * nsub + s);
        const float* rw = buf + (size_t)ss * SW + o + lane;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = __fadd_rn(acc[v], rw[32 * v]);
      }
    }
    __syncthreads();   // every warp is done with buffer c & 1 before chunk c + 2 lands there
  }
  if (warp < nd) {
    const int d = dfirst + warp;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int64_t t = t0 + lane + 32 * v;
      if (t < Td) D[(size_t)d * Dp + t] = acc[v];
      if (t < T) { s1 += (double)acc[v]; s2 += (double)acc[v] * (double)acc[v]; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) part[(size_t)d * ntile + tile] = make_double2(s1, s2);
  }
}

// mu_d = sum D / T, var_d = sum D^2 / T - mu_d^2 (at least 0), or their running
// update; (mu_d, sigma_d) to ms[d].
__global__ void k_stats_f32(const double2* __restrict__ part, int ntile, int ndm, int64_t T, int running, double lam,
                            double* __restrict__ run, double2* __restrict__ ms) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndm) return;
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < ntile; ++i) {
    const double2 v = part[(size_t)d * ntile + i];
    s1 += v.x;
    s2 += v.y;
  }
  double mu = s1 / (double)T;
  double var = fmax(s2 / (double)T - mu * mu, 0.0);
  if (running) {
    double* r = run + (size_t)d * 2;
    if (r[1] < 0.0) {
      r[0] = mu;
      r[1] = var;
    } else {
      mu = (1.0 - lam) * r[0] + lam * mu;
      var = (1.0 - lam) * r[1] + lam * var;
      r[0] = mu;
      r[1] = var;
    }
  }
  ms[d] = make_double2(mu, sqrt(var));
}

// ---- boxcar (Eq. 5) -------------------------------------------------------------
// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (s, c) += x, compensated: s + c carries the running sum to about twice the
// float precision (TwoSum of s and x, the rounding error added into c).
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
  float e;
  two_sum(s, x, s, e);
  c = __fadd_rn(c, e);
}

// One block per unit (fine DM d, tile of kBoxTile outputs). The window
// D[t0 + i], i < N = n + W_max - 1, is turned into compensated prefix sums
// C[i] = (hi_i, lo_i), hi_i + lo_i = D[t0] + ... + D[t0 + i - 1] to about twice
// float precision (TwoSum at every add, also across threads and warps), so that
//   B_W[t] = (hi[t+W] - hi[t]) + (lo[t+W] - lo[t])
// takes FP32 operations only and each difference of two floats is rounded
// once, relative to itself. Eq. 5 then subtracts W mu_d as a float pair (from
// double) and scales by 1 / (sigma_d sqrt W): S/N = ((dhi - Wmu_hi) + (dlo -
// Wmu_lo)) * inv (0 when sigma_d = 0). Outputs as the integer path's.
__global__ void __launch_bounds__(kThreads) k_boxcar_f32(const float* __restrict__ D, int64_t Dp, int64_t T,
                                                          int tileL, int ntile3, const double2* __restrict__ ms,
                                                          const int32_t* __restrict__ widths, int nw, int wmax,
                                                          int mode, float gamma, float* __restrict__ outf,
                                                          uint8_t* __restrict__ outw, tx_cand* __restrict__ cands,
                                                          unsigned long long* __restrict__ ncand, int64_t max_cands) {
  extern __shared__ float2 H[];   // [tileL + wmax]: the window, then its prefix sums (hi, lo)
  __shared__ float2 wtot[kThreads / 32];
  __shared__ int32_t sW[kMaxWidths];
  __shared__ float sInv[kMaxWidths], sMh[kMaxWidths], sMl[kMaxWidths];
  const int unit = blockIdx.x;
  const int d = unit / ntile3, tile = unit - d * ntile3;
  const int64_t t0 = (int64_t)tile * tileL;
  const int n = (int)min((int64_t)tileL, T - t0);
  const int N = n + wmax - 1;
  const double2 m = ms[d];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < nw) {
    const int W = widths[threadIdx.x];
    const double wmu = (double)W * m.x;
    const float h = __double2float_rn(wmu);
    sW[threadIdx.x] = W;
    sMh[threadIdx.x] = h;
    sMl[threadIdx.x] = __double2float_rn(wmu - (double)h);
    sInv[threadIdx.x] = m.y > 0.0 ? __double2float_rn(1.0 / (m.y * sqrt((double)W))) : 0.f;
  }
  const float* row = D + (size_t)d * Dp + t0;
  for (int i = threadIdx.x; i < N; i += kThreads) H[i].x = row[i];
  __syncthreads();
  // exclusive compensated scan of H[0..N] in place (element N enters no used sum)
  const int E = (N + 1 + kThreads - 1) / kThreads;
  const int beg = threadIdx.x * E, end = min(beg + E, N + 1);
  float ls = 0.f, lc = 0.f;                                 // this thread's elements
  for (int i = beg; i < end && i < N; ++i) comp_add(ls, lc, H[i].x);
  float xs = ls, xc = lc;                                   // inclusive scan over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float ys = __shfl_up_sync(0xffffffffu, xs, o), yc = __shfl_up_sync(0xffffffffu, xc, o);
    if (lane >= o) {
      float e;
      two_sum(ys, xs, xs, e);
      xc = __fadd_rn(__fadd_rn(xc, yc), e);
    }
  }
  if (lane == 31) wtot[warp] = make_float2(xs, xc);
  // this thread's exclusive prefix within the warp: the inclusive one less its own part
  const float ps = __shfl_up_sync(0xffffffffu, xs, 1), pc = __shfl_up_sync(0xffffffffu, xc, 1);
  __syncthreads();
  float s = 0.f, c = 0.f;
  for (int w = 0; w < warp; ++w) {
    comp_add(s, c, wtot[w].x);
    c = __fadd_rn(c, wtot[w].y);
  }
  if (lane > 0) {
    comp_add(s, c, ps);
    c = __fadd_rn(c, pc);
  }
  for (int i = beg; i < end; ++i) {
    const float v = i < N ? H[i].x : 0.f;
    H[i] = make_float2(s, c);
    comp_add(s, c, v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const float2 c0 = H[i];
    float best = -INFINITY;
    int bw = 0;
    for (int w = 0; w < nw; ++w) {
      const float2 c1 = H[i + sW[w]];
      const float B = __fadd_rn(__fsub_rn(__fsub_rn(c1.x, c0.x), sMh[w]), __fsub_rn(__fsub_rn(c1.y, c0.y), sMl[w]));
      const float snr = __fmul_rn(B, sInv[w]);
      if (mode == TX_OUT_CUBE) outf[((size_t)d * nw + w) * T + t0 + i] = snr;
      if (snr > best) { best = snr; bw = w; }
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

inline int64_t mod(int64_t a, int64_t r) { return ((a % r) + r) % r; }

// Channel sums, weights and the normalised samples of n samples at ring
// position pos (src in the plan's layout, FT rows of `pitch` bytes).
int normalise_into(const tx_plan* p, const uint8_t* src, int64_t n, int64_t pitch, float* ring, int64_t pos,
                   unsigned long long* S, float2* muw, cudaStream_t st) {
  if (n <= 0) return TX_OK;
  TX_CUDA(cudaMemsetAsync(S, 0, (size_t)p->nchan * 16, st));
  const unsigned nchunk = (unsigned)((n + kSumChunk - 1) / kSumChunk);
  if (p->layout == TX_LAYOUT_FT)
    k_chan_sums<<<dim3(nchunk, (unsigned)p->nchan), kThreads, 0, st>>>(src, p->layout, p->nchan, n, pitch, S);
  else
    k_chan_sums<<<dim3(nchunk, (unsigned)((p->nchan + kThreads - 1) / kThreads)), kThreads, 0, st>>>(
        src, p->layout, p->nchan, n, pitch, S);
  TX_CUDA(cudaGetLastError());
  k_chan_weights<<<(p->nchan + 127) / 128, 128, 0, st>>>(S, p->nchan, n, p->norm, muw);
  TX_CUDA(cudaGetLastError());
  pos = mod(pos, p->R);
  if (p->layout == TX_LAYOUT_FT)
    k_norm_ingest<<<dim3((unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 64), (unsigned)p->nchan), kThreads,
                    0, st>>>(src, p->layout, p->nchan, n, pitch, ring, p->R, pos, muw);
  else
    k_norm_ingest<<<dim3((unsigned)((n + 63) / 64), (unsigned)((p->nchan + 63) / 64)), kThreads, 0, st>>>(
        src, p->layout, p->nchan, n, pitch, ring, p->R, pos, muw);
  TX_CUDA(cudaGetLastError());
  return TX_OK;
}

}  // namespace

int float_prime(const tx_plan* p, tx_beam* b, const uint8_t* d_tail, void* stream) {
  // the primed tail is normalised by its own statistics, as a block of L samples
  if (p->L <= 0) return TX_OK;
  const int64_t pitch = p->L;
  return normalise_into(p, d_tail, p->L, pitch, reinterpret_cast<float*>(b->ring), b->head - p->L,
                        reinterpret_cast<unsigned long long*>(b->chan),
                        reinterpret_cast<float2*>(b->chan + (size_t)p->nchan * 16), (cudaStream_t)stream);
}

int float_execute(const tx_plan* p, tx_beam* b, const uint8_t* d_block, void* d_out, int64_t* d_ncand,
                  void* d_workspace, void* stream, void* const* evp) {
  cudaStream_t st = (cudaStream_t)stream;
  const cudaEvent_t* ev = reinterpret_cast<const cudaEvent_t*>(evp);
  auto mark = [&](int i) -> int {
    if (ev) TX_CUDA(cudaEventRecord(ev[i], st));
    return TX_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  uint8_t* ws = static_cast<uint8_t*>(d_workspace);
  float* P = reinterpret_cast<float*>(ws + p->ws_P);
  const bool series = p->output == TX_OUT_SERIES;
  float* D = series ? static_cast<float*>(d_out) : reinterpret_cast<float*>(ws + p->ws_D);
  const int64_t Dp = series ? p->Td : p->Dp;
  double2* part = reinterpret_cast<double2*>(ws + p->ws_part);
  double2* ms = reinterpret_cast<double2*>(ws + p->ws_const);
  unsigned long long* S = reinterpret_cast<unsigned long long*>(ws + p->ws_hoff);
  float2* muw = reinterpret_cast<float2*>(ws + p->ws_hoff + (size_t)p->nchan * 16);
  float* ring = reinterpret_cast<float*>(b->ring);

  // Sec. 2.1 then Sec. 2.3 data flow: the block is normalised as it lands behind the tail
  const int64_t start = mod(b->head - p->L, p->R);
  if ((rc = normalise_into(p, d_block, p->T, p->T, ring, b->head, S, muw, st))) return rc;
  b->head = mod(b->head + p->T, p->R);
  if ((rc = mark(1))) return rc;

  // stage 1: the plan's items (sub-band, coarse DMs, time tile), one block each
  const int sw = p->tile_f + p->span_f + 4;
  const int smem1 = p->m * sw * (int)sizeof(float);
  const int nit = (int)p->items_f.size();
#define TX_F1(VW)                                                                                                  \
  do {                                                                                                             \
    TX_CUDA(cudaFuncSetAttribute((const void*)k_stage1_f32<VW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1)); \
    k_stage1_f32<VW><<<nit, kThreads1, smem1, st>>>(ring, p->R, start, p->dev.items_f, p->dev.d1, p->dev.abase,     \
                                                   p->nchan, p->m, p->nsub, p->Pp, sw, P);                          \
  } while (0)
  switch (p->tile_f) {
    case 256: TX_F1(8); break;
    case 128: TX_F1(4); break;
    case 64: TX_F1(2); break;
    default: TX_F1(1); break;
  }
#undef TX_F1
  TX_CUDA(cudaGetLastError());
  if ((rc = mark(2))) return rc;

  // stage 2 with per-tile sums
  const dim3 g2((unsigned)p->ntile2, (unsigned)p->nk);
  const int threads2 = std::min(p->group, kStage2MaxGroup) * 32;
  // two buffers of chunks, about 56 KB in all, so that four blocks share an SM
  const int sc2 = std::max(1, std::min(p->nsub_chunk2, (28 * 1024) / (p->sw2_i32 * (int)sizeof(float))));
  const int smem2 = 2 * sc2 * p->sw2_i32 * (int)sizeof(float);
#define TX_F2(NW)                                                                                                 \
  do {                                                                                                            \
    TX_CUDA(cudaFuncSetAttribute((const void*)k_stage2_f32<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2)); \
    k_stage2_f32<NW><<<g2, threads2, smem2, st>>>(P, p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, sc2,            \
                                                  p->sw2_i32, D, Dp, p->Td, p->T, part, p->ntile2);              \
  } while (0)
  if (p->nw2 == 512) TX_F2(512);
  else TX_F2(256);
#undef TX_F2
  TX_CUDA(cudaGetLastError());
  if ((rc = mark(3))) return rc;

  if (!series) {
    k_stats_f32<<<(p->ndm + 127) / 128, 128, 0, st>>>(part, p->ntile2f, p->ndm, p->T, p->stats == TX_STATS_RUNNING,
                                                      p->lambda, b->run, ms);
    TX_CUDA(cudaGetLastError());
    if ((rc = mark(4))) return rc;
    if (p->output == TX_OUT_CANDS) TX_CUDA(cudaMemsetAsync(d_ncand, 0, sizeof(int64_t), st));
    // units of the plan's boxcar length (the longest that still leaves a full
    // GPU several units per resident block)
    const int tile = p->box_tile;
    const int smem = (tile + p->wmax) * (int)sizeof(float2);
    // the most any plan needs (the attribute belongs to the current device)
    TX_CUDA(cudaFuncSetAttribute((const void*)k_boxcar_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (4 * kBoxTile + kMaxWidth) * (int)sizeof(float2)));
    float* outf = static_cast<float*>(d_out);
    uint8_t* outw = p->output == TX_OUT_PLANE ? static_cast<uint8_t*>(d_out) + (size_t)p->ndm * p->T * 4 : nullptr;
    const int nt = (int)((p->T + tile - 1) / tile);   // units per DM
    k_boxcar_f32<<<p->ndm * nt, kThreads, smem, st>>>(
        D, Dp, p->T, tile, nt, ms, p->dev.widths, p->nw, p->wmax, p->output, p->gamma, outf, outw,
        static_cast<tx_cand*>(d_out), reinterpret_cast<unsigned long long*>(d_ncand), p->max_cands);
    TX_CUDA(cudaGetLastError());
  } else {
    if ((rc = mark(4))) return rc;
  }
  return mark(5);
}
