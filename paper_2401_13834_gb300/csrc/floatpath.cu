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
//   k_boxcar_f32    prefix sums of D - mu_d in double per tile, held as float (hi, lo) pairs,
//                   window sums B_W = C[t + W] - C[t], S/N = B_W / (sigma_d sqrt W), outputs
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
// P[k][s][j] for row positions j of this block (absolute time abase[k][s] + j):
// the sum over the sub-band's channels, in order, of x' at buffer position
// start + abase + j + d1[k][c] (mod R).
__global__ void __launch_bounds__(kThreads) k_stage1_f32(const float* __restrict__ ring, int64_t R, int64_t start,
                                                          const int32_t* __restrict__ d1, const int32_t* __restrict__ abase,
                                                          int nchan, int m, int nsub, int64_t Pp, float* __restrict__ P) {
  extern __shared__ int64_t rowpos[];   // [m]: the buffer position of this block's first output per channel
  const int s = blockIdx.y, k = blockIdx.z;
  const int64_t j0 = (int64_t)blockIdx.x * kThreads;
  const int64_t ab = abase[(size_t)k * nsub + s];
  for (int i = threadIdx.x; i < m; i += kThreads)
    rowpos[i] = (start + ab + j0 + d1[(size_t)k * nchan + s * m + i]) % R;
  __syncthreads();
  const int64_t j = j0 + threadIdx.x;
  if (j >= Pp) return;
  float acc = 0.f;
  const float* base = ring + (int64_t)s * m * R;
  for (int i = 0; i < m; ++i) {
    int64_t p = rowpos[i] + threadIdx.x;
    if (p >= R) p -= R;
    acc = __fadd_rn(acc, __ldg(base + (int64_t)i * R + p));
  }
  P[((size_t)k * nsub + s) * Pp + j] = acc;
}

// D[d][t] = sum over sub-bands, in order, of P[k(d)][s][t + e2[d][s]] for
// t < Td; the block's sums of D and D^2 over t < T in double to part[d][tile].
__global__ void __launch_bounds__(kThreads) k_stage2_f32(const float* __restrict__ P, int64_t Pp,
                                                          const int32_t* __restrict__ e2, int nsub, int G,
                                                          float* __restrict__ D, int64_t Dp, int64_t Td, int64_t T,
                                                          double2* __restrict__ part, int ntile) {
  extern __shared__ int32_t erow[];     // [nsub]
  const int d = blockIdx.y, tile = blockIdx.x;
  const int k = d / G;
  for (int i = threadIdx.x; i < nsub; i += kThreads) erow[i] = e2[(size_t)d * nsub + i];
  __syncthreads();
  const int64_t t = (int64_t)tile * kFloatTile + threadIdx.x;
  double s1 = 0.0, s2 = 0.0;
  if (t < Td) {
    float acc = 0.f;
    const float* rows = P + (size_t)k * nsub * Pp + t;
    for (int s = 0; s < nsub; ++s) acc = __fadd_rn(acc, __ldg(rows + (size_t)s * Pp + erow[s]));
    D[(size_t)d * Dp + t] = acc;
    if (t < T) {
      s1 = (double)acc;
      s2 = __dmul_rn((double)acc, (double)acc);
    }
  }
  __shared__ double r1[kThreads / 32], r2[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = s1; r2[threadIdx.x >> 5] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { a += r1[w]; b += r2[w]; }
    part[(size_t)d * ntile + tile] = make_double2(a, b);
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
// One block per unit (fine DM d, tile of kBoxTile outputs). The window
// v_i = D[t0 + i] - mu_d (double), i < N = n + W_max - 1, is scanned in double
// into C[i] = v_0 + ... + v_{i-1}; each C is kept as a float pair hi + lo
// (hi = float(C), lo = float(C - hi)), so that a window sum
//   B_W[t] = (hi[t+W] - hi[t]) + (lo[t+W] - lo[t])
// takes FP32 operations only and keeps about double accuracy: each difference
// of two floats is rounded once, relative to itself. S/N = B_W / (sigma_d sqrt W)
// (0 when sigma_d = 0); outputs as the integer path's (cube / plane / candidates).
__global__ void __launch_bounds__(kThreads) k_boxcar_f32(const float* __restrict__ D, int64_t Dp, int64_t T,
                                                          int ntile3, const double2* __restrict__ ms,
                                                          const int32_t* __restrict__ widths, int nw, int wmax,
                                                          int mode, float gamma, float* __restrict__ outf,
                                                          uint8_t* __restrict__ outw, tx_cand* __restrict__ cands,
                                                          unsigned long long* __restrict__ ncand, int64_t max_cands) {
  extern __shared__ double C[];   // [kBoxTile + wmax]
  __shared__ double wsum[kThreads / 32];
  __shared__ int32_t sW[kMaxWidths];
  __shared__ float sInv[kMaxWidths];
  const int unit = blockIdx.x;
  const int d = unit / ntile3, tile = unit - d * ntile3;
  const int64_t t0 = (int64_t)tile * kBoxTile;
  const int n = (int)min((int64_t)kBoxTile, T - t0);
  const int N = n + wmax - 1;
  const double2 m = ms[d];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < nw) {
    const int W = widths[threadIdx.x];
    sW[threadIdx.x] = W;
    sInv[threadIdx.x] = m.y > 0.0 ? __double2float_rn(1.0 / (m.y * sqrt((double)W))) : 0.f;
  }
  const float* row = D + (size_t)d * Dp + t0;
  for (int i = threadIdx.x; i < N; i += kThreads) C[i] = (double)row[i] - m.x;
  __syncthreads();
  // exclusive scan of C[0..N] in place (C[N] enters no window sum that is used)
  const int E = (N + 1 + kThreads - 1) / kThreads;
  const int beg = threadIdx.x * E, end = min(beg + E, N + 1);
  double local = 0.0;
  for (int i = beg; i < end && i < N; ++i) local += C[i];
  double x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  double pre = x - local;
  for (int w = 0; w < warp; ++w) pre += wsum[w];
  float2* H = reinterpret_cast<float2*>(C);
  for (int i = beg; i < end; ++i) {
    const double v = i < N ? C[i] : 0.0;
    const float hi = __double2float_rn(pre);
    H[i] = make_float2(hi, __double2float_rn(pre - (double)hi));
    pre += v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const float2 c0 = H[i];
    float best = -INFINITY;
    int bw = 0;
    for (int w = 0; w < nw; ++w) {
      const float2 c1 = H[i + sW[w]];
      const float B = __fadd_rn(__fsub_rn(c1.x, c0.x), __fsub_rn(c1.y, c0.y));
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

  // stage 1: every row position of every (coarse DM, sub-band)
  const dim3 g1((unsigned)((p->Pp + kThreads - 1) / kThreads), (unsigned)p->nsub, (unsigned)p->nk);
  k_stage1_f32<<<g1, kThreads, (size_t)p->m * sizeof(int64_t), st>>>(ring, p->R, start, p->dev.d1, p->dev.abase,
                                                                      p->nchan, p->m, p->nsub, p->Pp, P);
  TX_CUDA(cudaGetLastError());
  if ((rc = mark(2))) return rc;

  // stage 2 with per-tile sums
  const dim3 g2((unsigned)p->ntile2f, (unsigned)p->ndm);
  k_stage2_f32<<<g2, kThreads, (size_t)p->nsub * sizeof(int32_t), st>>>(P, p->Pp, p->dev.e2, p->nsub, p->group, D, Dp,
                                                                         p->Td, p->T, part, p->ntile2f);
  TX_CUDA(cudaGetLastError());
  if ((rc = mark(3))) return rc;

  if (!series) {
    k_stats_f32<<<(p->ndm + 127) / 128, 128, 0, st>>>(part, p->ntile2f, p->ndm, p->T, p->stats == TX_STATS_RUNNING,
                                                      p->lambda, b->run, ms);
    TX_CUDA(cudaGetLastError());
    if ((rc = mark(4))) return rc;
    if (p->output == TX_OUT_CANDS) TX_CUDA(cudaMemsetAsync(d_ncand, 0, sizeof(int64_t), st));
    const int smem = (kBoxTile + p->wmax) * (int)sizeof(double);
    // the most any plan needs (the attribute belongs to the current device)
    TX_CUDA(cudaFuncSetAttribute((const void*)k_boxcar_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (kBoxTile + kMaxWidth) * (int)sizeof(double)));
    float* outf = static_cast<float*>(d_out);
    uint8_t* outw = p->output == TX_OUT_PLANE ? static_cast<uint8_t*>(d_out) + (size_t)p->ndm * p->T * 4 : nullptr;
    k_boxcar_f32<<<p->ndm * p->ntile3, kThreads, smem, st>>>(
        D, Dp, p->T, p->ntile3, ms, p->dev.widths, p->nw, p->wmax, p->output, p->gamma, outf, outw,
        static_cast<tx_cand*>(d_out), reinterpret_cast<unsigned long long*>(d_ncand), p->max_cands);
    TX_CUDA(cudaGetLastError());
  } else {
    if ((rc = mark(4))) return rc;
  }
  return mark(5);
}
