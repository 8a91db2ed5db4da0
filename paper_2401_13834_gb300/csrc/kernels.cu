// Single-beam host side of the library (sm_103a): plan upload, beams, the
// per-block execute (Sec. 2.3 data flow, then Sec. 2.4 and 2.5), phase
// timers, the host-buffer execute and the allocation-free de-dispersion. The
// kernels themselves are in kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
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

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <typename T>
int upload(T** dst, const std::vector<T>& v) {
  TX_CUDA(cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(T)));
  if (!v.empty()) TX_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TX_OK;
}

// 16-bit intermediates (uint16 or half) share the staging kernels
bool is16(const tx_plan* p) { return p->interm == TX_INTERM_U16 || p->interm == TX_INTERM_F16; }

int stage2_smem(const tx_plan* p) {
  if (p->pipe2) return (int)stage2_pipe_smem(p->nsub_chunk2, p->sww2);
  if (is16(p)) return stage2_u16_smem_for(p->nsub_chunk2 * p->sww2, p->nsub_chunk2, p->e2w2);
  return p->nsub_chunk2 * p->sw2_i32 * 4;
}

int box_smem(const tx_plan* p) { return box_smem_for(p->box_tile, p->wmax); }

template <int Q, typename PT, bool HALF = false>
int set_stage1_attr(int bytes) {
  TX_CUDA(raise_smem_limit((const void*)k_stage1<Q, PT, OneBeam, HALF>, bytes));
  return TX_OK;
}

template <int NW, int MAXWARPS, int SPLIT>
int set_stage2_attr(int bytes) {
  TX_CUDA(raise_smem_limit((const void*)k_stage2_u16<NW, MAXWARPS, SPLIT, OneBeam, false>, bytes));
  TX_CUDA(raise_smem_limit((const void*)k_stage2_u16<NW, MAXWARPS, SPLIT, OneBeam, true>, bytes));
  return TX_OK;
}

template <int Q>
int set_stage1_attr_for(const tx_plan* p, int bytes) {
  if (p->interm == TX_INTERM_F16) return set_stage1_attr<Q, uint16_t, true>(bytes);
  if (p->interm == TX_INTERM_U16) return set_stage1_attr<Q, uint16_t>(bytes);
  return set_stage1_attr<Q, int32_t>(bytes);
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
  if ((rc = upload(&p->dev.tab1, p->tab1))) return rc;
  if ((rc = upload(&p->dev.tab2, p->tab2))) return rc;
  if ((rc = upload(&p->dev.items_f, p->items_f))) return rc;
  const int s1 = (int)stage1_smem_bytes(p->m, p->q1);
  switch (p->q1) {
    case 256: rc = set_stage1_attr_for<256>(p, s1); break;
    case 128: rc = set_stage1_attr_for<128>(p, s1); break;
    case 64: rc = set_stage1_attr_for<64>(p, s1); break;
    default: rc = set_stage1_attr_for<32>(p, s1); break;
  }
  if (rc) return rc;
  const int s2 = stage2_smem(p);
  if (p->pipe2) {
    TX_CUDA(raise_smem_limit(stage2_pipe_kernel<OneBeam>(p->split2, p->interm == TX_INTERM_F16), s2));
  } else if (is16(p)) {
    switch (stage2_split(p)) {
      case 8: rc = set_stage2_attr<512, 32, 8>(s2); break;
      case 4: rc = set_stage2_attr<512, 32, 4>(s2); break;
      case 2: rc = set_stage2_attr<512, 32, 2>(s2); break;
      default: rc = set_stage2_attr<256, 32, 1>(s2); break;
    }
    if (rc) return rc;
  } else if (p->nw2 == 512) {
    TX_CUDA(raise_smem_limit((const void*)k_stage2_i32<512>, s2));
  } else {
    TX_CUDA(raise_smem_limit((const void*)k_stage2_i32<256>, s2));
  }
  if (p->output != TX_OUT_SERIES) {
    const BoxKernel<OneBeam> bk = box_kernel<OneBeam>(p->nw, p->output);
    TX_CUDA(raise_smem_limit((const void*)bk, box_smem(p)));
    TX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->dev.box_blocks_per_sm, bk, kBoxThreads, box_smem(p)));
  }
  p->dev.box_blocks_per_sm = std::max(p->dev.box_blocks_per_sm, 1);
  return TX_OK;
}

template <int Q, typename PT, bool HALF = false>
void launch_stage1_t(const tx_plan* p, const BeamArgs& a, int32_t* ictr, cudaStream_t st) {
  const int nitems = (int)p->items1.size();
  const int grid = std::min(nitems, std::max(p->dev.num_sms, 1));
  launch_pdl(k_stage1<Q, PT, OneBeam, HALF>, grid, kStage1Warps * 32, (size_t)stage1_smem_bytes(p->m, Q), st,
             OneBeam{a}, nullptr, nullptr, 1, nitems, p->m, 1u, ictr);
}

// stage 1 with its item counter `ictr` (zeroed before, by the ingest)
template <int Q>
int launch_stage1(const tx_plan* p, const BeamArgs& a, int32_t* ictr, cudaStream_t st) {
  if (p->interm == TX_INTERM_F16) launch_stage1_t<Q, uint16_t, true>(p, a, ictr, st);
  else if (p->interm == TX_INTERM_U16) launch_stage1_t<Q, uint16_t>(p, a, ictr, st);
  else launch_stage1_t<Q, int32_t>(p, a, ictr, st);
  return TX_OK;
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
// physical positions [pos, pos + n) mod R, splitting at the wrap; zeroes
// *zero on the way (when given).
int ingest(const tx_plan* p, const uint8_t* src, int64_t n, uint8_t* ring, int64_t pos, cudaStream_t st,
           int32_t* zero = nullptr) {
  if (n <= 0) return TX_OK;
  const int64_t R = p->R;
  int64_t done = 0;
  pos = mod(pos, R);
  while (done < n) {
    const int64_t len = std::min(n - done, R - pos);
    if (p->layout == TX_LAYOUT_TF) {
      const int vec = (p->nchan % 16 == 0) && (pos % 16 == 0) && (((uintptr_t)src & 15) == 0);
      dim3 grid((unsigned)((len + 64 * kIngestTiles - 1) / (64 * kIngestTiles)), (unsigned)((p->nchan + 63) / 64));
      TX_CUDA(launch_pdl(k_ingest_tf, grid, 256, 0, st, src, done, len, p->nchan, ring, R, pos, vec, zero));
    } else {
      const int vec = (n % 16 == 0) && (done % 16 == 0) && (len % 16 == 0) && (pos % 16 == 0) &&
                      (((uintptr_t)src & 15) == 0);
      dim3 grid((unsigned)std::min<int64_t>((len + 4095) / 4096, 64), (unsigned)p->nchan);
      TX_CUDA(launch_pdl(k_ingest_ft, grid, 256, 0, st, src, n, done, len, ring, R, pos, vec, zero));
    }
    TX_CUDA(cudaGetLastError());
    done += len;
    pos = 0;
  }
  return TX_OK;
}

// Copies the carried tail (the L samples before `head`, per channel; a
// compact beam's tail store) between the beam and a host buffer [nchan][L].
int copy_tail(const tx_plan* p, const tx_beam* b, uint8_t* host, bool to_host) {
  const int64_t L = p->L, R = p->R;
  if (L <= 0) return TX_OK;
  if (b->compact) {
    uint8_t* t = b->tail + p->tail_pad;
    const size_t pitch = (size_t)p->tail_pitch;
    if (to_host)
      TX_CUDA(cudaMemcpy2D(host, (size_t)L, t, pitch, (size_t)L, (size_t)p->nchan, cudaMemcpyDeviceToHost));
    else
      TX_CUDA(cudaMemcpy2D(t, pitch, host, (size_t)L, (size_t)L, (size_t)p->nchan, cudaMemcpyHostToDevice));
    return TX_OK;
  }
  const int64_t a = mod(b->head - L, R);
  const int64_t first = std::min(L, R - a);
  const size_t e = (size_t)p->esz;   // bytes per sample of the buffer (normalised floats on the float path)
  if (to_host) {
    TX_CUDA(cudaMemcpy2D(host, L * e, b->ring + a * e, R * e, first * e, (size_t)p->nchan, cudaMemcpyDeviceToHost));
    if (first < L)
      TX_CUDA(cudaMemcpy2D(host + first * e, L * e, b->ring, R * e, (L - first) * e, (size_t)p->nchan,
                           cudaMemcpyDeviceToHost));
  } else {
    TX_CUDA(cudaMemcpy2D(b->ring + a * e, R * e, host, L * e, first * e, (size_t)p->nchan, cudaMemcpyHostToDevice));
    if (first < L)
      TX_CUDA(cudaMemcpy2D(b->ring, R * e, host + first * e, L * e, (L - first) * e, (size_t)p->nchan,
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
    cudaFree(p->dev.tab1);
    cudaFree(p->dev.tab2);
    cudaFree(p->dev.items_f);
    cudaSetDevice(prev);
  }
  delete p;
}

}  // extern "C"

namespace {

int beam_create(const tx_plan* p, tx_beam** out, int compact) {
  if (!p || !out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  int rc = tx_upload_plan(p);
  if (rc) return rc;
  if (compact && p->norm != TX_NORM_NONE) { set_error("the float path (a normalisation) runs full beams only"); return TX_ERR_UNSUPPORTED; }
  tx_beam* b = new (std::nothrow) tx_beam();
  if (!b) { set_error("out of host memory"); return TX_ERR_OOM; }
  b->plan = p;
  b->compact = compact;
  cudaGetDevice(&b->device);
  cudaError_t e = compact ? cudaMalloc((void**)&b->tail, std::max<size_t>((size_t)p->nchan * p->tail_pitch, 16))
                          : cudaMalloc((void**)&b->ring, (size_t)p->nchan * p->R * p->esz);
  if (e == cudaSuccess && p->norm != TX_NORM_NONE) e = cudaMalloc((void**)&b->chan, (size_t)p->nchan * 24);
  // the running statistics, then the beam's count of waits its kernels gave up
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->run, (size_t)p->ndm * 2 * sizeof(double) + 16);
  if (e == cudaSuccess) b->fail = reinterpret_cast<int32_t*>(b->run + (size_t)p->ndm * 2);
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

}  // namespace

extern "C" {

int32_t tx_beam_create(const tx_plan* p, tx_beam** out) { return beam_create(p, out, 0); }

int32_t tx_beam_create_compact(const tx_plan* p, tx_beam** out) { return beam_create(p, out, 1); }

int32_t tx_beam_reset(const tx_plan* p, tx_beam* b, void* stream) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->compact)
    TX_CUDA(cudaMemsetAsync(b->tail, 0, (size_t)p->nchan * p->tail_pitch, st));
  else
    TX_CUDA(cudaMemsetAsync(b->ring, 0, (size_t)p->nchan * p->R * p->esz, st));
  TX_CUDA(cudaMemsetAsync(b->run, 0, (size_t)p->ndm * 2 * sizeof(double) + 16, st));
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
  if (b->compact) {
    if (p->L <= 0) return TX_OK;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* t = b->tail + p->tail_pad;
    if (p->layout == TX_LAYOUT_TF) {
      const int vec = (p->tail_pad % 16 == 0) && (p->nchan % 16 == 0) && (((uintptr_t)d_tail & 15) == 0);
      dim3 grid((unsigned)((p->L + 64 * kIngestTiles - 1) / (64 * kIngestTiles)), (unsigned)((p->nchan + 63) / 64));
      k_ingest_tf<<<grid, 256, 0, st>>>(d_tail, 0, p->L, p->nchan, b->tail, p->tail_pitch, p->tail_pad, vec,
                                        nullptr);
      TX_CUDA(cudaGetLastError());
    } else {
      TX_CUDA(cudaMemcpy2DAsync(t, (size_t)p->tail_pitch, d_tail, (size_t)p->L, (size_t)p->L, (size_t)p->nchan,
                                cudaMemcpyDeviceToDevice, st));
    }
    return TX_OK;
  }
  if (p->norm != TX_NORM_NONE) return float_prime(p, b, d_tail, stream);
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
  TX_CUDA(cudaMemcpy(h + 64 + (size_t)p->nchan * p->L * p->esz, b->run, (size_t)p->ndm * 16, cudaMemcpyDeviceToHost));
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
  TX_CUDA(cudaMemcpy(b->run, h + 64 + (size_t)p->nchan * p->L * p->esz, (size_t)p->ndm * 16, cudaMemcpyHostToDevice));
  TX_CUDA(cudaMemset(b->fail, 0, sizeof(int32_t)));   // an imported state is a valid one
  b->nblocks = hdr[3];
  return TX_OK;
}

int32_t tx_beam_failed(const tx_plan* p, const tx_beam* b, int64_t* count) {
  int rc = check_beam(p, b);
  if (rc) return rc;
  if (!count) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  TX_CUDA(cudaDeviceSynchronize());
  int32_t v = 0;
  TX_CUDA(cudaMemcpy(&v, b->fail, sizeof(v), cudaMemcpyDeviceToHost));
  *count = v;
  return TX_OK;
}

void tx_beam_destroy(tx_beam* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (b->device >= 0) cudaSetDevice(b->device);
  cudaFree(b->ring);
  cudaFree(b->tail);
  cudaFree(b->run);
  cudaFree(b->chan);
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
  if (((uintptr_t)d_workspace & 15) != 0) { set_error("d_workspace must be 16-byte aligned"); return TX_ERR_INVALID_ARG; }
  // the series are stored two outputs at a time (8-byte stores), the other outputs as 4-byte words
  if (((uintptr_t)d_out & (p->output == TX_OUT_SERIES ? 7 : 3)) != 0) {
    set_error("d_out must be %d-byte aligned", p->output == TX_OUT_SERIES ? 8 : 4);
    return TX_ERR_INVALID_ARG;
  }
  if ((rc = tx_upload_plan(p))) return rc;
  if (p->norm != TX_NORM_NONE) {   // the float path: normalisation, FP32 de-dispersion and boxcar
    rc = float_execute(p, b, d_block, d_out, d_ncand, d_workspace, stream, reinterpret_cast<void* const*>(ev));
    if (rc == TX_OK) ++b->nblocks;
    return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  TX_MARK(0);

  // Sec. 2.3 data flow: the block lands behind the carried tail (steps 1, 2, 4)
  const int64_t start = mod(b->head - p->L, p->R);
  const BeamArgs a = make_args(p, b, d_block, d_out, d_ncand, d_workspace, b->head, start);
  // the stage-1 item counter, zeroed by the ingest
  int32_t* ictr = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(d_workspace) + p->ws_ctr);
  if (b->compact) {
    // tail into the borrowed ring, the block behind it, the new tail back out
    const int nunits = p->nchan * (int)((p->tail_pitch + 4095) / 4096);
    const int tgrid = std::min(nunits, std::max(p->dev.num_sms, 1) * 8);
    if (nunits > 0) k_tail<OneBeam><<<tgrid, 256, 0, st>>>(OneBeam{a}, 0, nullptr, nullptr, 1, nunits);
    TX_CUDA(cudaGetLastError());
    if ((rc = ingest(p, d_block, p->T, a.ring, a.head, st, ictr))) return rc;
    if (nunits > 0) k_tail<OneBeam><<<tgrid, 256, 0, st>>>(OneBeam{a}, 1, nullptr, nullptr, 1, nunits);
    TX_CUDA(cudaGetLastError());
  } else {
    if ((rc = ingest(p, d_block, p->T, b->ring, b->head, st, ictr))) return rc;
    b->head = mod(b->head + p->T, p->R);
  }
  TX_MARK(1);

  // half intermediates: the per-sub-band offsets of this block
  const bool half = p->interm == TX_INTERM_F16;
  if (half) {
    TX_CUDA(cudaMemsetAsync(a.hoff, 0, (size_t)(p->nsub + 1) * 4, st));
    k_offsets<OneBeam><<<std::min(p->nchan, std::max(p->dev.num_sms, 1) * 8), 256, 0, st>>>(OneBeam{a}, nullptr,
                                                                                           nullptr, 1, p->nchan);
    TX_CUDA(cudaGetLastError());
  }

  // stage 1
  switch (p->q1) {
    case 256: rc = launch_stage1<256>(p, a, ictr, st); break;
    case 128: rc = launch_stage1<128>(p, a, ictr, st); break;
    case 64: rc = launch_stage1<64>(p, a, ictr, st); break;
    default: rc = launch_stage1<32>(p, a, ictr, st); break;
  }
  if (rc) return rc;
  TX_CUDA(cudaGetLastError());
  TX_MARK(2);

  // stage 2 (+ exact per-tile sums)
  const bool series = p->output == TX_OUT_SERIES;
  {
    if (p->pipe2) {
      const int nunits = p->nk * p->ntile2;
      launch_stage2_pipe<OneBeam>(p->split2, half, std::min(nunits, std::max(p->dev.num_sms, 1)), stage2_threads(p),
                                  stage2_smem(p), st, OneBeam{a}, nullptr, nullptr, 1, nunits, p->nsub_chunk2,
                                  p->nsub_chunk2 * p->sww2, true);
    } else if (is16(p)) {
      const int nunits = p->nk * p->ntile2;
      const int grid = std::min(nunits, std::max(p->dev.num_sms, 1));
      const int slot = p->nsub_chunk2 * p->sww2;
#define TX_S2(NW, SP)                                                                                          \
  do {                                                                                                         \
    launch_pdl(half ? k_stage2_u16<NW, 32, SP, OneBeam, true> : k_stage2_u16<NW, 32, SP, OneBeam, false>, grid,  \
               stage2_threads(p), (size_t)stage2_smem(p), st, OneBeam{a}, nullptr, nullptr, 1, nunits, slot,       \
               p->e2w2);                                                                                       \
  } while (0)
      switch (stage2_split(p)) {
        case 8: TX_S2(512, 8); break;
        case 4: TX_S2(512, 4); break;
        case 2: TX_S2(512, 2); break;
        default: TX_S2(256, 1); break;
      }
#undef TX_S2
    } else {
      const int threads = std::min(p->group, kStage2MaxGroup) * 32;
      dim3 grid((unsigned)p->ntile2, (unsigned)p->nk);
      const int32_t* P = static_cast<const int32_t*>(a.P);
      launch_pdl(p->nw2 == 512 ? k_stage2_i32<512> : k_stage2_i32<256>, grid, threads, (size_t)stage2_smem(p), st, P,
                 p->Pp, p->dev.e2, p->ndm, p->nsub, p->group, p->nsub_chunk2, p->sw2_i32, a.D, a.Dp, p->Td, p->T,
                 a.part, p->ntile2);
    }
    TX_CUDA(cudaGetLastError());
  }
  TX_MARK(3);

  if (!series) {
    TX_CUDA(launch_pdl(k_stats<OneBeam>, (p->ndm + 3) / 4, 128, 0, st, OneBeam{a}, nullptr, nullptr, 1, p->ndm));
    TX_CUDA(cudaGetLastError());
    TX_MARK(4);
    const int nunits = p->ndm * p->ntile3;   // k_stats zeroed the candidate counter
    const int grid = std::min(nunits, std::max(p->dev.num_sms, 1) * p->dev.box_blocks_per_sm);
    TX_CUDA(launch_pdl(box_kernel<OneBeam>(p->nw, p->output), grid, kBoxThreads, (size_t)box_smem(p), st, OneBeam{a},
                       nullptr, nullptr, 1, nunits, p->box_tile, p->wmax));
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
  int32_t failed = 0;
  TX_CUDA(cudaMemcpyAsync(&failed, b->fail, sizeof(failed), cudaMemcpyDeviceToHost, st));
  if (p->output == TX_OUT_CANDS) {
    TX_CUDA(cudaMemcpyAsync(h_ncand, d_ncand, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TX_CUDA(cudaStreamSynchronize(st));
    const int64_t n = std::min<int64_t>(*h_ncand, p->max_cands);
    if (n > 0) TX_CUDA(cudaMemcpyAsync(h_out, d_out, (size_t)n * sizeof(tx_cand), cudaMemcpyDeviceToHost, st));
    TX_CUDA(cudaStreamSynchronize(st));
    if (failed) { set_error("the beam's kernels gave up %d waits: results not valid (reset the beam)", failed); return TX_ERR_ABORTED; }
    if (*h_ncand > p->max_cands) { set_error("%lld candidates, capacity %lld", (long long)*h_ncand, (long long)p->max_cands); return TX_ERR_CAND_OVERFLOW; }
    return TX_OK;
  }
  TX_CUDA(cudaMemcpyAsync(h_out, d_out, (size_t)p->out_bytes, cudaMemcpyDeviceToHost, st));
  TX_CUDA(cudaStreamSynchronize(st));
  if (failed) { set_error("the beam's kernels gave up %d waits: results not valid (reset the beam)", failed); return TX_ERR_ABORTED; }
  return TX_OK;
}

}  // extern "C"

extern "C" {

int32_t tx_wait_timeouts(int64_t* count) {
  if (!count) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  int v = 0;
  TX_CUDA(cudaMemcpyFromSymbol(&v, g_tx_wait_timeouts, sizeof(int)));
  int64_t nb = 0;
  const int rc = batch_wait_timeouts(&nb);
  if (rc) return rc;
  *count = v + nb;
  return TX_OK;
}

}  // extern "C"

namespace {

// Shared-memory read bandwidth: every thread of a 1024-thread block reads
// 32-bit words of a 32 KB buffer, a warp 32 consecutive words (one 128-byte
// wavefront) per load, eight independent loads in flight per thread, for
// `iters` rounds, each round one row further on; the loads are volatile and
// their words are folded into a value that may be written out, so that none
// is dropped or merged. One block per SM.
constexpr int kProbeWords = 8192;   // 32 KB
__device__ uint32_t g_probe_sink[1024];

__global__ void __launch_bounds__(1024, 1) k_smem_probe(int iters) {
  __shared__ uint32_t buf[kProbeWords];
  for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x) buf[i] = (uint32_t)i * 2654435761u;
  __syncthreads();
  const uint32_t base = smem_addr(buf);
  uint32_t acc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  uint32_t off = (uint32_t)threadIdx.x;                  // word index of this thread's first load
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t v;
      const uint32_t w = (off + (uint32_t)k * 1024u) & (kProbeWords - 1);
      // volatile: every load is issued, none is merged with an earlier one
      asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + 4u * w));
      acc[k] ^= v;
    }
    off = (off + 32u) & (kProbeWords - 1);               // the next 32-word row of each warp
  }
  uint32_t r = 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) r += acc[k];
  if (r == 0x9e3779b9u) g_probe_sink[blockIdx.x & 1023] = r;   // rarely taken; keeps the loads live
}

}  // namespace

extern "C" {

int32_t tx_measure_smem_bandwidth(int32_t iters, double* h_bytes_per_s, void* stream) {
  if (!h_bytes_per_s || iters < 1 || iters > (1 << 20)) { set_error("need 1 <= iters <= 2^20 and an output"); return TX_ERR_INVALID_ARG; }
  int dev = 0, nsm = 0;
  TX_CUDA(cudaGetDevice(&dev));
  TX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TX_CUDA(cudaEventCreate(&e0));
  TX_CUDA(cudaEventCreate(&e1));
  float ms = 0.f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) k_smem_probe<<<nsm, 1024, 0, st>>>(iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) { set_error("shared-memory probe failed: %s", cudaGetErrorString(e)); return TX_ERR_CUDA; }
  *h_bytes_per_s = (double)nsm * 1024.0 * 8.0 * 4.0 * (double)iters / ((double)ms * 1e-3);
  return TX_OK;
}

int32_t tx_downsample(const uint8_t* d_in, int32_t layout, int32_t nchan, int64_t nsamp, int32_t factor,
                      uint8_t* d_out, void* stream) {
  if (!d_in || !d_out || nchan < 1 || nsamp < 1 || factor < 1 || factor > 1024 || (factor & (factor - 1))) {
    set_error("need device buffers, nchan >= 1, nsamp >= 1 and a power-of-two factor <= 1024");
    return TX_ERR_INVALID_ARG;
  }
  if (layout != TX_LAYOUT_FT && layout != TX_LAYOUT_TF) { set_error("bad layout"); return TX_ERR_INVALID_ARG; }
  if (nsamp % factor) { set_error("nsamp (%lld) is not a multiple of the factor %d", (long long)nsamp, factor); return TX_ERR_NOT_DIVISIBLE; }
  int dev = 0, nsm = 0;
  TX_CUDA(cudaGetDevice(&dev));
  TX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int vec = layout == TX_LAYOUT_TF && nchan % 4 == 0 && ((uintptr_t)d_in & 3) == 0 && ((uintptr_t)d_out & 3) == 0;
  const int64_t work = (nsamp / factor) * (vec ? nchan / 4 : nchan);
  const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)std::max(nsm, 1) * 16);
  k_downsample<<<std::max(grid, 1), 256, 0, (cudaStream_t)stream>>>(d_in, layout, nchan, nsamp, factor, vec, d_out);
  TX_CUDA(cudaGetLastError());
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
  if (((uintptr_t)d_series & 7) != 0) {  // the series are stored two outputs at a time
    set_error("d_series must be 8-byte aligned");
    return TX_ERR_INVALID_ARG;
  }
  // scratch layout: stage-1 work items, d1, abase, e2, stage-1 sums, per-tile sums
  const size_t b_items = align256(p->items1.size() * sizeof(Stage1Item));
  const size_t b_d1 = align256(p->d1.size() * 4);
  const size_t b_abase = align256(p->abase.size() * 4);
  const size_t b_e2 = align256(p->e2.size() * 4);
  const size_t b_P = align256((size_t)p->nk * p->nsub * p->Pp * 2);
  const size_t b_part = align256((size_t)p->ndm * p->ntile2 * (p->pipe2 ? p->split2 : 1) * 16);
  const size_t b_tab2 = align256(p->tab2.size() * 4);
  const size_t b_ctr = 256;   // the stage-1 item counter
  const size_t need = b_items + b_d1 + b_abase + b_e2 + b_P + b_part + b_tab2 + b_ctr;
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
  int32_t* tab2 = reinterpret_cast<int32_t*>(base + b_items + b_d1 + b_abase + b_e2 + b_P + b_part);
  int32_t* ictr = reinterpret_cast<int32_t*>(base + b_items + b_d1 + b_abase + b_e2 + b_P + b_part + b_tab2);
  cudaStream_t st = (cudaStream_t)stream;
  TX_CUDA(cudaMemcpyAsync(items, p->items1.data(), p->items1.size() * sizeof(Stage1Item), cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(d1, p->d1.data(), p->d1.size() * 4, cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(abase, p->abase.data(), p->abase.size() * 4, cudaMemcpyHostToDevice, st));
  TX_CUDA(cudaMemcpyAsync(e2, p->e2.data(), p->e2.size() * 4, cudaMemcpyHostToDevice, st));
  if (!p->tab2.empty())
    TX_CUDA(cudaMemcpyAsync(tab2, p->tab2.data(), p->tab2.size() * 4, cudaMemcpyHostToDevice, st));
  // Nothing in the scratch must start at zero: stage 1 writes every stage-1
  // sum that stage 2 reads, and stage 2 writes every per-tile sum.

  // the window as a beam: a linear buffer read as a ring of length ld, time 0 at 0
  BeamArgs a{};
  a.ring = const_cast<uint8_t*>(d_x);
  a.P = P;
  a.D = d_series;
  a.part = part;
  a.d1 = d1;
  a.abase = abase;
  a.e2 = e2;
  a.tab2 = tab2;
  a.items = items;
  a.R = ld;
  a.start = 0;
  a.T = p->T;
  a.Pp = p->Pp;
  a.Dp = p->Td;
  a.Td = p->Td;
  a.nchan = p->nchan;
  a.m = p->m;
  a.nsub = p->nsub;
  a.ndm = p->ndm;
  a.G = p->group;
  a.split2 = p->pipe2 ? p->split2 : 1;
  a.SC = p->nsub_chunk2;
  a.SWW = p->sww2;
  a.ntile2 = p->ntile2;
  a.polls = first_wait_polls();   // a wait that gives up counts in tx_wait_timeouts only

  // stage 1
  const int nitems = (int)p->items1.size();
  const int smem1 = (int)stage1_smem_bytes(p->m, p->q1);
  const int grid1 = std::min(nitems, std::max(nsm, 1));
  TX_CUDA(cudaMemsetAsync(ictr, 0, sizeof(int32_t), st));
#define TX_NA_S1(Q)                                                                                               \
  do {                                                                                                            \
    TX_CUDA(raise_smem_limit((const void*)k_stage1<Q, uint16_t, OneBeam>, smem1));                           \
    k_stage1<Q, uint16_t, OneBeam><<<grid1, kStage1Warps * 32, smem1, st>>>(OneBeam{a}, nullptr, nullptr, 1, nitems, \
                                                                            p->m, 1u, ictr);                  \
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
  const int slot = p->nsub_chunk2 * p->sww2;
  const int smem2 = p->pipe2 ? (int)stage2_pipe_smem(p->nsub_chunk2, p->sww2)
                             : stage2_u16_smem_for(slot, p->nsub_chunk2, p->e2w2);
  const int nunits = p->nk * p->ntile2;
  const int grid2 = std::min(nunits, std::max(nsm, 1));
  if (p->pipe2) {
    TX_CUDA(raise_smem_limit(stage2_pipe_kernel<OneBeam>(p->split2, false), smem2));
    launch_stage2_pipe<OneBeam>(p->split2, false, grid2, stage2_threads(p), smem2, st, OneBeam{a}, nullptr, nullptr, 1,
                                nunits, p->nsub_chunk2, slot);
    TX_CUDA(cudaGetLastError());
    return TX_OK;
  }
#define TX_NA_S2(NW, SP)                                                                                       \
  do {                                                                                                         \
    TX_CUDA(raise_smem_limit((const void*)k_stage2_u16<NW, 32, SP, OneBeam>, smem2));                          \
    k_stage2_u16<NW, 32, SP, OneBeam><<<grid2, stage2_threads(p), smem2, st>>>(OneBeam{a}, nullptr, nullptr, 1,   \
                                                                               nunits, slot, p->e2w2);           \
  } while (0)
  switch (stage2_split(p)) {
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
