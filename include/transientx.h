/*
 * transientx.h -- C ABI of a GB300 (sm_103a) implementation of TransientX's
 * de-dispersion + matched-filter hot path (Men & Barr, arXiv 2401.13834).
 *
 * What the library computes, per block of T new samples of a beam:
 *
 *   1. Sub-band de-dispersion (Sec. 2.3, Fig. 3), with the cold-plasma delay
 *      of Eq. 1, tau = K DM (f^-2 - f_ref^-2), K = 4.148808e3 s MHz^2 pc^-1 cm^3:
 *        stage 1:  P[k][s][t] = sum_{c in s} X[c][t + d1[k][c]]
 *        stage 2:  D[d][t]    = sum_s     P[k(d)][s][t + d2[d][s]]
 *      d1 = rnd(K DM_k (f_c^-2 - f_ref,s^-2) / t_samp) at the coarse DM k of the
 *      trial's group, d2 = rnd(K DM_d (f_ref,s^-2 - f_ref^-2) / t_samp) at the fine
 *      DM; rnd rounds half away from zero; f_ref = highest channel centre,
 *      f_ref,s = highest centre in sub-band s; sub-band s = channels
 *      [s m, (s+1) m); fine DMs are grouped G at a time in order and a group's
 *      coarse DM is the midpoint of its first and last fine DM.
 *   2. Block statistics of each series over t in [0, T): exact integer sums,
 *      mean and population standard deviation (Sec. 2.4 takes sigma as the
 *      noise's spread; here that of the block's series), or their running
 *      (exponential) update across blocks.
 *   3. The boxcar matched filter of Eq. 5 computed by prefix sums (Sec. 2.4):
 *        S/N[d][w][t] = (sum_{i=t}^{t+W_w-1} D[d][i] - W_w mu_d) / (sigma_d sqrt(W_w))
 *      (window reported at its start t; sigma = 0 gives S/N = 0).
 *   4. Output: the S/N cube, the DM-time plane of the best width (Sec. 2.5;
 *      ties go to the smaller width), or the plane's points with
 *      S/N >= threshold as candidate records.
 *
 * Blocking (Sec. 2.3 data flow, steps 1-4): each beam keeps the last L samples
 * of every channel on the device (L = overlap = max over (d, c) of
 * d1 + d2 + W_max - 1). An execute appends the T new samples behind that tail,
 * computes outputs for buffer positions t in [0, T), and keeps the last L
 * samples as the next tail. Output t of block b therefore refers to stream
 * time b T - L + t at f_ref. A fresh beam's tail is zero; tx_beam_prime sets it.
 *
 * Conventions:
 *  - Every function returns an int status: TX_OK (0) or a negative TX_ERR_*.
 *    tx_last_error() gives a message for the calling thread's last failure.
 *  - Pointers named d_* are device pointers (cudaMalloc / PyTorch CUDA
 *    tensors); h_* are host pointers. The caller owns every buffer it passes.
 *    The library owns what a plan or beam allocates and frees it in
 *    tx_plan_destroy / tx_beam_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Device calls only enqueue work; nothing synchronises unless a
 *    function says so.
 *  - Distinct beams may be used from distinct threads concurrently. One beam
 *    must not be used by two calls at once.
 */
#ifndef TRANSIENTX_H
#define TRANSIENTX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TX_OK                  0
#define TX_ERR_INVALID_ARG    -1  /* a pointer, size or enum out of range            */
#define TX_ERR_NOT_DIVISIBLE  -2  /* nchan is not a multiple of nsub                  */
#define TX_ERR_OOM            -3  /* a device or host allocation failed               */
#define TX_ERR_CUDA           -4  /* a CUDA call failed (message in tx_last_error)    */
#define TX_ERR_TIMEOUT        -5  /* a bounded wait ran out                           */
#define TX_ERR_CAND_OVERFLOW  -6  /* more candidates than max_cands (results kept)    */
#define TX_ERR_BUDGET         -7  /* an allocation would exceed a caller's budget     */
#define TX_ERR_UNSUPPORTED    -8  /* valid but not supported by this build            */
#define TX_ERR_ABORTED        -9  /* a kernel gave up a bounded wait: the beam's
                                     results and state are not valid (see
                                     tx_beam_failed)                                 */

/* ---- enums ---- */
enum tx_layout { TX_LAYOUT_FT = 0,   /* block is channel-major  uint8 [nchan][T]      */
                 TX_LAYOUT_TF = 1 }; /* block is time-major     uint8 [T][nchan]
                                        (filterbank order; transposed on ingest,
                                        Sec. 2.3 data-flow step 2)                   */
enum tx_interm { TX_INTERM_U16 = 0,  /* stage-1 sums stored as uint16 (exact for
                                        nchan/nsub <= 257)                          */
                 TX_INTERM_I32 = 1,  /* stored as int32                              */
                 TX_INTERM_F16 = 2,  /* stored as FP16 after subtracting an integer
                                        offset per sub-band (the sum of its channels'
                                        rounded block means), rounded to nearest even
                                        and saturated at +-65504; stage 2 sums the
                                        halves in FP32 and adds the offsets back.
                                        Exact while |sum - offset| <= 2048.         */
                 TX_INTERM_F32 = 3 };/* the float path (normalised data, tx_norm):
                                        FP32 sums stored as FP32                     */
/* Per-channel normalisation (Sec. 2.1): each block is brought to zero mean and
   unit variance per channel as it arrives, x' = (x - mu_c) / sigma_c, with mu_c
   and sigma_c the mean and population standard deviation of channel c over the
   block's T new samples (exact integer sums); TX_NORM_INVVAR weights by the
   reciprocal of the variance instead, x' = (x - mu_c) / sigma_c^2, which
   down-weights noisy channels further. A channel with sigma_c = 0 gets weight
   0. The carried tail keeps the normalisation of the block it arrived with.
   x' is computed in FP32 as (float(x) - float(mu_c)) * float(w_c), w_c = 1 /
   sigma_c or 1 / sigma_c^2 rounded from double, and kept in a float32 buffer. */
enum tx_norm   { TX_NORM_NONE   = 0,  /* raw uint8, equal weights: the integer path  */
                 TX_NORM_UNIT   = 1,  /* zero mean, unit variance per channel        */
                 TX_NORM_INVVAR = 2 };/* zero mean, weight 1 / variance              */
enum tx_output { TX_OUT_CANDS  = 0,  /* tx_cand records, S/N >= snr_threshold        */
                 TX_OUT_PLANE  = 1,  /* float32 [ndm][T] best S/N, then uint8 [ndm][T]
                                        index of the best width                      */
                 TX_OUT_CUBE   = 2,  /* float32 [ndm][nwidth][T]                     */
                 TX_OUT_SERIES = 3 };/* int32 [ndm][T + W_max - 1] de-dispersed series
                                        (no matched filter); float32 on the float
                                        path                                         */
enum tx_stats  { TX_STATS_BLOCK   = 0,  /* mu, sigma of this block                   */
                 TX_STATS_RUNNING = 1 };/* mu, var <- (1-l) prev + l block; the first
                                          block after create/reset initialises      */

/* ---- plan description (all host pointers; copied by tx_plan_create) ---- */
typedef struct tx_plan_desc {
  int32_t        nchan;          /* channels, >= 1                                  */
  const double*  freq_mhz;       /* [nchan] channel centre frequencies, MHz, > 0,
                                    any order (sub-bands are index ranges)          */
  double         tsamp_s;        /* sampling time, s, > 0                           */
  int32_t        ndm;            /* fine DM trials, >= 1                            */
  const double*  dm;             /* [ndm] ascending (non-decreasing), >= 0          */
  int32_t        nsub;           /* sub-bands, divides nchan; nchan/nsub <= 257     */
  int32_t        group;          /* fine DMs per coarse DM, 0 = automatic rule      */
  int32_t        nwidth;         /* boxcar widths, 1..32                            */
  const int32_t* widths;         /* [nwidth] strictly ascending, 1..4096 samples    */
  int64_t        nsamp;          /* T, new samples per block, >= 1                  */
  int32_t        layout;         /* enum tx_layout of blocks passed to execute      */
  int32_t        interm;         /* enum tx_interm                                  */
  int32_t        output;         /* enum tx_output                                  */
  float          snr_threshold;  /* gamma for TX_OUT_CANDS (inclusive)              */
  int64_t        max_cands;      /* capacity of the candidate buffer, >= 1          */
  int32_t        stats;          /* enum tx_stats                                   */
  double         stats_lambda;   /* weight of a new block in TX_STATS_RUNNING, (0,1]*/
  /* Tile shapes (results do not depend on them; 0 = automatic choice):     */
  int32_t        tile_q1;        /* stage-1 tile of 4 * tile_q1 samples: 32, 64, 128
                                    or 256 (must fit shared memory); 0 = the
                                    largest that fits                               */
  int32_t        tile_split2;    /* stage-2 warps per fine DM: 1 (tiles of 512
                                    outputs) or 2, 4, 8 (tiles of 1024), with
                                    min(group, 32) * tile_split2 <= 32; 0 = 8, 4, 2
                                    or 1 for groups of <= 4, 8, 16 or more; used by
                                    groups of more than 16 DMs (smaller groups run
                                    the pipelined stage 2, which sizes itself)   */
  int32_t        norm;           /* enum tx_norm; TX_NORM_NONE unless interm is
                                    TX_INTERM_F32, which needs another mode. The
                                    float path runs single beams (tx_execute,
                                    tx_execute_host, pipelines); it is not taken by
                                    compact beams, batches or tx_dedisperse_noalloc */
  int32_t        tile_box;       /* boxcar outputs per work unit: 2048, 4096 or 8192;
                                    0 = the longest that leaves at least 4864
                                    (DM, unit) pairs (results do not depend on it) */
} tx_plan_desc;

typedef struct tx_plan_info {
  int32_t nchan, nsub, ndm, ncoarse, group, nwidth, wmax;
  int32_t tile_box;         /* the boxcar unit chosen (see tx_plan_desc)            */
  int64_t nsamp;            /* T                                                    */
  int64_t overlap;          /* L: carried samples per channel                       */
  int64_t max_delay;        /* max over (d, c) of d1 + d2                           */
  int64_t series_len;       /* T + W_max - 1                                        */
  int64_t workspace_bytes;  /* device scratch an execute needs (d_workspace)        */
  int64_t beam_state_bytes; /* device memory one beam holds                         */
  int64_t out_bytes;        /* size of d_out for the plan's output mode             */
  int64_t export_bytes;     /* host bytes for tx_beam_export / import               */
  int64_t block_bytes;      /* nchan * T, bytes of one input block                  */
  int64_t ring_len;         /* samples per channel of a beam's circular buffer (>= L + T);
                               a block that wraps its end is ingested in two launches */
  int64_t ring_head0;       /* where a fresh beam's first block lands in it        */
  int32_t tile_q1;          /* the stage-1 tile chosen (see tx_plan_desc)           */
  int32_t tile_split2;      /* the stage-2 warps per fine DM chosen                 */
  int64_t workspace_bytes_compact;   /* d_workspace of an execute on a compact beam */
  int64_t compact_beam_state_bytes;  /* device memory one compact beam holds        */
} tx_plan_info;

/* One candidate of TX_OUT_CANDS: a DM-time plane point with S/N >= threshold. */
typedef struct tx_cand {
  int32_t dm_index;   /* fine DM trial                                              */
  int32_t t;          /* output position in [0, T) (window start)                   */
  int32_t w_index;    /* index into widths of the best width                        */
  float   snr;        /* its S/N                                                    */
} tx_cand;

typedef struct tx_plan tx_plan;
typedef struct tx_beam tx_beam;

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t tx_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated to
   `size`) into `buf`; returns the message length. */
int32_t tx_last_error(char* buf, size_t size);

/* Builds a plan on the host: delay tables (Eq. 1 in double, rounded half away
   from zero), coarse grouping, overlap, kernel work lists. No GPU is touched.
   Errors: INVALID_ARG, NOT_DIVISIBLE, OOM. */
int32_t tx_plan_create(const tx_plan_desc* desc, tx_plan** out);

/* Sizes and shape of a plan. */
int32_t tx_plan_get_info(const tx_plan* plan, tx_plan_info* info);

/* Host copies of the plan's tables (any pointer may be NULL to skip it):
     d1             int32 [ncoarse][nchan]  stage-1 delays (samples)
     d2             int32 [ndm][nsub]       stage-2 delays (samples)
     coarse_of_fine int32 [ndm]             group index k(d)
     coarse_dm      double [ncoarse]        coarse DMs
   These follow Eq. 1 and the sub-band scheme of Sec. 2.3. */
int32_t tx_plan_tables(const tx_plan* plan, int32_t* d1, int32_t* d2,
                       int32_t* coarse_of_fine, double* coarse_dm);

/* Geometric boxcar ladder (Sec. 2.4: each width a fixed multiple of the one
   before, the multiple set by the caller): w_i = floor(ratio^i + 0.5),
   duplicates dropped, w_i <= wmax.
   Writes at most `cap` widths to h_widths; returns the count (or an error). */
int32_t tx_geometric_widths(double ratio, int32_t wmax, int32_t* h_widths, int32_t cap);

/* Layout of the stage-1 intermediate inside d_workspace (for parity checks):
     *p_offset  byte offset of P in the workspace
     *p_pitch   elements per (k, s) row
     h_base     int32 [ncoarse][nsub] (may be NULL): row (k, s) holds the stage-1
                sum at times h_base[k][s] + j, j in [0, p_pitch)
   P rows are uint16 or int32 per the plan's interm, row index k * nsub + s. */
int32_t tx_plan_stage1_layout(const tx_plan* plan, int64_t* p_offset, int64_t* p_pitch,
                              int32_t* h_base);

void tx_plan_destroy(tx_plan* plan);

/* Allocates a beam's device state (two channel-major rings of L + T samples per
   channel, running statistics) on the current CUDA device and zeroes it.
   Synchronous. Errors: INVALID_ARG, OOM, CUDA. */
int32_t tx_beam_create(const tx_plan* plan, tx_beam** out);

/* A compact beam keeps only the carried tail (nchan * L bytes) and the
   running statistics resident; each execute borrows its circular buffer
   from the workspace (info.workspace_bytes_compact instead of
   info.workspace_bytes), copying the tail in before the block lands and the
   new tail out after. The results are those of a full beam; the cost is two
   copies of the tail per block. Everything else that takes a beam takes a
   compact one. Errors as tx_beam_create. */
int32_t tx_beam_create_compact(const tx_plan* plan, tx_beam** out);

/* Zeroes the carried tail and the running statistics (enqueued on `stream`). */
int32_t tx_beam_reset(const tx_plan* plan, tx_beam* beam, void* stream);

/* Sets the carried tail to L given samples, d_tail in the plan's layout:
   uint8 [nchan][L] (FT) or [L][nchan] (TF). Enqueued on `stream`. */
int32_t tx_beam_prime(const tx_plan* plan, tx_beam* beam, const uint8_t* d_tail, void* stream);

/* Checkpoint: copies the carried tail, running statistics and block counter to
   host memory of info.export_bytes bytes (synchronous), and back. Resuming from
   an export reproduces the uninterrupted outputs exactly. */
int32_t tx_beam_export(const tx_plan* plan, const tx_beam* beam, void* h_dst, int64_t bytes);
int32_t tx_beam_import(const tx_plan* plan, tx_beam* beam, const void* h_src, int64_t bytes);

/* Blocks processed since create/reset/import. */
int32_t tx_beam_blocks(const tx_beam* beam, int64_t* nblocks);

/* Waits the beam's kernels gave up since create/reset/import (a bulk copy
   into shared memory that had not completed after the polling limit; see
   tx_set_wait_polls). A kernel that gives up returns early, so once this is
   nonzero every result since the last check is not valid, and neither is the
   beam's state (carried tail, running statistics): reset or import it before
   going on. The host-synchronous calls (tx_execute_host, tx_pipeline_pop,
   tx_batch_wait) check it and return TX_ERR_ABORTED. Waits for the device
   (cudaDeviceSynchronize), then reads the count into *count. */
int32_t tx_beam_failed(const tx_plan* plan, const tx_beam* beam, int64_t* count);

void tx_beam_destroy(tx_beam* beam);

/* Processes one block (Sec. 2.3 data flow, then Sec. 2.4 and 2.5):
     d_block     uint8, nchan * T bytes in the plan's layout
     d_out       info.out_bytes bytes; format set by the plan's output mode;
                 8-byte aligned for TX_OUT_SERIES, 4-byte aligned otherwise
     d_ncand     int64 [1], TX_OUT_CANDS only (else may be NULL): set to the number
                 of candidates found; records beyond max_cands are dropped, so a
                 value above max_cands means the buffer overflowed
     d_workspace info.workspace_bytes bytes of device scratch (not kept),
                 16-byte aligned; info.workspace_bytes_compact for a compact beam
   All kernels go on `stream`; the call returns once they are enqueued. They
   are launched with programmatic stream serialization: each one may begin
   launching while the kernel before it in `stream` is finishing, and waits
   for that kernel (and so for everything enqueued before it) before it
   touches memory; ordering against other work on `stream` is unchanged.
   A workspace must not be shared by executes that can run at the same time
   (it holds their sums and a work counter).
   Errors: INVALID_ARG (null or misaligned buffer, beam of another plan or
   device) before anything is enqueued, CUDA. */
int32_t tx_execute(const tx_plan* plan, tx_beam* beam, const uint8_t* d_block, void* d_out,
                   int64_t* d_ncand, void* d_workspace, void* stream);

/* tx_execute from and to host memory: copies h_block (nchan * T bytes, the
   plan's layout; pinned memory for full speed) to d_block_staging, executes,
   and copies the result back, then synchronises `stream`:
     TX_OUT_CANDS: *h_ncand and min(*h_ncand, max_cands) records to h_out
     other modes:  info.out_bytes bytes to h_out
   d_block_staging / d_out / d_ncand / d_workspace are device scratch as in
   tx_execute. Returns TX_ERR_CAND_OVERFLOW (results kept) if candidates were
   dropped, TX_ERR_ABORTED if the beam's kernels have given up a wait (see
   tx_beam_failed). */
int32_t tx_execute_host(const tx_plan* plan, tx_beam* beam, const uint8_t* h_block,
                        void* h_out, int64_t* h_ncand, uint8_t* d_block_staging, void* d_out,
                        int64_t* d_ncand, void* d_workspace, void* stream);

/* ---- pipelined host execution (Sec. 2.3 block flow, overlapped) -------------
   A stream of one beam's blocks from host memory with up to `depth` (1..4)
   blocks in flight: tx_pipeline_push copies a block into one of `depth`
   device staging buffers on a copy stream of the pipeline's own and enqueues
   its tx_execute on `stream` behind that copy; tx_pipeline_pop waits for the
   oldest block pushed and copies its results back on a second copy stream.
   Block k's kernels thus overlap block k + 1's host-to-device copy and block
   k - 1's results, and a steady stream runs at the kernels' rate when the
   copies are shorter than the kernels. The pipeline owns its staging, output,
   counter and workspace buffers (device, about depth * (nchan * T +
   info.out_bytes) bytes plus one workspace) and its copy streams; plan and
   beam remain the caller's and must outlive it. One thread at a time. */
typedef struct tx_pipeline tx_pipeline;

/* The beam must belong to `plan` and live on the current device. */
int32_t tx_pipeline_create(const tx_plan* plan, tx_beam* beam, int32_t depth, void* stream,
                           tx_pipeline** out);

/* Enqueues one block: h_block is nchan * T bytes in the plan's layout (pinned
   host memory for an asynchronous copy), left unchanged by the caller until
   the block's pop returns. Returns TX_ERR_BUDGET when `depth` blocks are in
   flight already (pop first); on an error nothing is enqueued. */
int32_t tx_pipeline_push(tx_pipeline* pipeline, const uint8_t* h_block);

/* Waits, polling, at most timeout_us microseconds (< 0: no limit) for the
   oldest block in flight and copies its results to host memory:
     TX_OUT_CANDS: *h_ncand and min(*h_ncand, max_cands) records to h_out
     other modes:  info.out_bytes bytes to h_out
   Returns TX_ERR_TIMEOUT when the limit ran out first (the block stays in
   flight: pop again), TX_ERR_INVALID_ARG when no block is in flight, and
   TX_ERR_CAND_OVERFLOW (results kept, block popped) and TX_ERR_ABORTED (block
   popped, results not valid) as tx_execute_host. */
int32_t tx_pipeline_pop(tx_pipeline* pipeline, void* h_out, int64_t* h_ncand, int64_t timeout_us);

/* Waits for the blocks in flight, then frees everything the pipeline owns. */
void tx_pipeline_destroy(tx_pipeline* pipeline);

/* Waits that the library's kernels gave up on the current device since the
   library was loaded: a bulk copy into shared memory that had not completed
   after the kernel's polling limit (seconds). The kernel that saw one
   returned early and the results of that launch are not valid; 0 in normal
   operation. Synchronises with the device. */
int32_t tx_wait_timeouts(int64_t* count);

/* Sets the polling limit of the first wait for each bulk copy in kernels
   launched from now on (process-wide; default and maximum 2^22 polls, which
   is seconds). With 0 every such wait gives up at once, which drives the
   failure path (tx_beam_failed, TX_ERR_ABORTED, tx_wait_timeouts) without
   any fault: for tests only. Whatever the setting, a kernel that gives up
   waits at the full limit for the copies it has in flight before it returns.
   The previous limit goes to *previous (may be NULL). */
int32_t tx_set_wait_polls(int64_t polls, int64_t* previous);

/* Measures the shared-memory read bandwidth of the current device, the
   on-chip bound of both de-dispersion stages (stage 1 reads one byte of
   shared memory per sample-add, stage 2 two): one 1024-thread block per SM
   streams conflict-free 32-bit loads (a warp reads one 128-byte row per
   load) `iters` x 8 times each from a 32 KB buffer; the second of two
   launches is timed with CUDA events on `stream`. Writes bytes per second
   over all SMs to *h_bytes_per_s. Synchronises `stream`. */
int32_t tx_measure_smem_bandwidth(int32_t iters, double* h_bytes_per_s, void* stream);

/* ---- phase timing (CUDA events recorded on the execute's stream) ----
   Phases of one execute, in order:
     TX_PHASE_INGEST  carried tail + new block into the ring (Sec. 2.3 steps 1, 2, 4)
     TX_PHASE_STAGE1  sub-bands at the coarse DMs (Sec. 2.3 sub-band step 1)
     TX_PHASE_STAGE2  fine DMs from the sub-bands + exact sums (sub-band step 3)
     TX_PHASE_STATS   mean / sigma per DM (Eq. 5's sigma)
     TX_PHASE_BOXCAR  boxcar S/N and outputs (Eq. 5, Sec. 2.5)
   A timer owns (TX_NPHASES + 1) * max_steps events created on the current
   device; each tx_execute_timed call records one step's boundaries. */
#define TX_PHASE_INGEST 0
#define TX_PHASE_STAGE1 1
#define TX_PHASE_STAGE2 2
#define TX_PHASE_STATS  3
#define TX_PHASE_BOXCAR 4
#define TX_NPHASES      5

typedef struct tx_timer tx_timer;

int32_t tx_timer_create(int32_t max_steps, tx_timer** out);

/* Forgets recorded steps (the events are reused). */
int32_t tx_timer_clear(tx_timer* timer);

/* tx_execute, recording the phase boundaries of the timer's next step on
   `stream`. Errors as tx_execute, plus INVALID_ARG when the timer is full. */
int32_t tx_execute_timed(const tx_plan* plan, tx_beam* beam, const uint8_t* d_block, void* d_out,
                         int64_t* d_ncand, void* d_workspace, void* stream, tx_timer* timer);

/* Waits for the last recorded event, then writes the summed milliseconds per
   phase over all recorded steps to h_ms[TX_NPHASES], the step count, and (if
   h_step_ms is not NULL) each step's total milliseconds to h_step_ms[nsteps]. */
int32_t tx_timer_read(tx_timer* timer, double* h_ms, int32_t* nsteps, double* h_step_ms);

void tx_timer_destroy(tx_timer* timer);

/* ---- batched execute: many beams of uneven shape per step ----
   The paper processes a beam block by block (Sec. 2.3 data flow, Sec. 3:
   blocks of about a second) on CPU cores; on one GPU many beams share each
   step. A batch binds n (plan, beam) pairs -- any mix of channel counts,
   block lengths, DM grids, width ladders, layouts, statistics and output
   modes, all with uint16 intermediates -- and runs one block of every beam
   per tx_execute_batch: one ingest launch for all beams, then, per wave, one
   persistent launch per phase and kernel variant over the concatenated work
   of the wave's beams (stage 1 per tile length, stage 2 per warp split,
   statistics, boxcar per width-count class and output mode). Each beam's
   results are exactly those tx_execute would give for the same block, and
   its beam state (tail, running statistics, block count) advances the same way.

   Waves: the beams are split, in order, into waves of at most 92 beams
   whose summed per-beam workspace (tx_plan_info.workspace_bytes, or
   workspace_bytes_compact for a compact beam) fits workspace_budget when it
   is > 0; waves run one after another in the same workspace. At most two
   batches may exist per device at a time (their per-beam arguments live in
   one of two constant-memory slots; a third create returns TX_ERR_BUDGET).

   TX_BATCH_GRAPH: the first two steps are captured (on a private stream) as
   CUDA graphs, one per argument buffer, and later steps replay them; without
   the flag every step enqueues its launches directly. Either way a step first
   copies the per-beam arguments (pointers, ring positions) from one of two
   pinned host buffers, and a call waits for the step two calls back to finish
   before it rewrites that step's buffer. Consecutive calls on one batch must
   go to the same stream. A beam in a batch must not be used by other calls
   while the batch is in use. */
#define TX_BATCH_GRAPH   1
/* TX_BATCH_PROFILE (direct launches only): CUDA events around every launch;
   each call first waits for the previous step's events and adds its launch
   times to per-phase sums read by tx_batch_read_profile. */
#define TX_BATCH_PROFILE 2

typedef struct tx_batch tx_batch;

typedef struct tx_batch_info {
  int32_t nbeams;           /* n                                                    */
  int32_t nwaves;           /* waves under the workspace budget                     */
  int32_t nlaunches;        /* kernel launches per step                             */
  int32_t flags;            /* TX_BATCH_* flags of the batch                        */
  int64_t workspace_bytes;  /* d_workspace bytes tx_execute_batch needs             */
  int64_t dm_trial_samples; /* sum over beams of ndm * T: DM-trial x samples a step */
} tx_batch_info;

/* Builds a batch on the current device: plans[i] with beams[i] (created for
   that plan on this device, each beam at most once). Uploads the plans'
   tables if needed and allocates the batch's work lists and argument
   buffers. Errors: INVALID_ARG, UNSUPPORTED (int32 intermediates, or shapes
   beyond a launch's limits), BUDGET (one beam's workspace exceeds the
   budget), OOM, CUDA. */
int32_t tx_batch_create(int32_t n, const tx_plan* const* plans, tx_beam* const* beams,
                        int64_t workspace_budget, int32_t flags, tx_batch** out);

int32_t tx_batch_get_info(const tx_batch* batch, tx_batch_info* info);

/* One step of every beam of the batch. Host arrays of n device pointers:
     d_blocks[i]  beam i's block, as d_block of tx_execute
     d_outs[i]    beam i's output, info.out_bytes of its plan
     d_ncands     may be NULL when no beam is in TX_OUT_CANDS mode; else
                  d_ncands[i] is beam i's int64 counter (NULL for other modes)
     d_workspace  tx_batch_info.workspace_bytes of device scratch
   Enqueued on `stream`; may block the host until the step two calls back
   has finished (see above). d_workspace must be 16-byte aligned; each
   d_outs[i] is aligned as tx_execute's d_out. */
int32_t tx_execute_batch(tx_batch* batch, const uint8_t* const* d_blocks, void* const* d_outs,
                         int64_t* const* d_ncands, void* d_workspace, void* stream);

/* Waits, polling, until the batch's last enqueued step has finished on the
   GPU, at most timeout_us microseconds (< 0: no limit). Returns TX_OK, or
   TX_ERR_TIMEOUT when the limit ran out first (the step keeps running and
   can be waited for again), TX_ERR_ABORTED when the kernels of a member beam
   have given up a wait (tx_last_error names it; see tx_beam_failed), or
   TX_ERR_CUDA if the step failed. */
int32_t tx_batch_wait(tx_batch* batch, int64_t timeout_us);

/* TX_BATCH_PROFILE batches: waits for the last step, then writes the summed
   milliseconds of each phase's launches over all steps to h_ms[TX_NPHASES]
   (indexed by TX_PHASE_*) and the step count to *nsteps (may be NULL). */
int32_t tx_batch_read_profile(tx_batch* batch, double* h_ms, int32_t* nsteps);

/* Waits for the batch's steps in flight, then frees what it holds (not the
   plans or beams). */
void tx_batch_destroy(tx_batch* batch);

/* ---- candidate clustering (Sec. 2.5: DBSCAN on the DM-time plane) ----
   The candidates of a block (tx_cand records, the DM-time plane's points at or
   above the threshold) are clustered with DBSCAN after DM is converted to the
   dispersion delay across the band (Eq. 1, lowest to highest channel centre,
   ms) and time to t * t_samp (ms):
     core point   more than k other points at Euclidean distance <= radius_ms
     cluster      core points joined by chains of core neighbours, plus every
                  non-core point within radius_ms of one of them
     outlier      any other point (label -1)
   Points are taken in canonical order, sorted by (dm_index, t); a cluster's id
   is the canonical index of its first core point; a non-core point next to
   several clusters joins the one of smallest id. Results do not depend on the
   order of the input records. The paper searches neighbours with a kd-tree;
   here a uniform grid of cells of side ~radius_ms does it (section 2.5's
   prune rules become "only the 3 x 3 cells around a point"). */
typedef struct tx_cluster {
  int32_t id;                 /* canonical index of the cluster's first core point     */
  int32_t dm_index, t, w_index;
  float   snr;                /* the member of highest S/N (ties: first in canonical
                                 order), reported for the cluster                        */
  int32_t members;            /* points in the cluster                                 */
  int32_t dm_lo, dm_hi;       /* DM-index and time extent of the members               */
  int32_t t_lo, t_hi;
} tx_cluster;

typedef struct tx_clusterer tx_clusterer;

/* The delay of each DM trial of a plan as used for clustering: double
   [ndm], K DM (f_min^-2 - f_max^-2) in ms (f_min, f_max the lowest and highest
   channel centres). */
int32_t tx_plan_delay_table(const tx_plan* plan, double* h_delay_ms);

/* Scratch for clustering up to max_points candidates of the plan's blocks on
   the current device (about 90 bytes per point). Errors: INVALID_ARG, OOM, CUDA. */
int32_t tx_clusterer_create(const tx_plan* plan, double radius_ms, int32_t k, int64_t max_points,
                            tx_clusterer** out);

/* Clusters n records at d_cands (device; may be NULL when n is 0). Writes the clusters in id order to
   d_out (room for n records) and their count to *d_nclusters (device int64);
   d_labels (may be NULL) receives the cluster id of each point in canonical
   order (-1: outlier) and d_order (may be NULL) the record index of each
   canonical position. Enqueued on `stream`; n <= max_points. */
int32_t tx_cluster_run(tx_clusterer* c, const tx_cand* d_cands, int64_t n, tx_cluster* d_out,
                       int64_t* d_nclusters, int32_t* d_labels, int32_t* d_order, void* stream);

void tx_clusterer_destroy(tx_clusterer* c);

/* ---- de-dispersion plans with downsampling (Sec. 2.3, last paragraph) ----
   At high DM the smearing inside one channel exceeds the sampling time, so
   the DM range can be split into segments de-dispersed on downsampled data
   (a plan per segment with sampling time f t_samp and blocks of T / f
   samples). The paper gives no rule; the library's:
     h_factor[d] = the largest power of two (at least 1, at most f_max) not
                   above the Eq. 1 delay of DM d across the lowest-frequency
                   channel (edges at its centre -+ half the channel spacing),
                   in samples.
   Consecutive DMs with the same factor form a segment. */
int32_t tx_plan_segments(int32_t nchan, const double* freq_mhz, double tsamp_s, int32_t ndm, const double* dm,
                         int32_t f_max, int32_t* h_factor);

/* A downsampled plan: the DM grid of `desc` split into those segments, each
   with its own plan (f_max first drops to the largest power of two dividing
   T, so every factor divides the block):
     segment j   DM trials [dm_lo, dm_hi) of desc's grid with factor f
     its plan    desc with sampling time f t_samp, those DMs, blocks of T / f
                 samples and widths W / f (at least 1, duplicates dropped, so
                 the physical widths that are resolved are kept)
   Its input is the block averaged over f samples (tx_downsample). The
   segment plan's output t' covers native samples [f t', f (t' + 1)) of its
   own window, which starts f L_j native samples before the block (L_j its
   overlap); with the native overlap L = max_j f L_j, that is native window
   time f t' + native_offset, native_offset = L - f L_j.
   The segment plans belong to the downsampled plan: do not destroy them.
   Errors: as tx_plan_create for any segment, and INVALID_ARG. */
typedef struct tx_segment {
  int32_t dm_lo, dm_hi;     /* DM trials [dm_lo, dm_hi) of the full grid                */
  int32_t factor;           /* f                                                        */
  int32_t nwidth;           /* widths of the segment plan, in downsampled samples       */
  int32_t widths[32];
  int64_t nsamp;            /* T / f                                                    */
  int64_t overlap;          /* L_j, downsampled samples                                 */
  int64_t native_offset;    /* L - f L_j, native samples                                */
} tx_segment;

typedef struct tx_dsplan tx_dsplan;

int32_t tx_dsplan_create(const tx_plan_desc* desc, int32_t f_max, tx_dsplan** out);
/* Number of segments and the native overlap L (either pointer may be NULL). */
int32_t tx_dsplan_get_info(const tx_dsplan* ds, int32_t* nseg, int64_t* overlap);
/* Segment j's description and plan (either pointer may be NULL). */
int32_t tx_dsplan_segment(const tx_dsplan* ds, int32_t j, tx_segment* seg, const tx_plan** plan);
/* Frees the downsampled plan and its segment plans. */
void tx_dsplan_destroy(tx_dsplan* ds);

/* Averages `factor` consecutive samples of every channel, rounding half up:
   out[t'] = (sum_{i<factor} in[factor t' + i] + factor / 2) / factor for
   t' < nsamp / factor, in the same layout (FT [nchan][n] or TF [n][nchan]).
   factor is a power of two <= 1024 dividing nsamp. Enqueued on `stream`. */
int32_t tx_downsample(const uint8_t* d_in, int32_t layout, int32_t nchan, int64_t nsamp, int32_t factor,
                      uint8_t* d_out, void* stream);

/* ---- allocation-free de-dispersion (the paper has no counterpart) ----
   For callers that cannot call cudaMalloc: real-time loops that must not take
   the allocator's locks or its implicit synchronisation, hosts that embed the
   library under a device-memory budget another framework owns, and code that
   must not fail for lack of memory once running.

   Computes the de-dispersed series of one window, as TX_OUT_SERIES does, and
   allocates nothing (no cudaMalloc, cudaFree or allocating library call):
     d_x       uint8 [nchan][ld] channel-major window: the L carried samples
               then the T new ones (T + L <= ld); 16-byte aligned start, ld a
               multiple of 64 (samples past T + L are read but never affect
               the result)
     d_series  int32 [ndm][T + W_max - 1], written; 8-byte aligned
   The stage-1 sums, per-tile sums and copies of the plan's tables live in one
   32 MiB static device array that every GPU loading this library holds until
   the process exits; plans that need more return TX_ERR_BUDGET with the size
   in tx_last_error(). Only uint16-intermediate plans are supported.
   The first call on each device looks up the array's device address; make
   that first call outside any stream capture. Every call uses the same array
   and leaves its contents behind (nothing in it needs to start at zero):
   calls that overlap on the GPU, on any streams, race with each other. The
   plan's tables are copied in from host memory on every call. A kernel that
   gives up a wait (see tx_set_wait_polls) is counted by tx_wait_timeouts
   only; the series of that call are then not valid.
   Errors: INVALID_ARG (null or misaligned pointer, bad ld), UNSUPPORTED,
   BUDGET, before anything is enqueued; CUDA. */
int32_t tx_dedisperse_noalloc(const tx_plan* plan, const uint8_t* d_x, int64_t ld, int32_t* d_series,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRANSIENTX_H */
