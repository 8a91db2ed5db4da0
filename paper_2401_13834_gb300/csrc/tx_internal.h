// Internal declarations shared by the host plan (plan.cpp) and the CUDA side
// (kernels.cu). Nothing here is part of the public C ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "transientx.h"

namespace tx {

// Eq. 1 constant e^2 / (2 pi m_e c) in s MHz^2 pc^-1 cm^3.
constexpr double kDispersion = 4.148808e3;

// ---- stage 1 (channels -> sub-bands at coarse DMs) tiling -------------------
// A stage-1 tile covers 4*q consecutive times: a shared-memory word holds the
// samples of times j, j+q, j+2q, j+3q of one channel, so one 32-bit load feeds
// four outputs whatever the per-channel delay.
constexpr int kStage1MaxCoarse = 64;   // coarse DMs that share one staged tile (two per warp at most)
constexpr int kStage1Warps = 32;
// Staged words per channel for quarter length q: the tile (q words), the
// chunk's delay spread (<= q - 16), the window's misalignment (< 16) and
// rounding to 4-word groups: at most 2q + 2, so 2q + 4 words. Word j of a
// channel takes raw bytes j + iq (i = 0..3): the transform reads bytes up to
// 4 (Q + span + 18) / 4 - 1 + 3q <= 5q + 1 of the window, which spans 5q + 2
// bytes rounded up to 16-byte chunks.
constexpr int kStage1StagedWords(int q) { return 2 * q + 4; }
constexpr int kStage1RawBytes(int q) { return (5 * q + 2 + 15) / 16 * 16; }
constexpr int kSmemMax = 232448;       // opt-in dynamic shared memory per block (227 KB)

// Polls of an mbarrier before a kernel gives up waiting for a bulk copy; each
// poll may suspend the thread for a while, so this is seconds in all.
constexpr uint32_t kWaitPolls = 1u << 22;

// ---- stage 2 (sub-bands -> fine DMs) tiling ---------------------------------
// A stage-2 tile is nw2 32-bit words of uint16 pairs (two outputs each):
// 512 words for groups of up to 16 fine DMs (16 warps), 256 beyond.
constexpr int kStage2MaxGroup = 32;    // one warp per fine DM of a group
// The pipelined 16-bit stage 2: stages of sub-band chunks in flight, producer
// warps, and the largest group it takes (consumer warps = group x warps per DM <= 28).
constexpr int kPipeStages2 = 3;
constexpr int kPipeProd2 = 4;
constexpr int kPipeMaxGroup2 = 16;
// shared-memory bytes of the pipelined stage 2 for `sc` sub-bands of `sww` words per stage
constexpr int64_t stage2_pipe_smem(int sc, int sww) {
  return (int64_t)kPipeStages2 * (2 * (int64_t)sc * sww + (int64_t)(kPipeMaxGroup2 + 1) * ((sc + 3) & ~3)) * 4;
}

// ---- matched filter ---------------------------------------------------------
constexpr int kBoxTile = 2048;         // outputs per boxcar sub-tile (a unit holds 1, 2 or 4)
constexpr int64_t kBoxMinUnits = 152 * 4 * 8;   // units a plan keeps for a full GPU before lengthening them
constexpr int kBoxThreads = 256;
constexpr int kMaxWidths = 32;
constexpr int kMaxWidth = 4096;



// Stage-1 work item: sub-band s, coarse DMs [kb, ke), times [tau0, tau0 + 4 q1),
// span = max over the sub-band's channels of d1[ke-1][c] - d1[kb][c]; tab =
// word offset of the item's precomputed offset table in the plan's tab1
// (shared by the items of one (s, kb, ke) at every time).
struct Stage1Item {
  int32_t s, kb, ke, tau0, span, tab, pad1, pad2;
};

// Per (fine DM, width) constants of the S/N normalisation (Eq. 5):
// S/N = (float(B - hi) - lo) * inv with hi + lo = W * mu and inv = 1 / (sigma sqrt W);
// thr = ceil(W mu + gamma sigma sqrt W), so S/N >= gamma exactly when B >= thr.
struct SnrConst {
  int32_t hi;
  float lo;
  float inv;
  int32_t thr;
};

struct DevicePlan {
  int device = -1;
  int num_sms = 0;
  int box_blocks_per_sm = 1;     // resident boxcar blocks per SM (persistent grid)
  int32_t* d1 = nullptr;         // [nk][nchan]
  int32_t* abase = nullptr;      // [nk][nsub]
  int32_t* e2 = nullptr;         // [ndm][nsub]
  int32_t* widths = nullptr;     // [nw]
  Stage1Item* items1 = nullptr;  // [n_items1]
  int32_t* tab1 = nullptr;       // stage-1 offset tables of the item groups
  int32_t* tab2 = nullptr;       // pipelined stage 2: offset tables per (coarse group, sub-band chunk)
  Stage1Item* items_f = nullptr; // float path stage-1 items
};

void set_error(const char* fmt, ...);
int64_t stage1_smem_bytes(int m, int q);
// Polling limit of the first wait for each bulk copy in the kernels launched
// from now on (tx_set_wait_polls; kWaitPolls unless changed).
uint32_t first_wait_polls();

}  // namespace tx

struct tx_plan {
  // ---- description -------------------------------------------------------
  int32_t nchan = 0, nsub = 0, m = 0, ndm = 0, nk = 0, group = 0, nw = 0, wmax = 0;
  int32_t box_vec = 0;            // widths 1, 2, then multiples of 4: the boxcar's 4-output test
  int64_t T = 0;
  int32_t layout = 0, interm = 0, output = 0, stats = 0;
  int32_t norm = 0;               // enum tx_norm: the float path when not TX_NORM_NONE
  int32_t esz = 1;                // bytes per sample of a beam's buffer (4 on the float path)
  float gamma = 0.f;
  int64_t max_cands = 0;
  double lambda = 1.0;
  double tsamp = 0.0, f_ref = 0.0;
  std::vector<double> freq, dm, coarse_dm, f_ref_s;
  std::vector<int32_t> widths;

  // ---- tables (Eq. 1, Sec. 2.3) -------------------------------------------
  std::vector<int32_t> d1;        // [nk][nchan]
  std::vector<int32_t> d2;        // [ndm][nsub]
  std::vector<int32_t> kof;       // [ndm]
  std::vector<double> delay_ms;   // [ndm] Eq. 1 across the band (lowest to highest centre), ms
  int64_t max_delay = 0, L = 0;

  // ---- derived layout -----------------------------------------------------
  std::vector<int32_t> abase;     // [nk][nsub] absolute time of P row start
  std::vector<int32_t> e2;        // [ndm][nsub] = d2 - abase
  int64_t Td = 0;                 // series length T + wmax - 1
  int64_t Pp = 0;                 // P row pitch (elements)
  int64_t Dp = 0;                 // D row pitch (int32 elements)
  int64_t R = 0;                  // ring bytes per channel (circular)
  int64_t head0 = 0;              // where a fresh beam's first block lands
  int32_t q1 = 256;               // stage-1 quarter length (words)
  int32_t span1_max = 256;        // staged delay spread limit of stage 1
  int32_t span2_max = 0;          // max stage-2 delay spread within a group
  int32_t nw2 = 512;              // stage-2 tile words (2 * nw2 outputs)
  int32_t split2 = 2;             // stage-2 warps per fine DM (uint16 path)
  int32_t pipe2 = 0;              // 16-bit stage 2 runs as the barrier-free pipeline (groups <= 16)
  int32_t ntile2 = 0;             // stage-2 tiles over the series
  int32_t sww2 = 0;               // stage-2 staged words per sub-band (uint16 path)
  int32_t sw2_i32 = 0;            // stage-2 staged elements per sub-band (int32 path)
  int32_t nsub_chunk2 = 0;        // sub-bands staged at once by stage 2
  int32_t e2w2 = 0;               // words of one stage-2 group's delays in shared memory (rounded to 4)
  int32_t box_tile = tx::kBoxTile;  // boxcar outputs per unit (a multiple of kBoxTile)
  int32_t ntile3 = 0;             // boxcar units per DM over [0, T)
  int32_t ntile2f = 0;            // float path: stage-2 tiles over the series (those of ntile2)
  int32_t tile_f = 0, span_f = 0;  // float path: stage-1 item length and delay spread limit
  std::vector<tx::Stage1Item> items_f;  // float path stage-1 items (s, coarse DMs [kb, ke), times)
  std::vector<tx::Stage1Item> items1;
  // stage-1 offset tables, per (s, kb, ke): rows kk < ke - kb of (m + 3) & ~3
  // words, word c = c * staged words + ((tab1_phase + d1[kb][c]) & 15) +
  // d1[kb + kk][c] - d1[kb][c], then abase[kb + kk][s] for kk < ke - kb
  // (padded to 4); valid for executes whose window start has tab1_phase as
  // its residue mod 16 (every block when T is a multiple of 16)
  std::vector<int32_t> tab1;
  int32_t tab1_phase = 0;
  // pipelined stage 2, per (coarse group k, sub-band chunk): rows g < group of
  // SCq = (nsub_chunk2 + 3) & ~3 words, word ss = the element offset of fine
  // DM kG + g's pairs in sub-band s = chunk * nsub_chunk2 + ss from the start
  // of that sub-band's staged row, then one row of those starts relative to
  // the tile start (multiples of 8: the 16-byte alignment of bulk copies)
  std::vector<int32_t> tab2;

  // ---- workspace carve-up (bytes) -------------------------------------------
  int64_t ws_P = 0, ws_D = 0, ws_part = 0, ws_const = 0, ws_hoff = 0, ws_ctr = 0, ws_bytes = 0;
  int64_t out_bytes = 0, beam_bytes = 0, export_bytes = 0;
  // compact beams: the tail lives in [nchan][tail_pitch] (samples at
  // tail_pad.. so that they share the ring's 16-byte phase); an execute
  // borrows the ring from the workspace at ws_ring
  int64_t tail_pad = 0, tail_pitch = 0, ws_ring = 0, ws_bytes_compact = 0, compact_beam_bytes = 0;

  // ---- device copy, uploaded once ------------------------------------------
  std::once_flag dev_once;
  int dev_status = 0;
  tx::DevicePlan dev;
};

struct tx_beam {
  const tx_plan* plan = nullptr;
  int device = -1;
  int compact = 0;                // tail store instead of a resident ring
  uint8_t* ring = nullptr;        // [nchan][R] circular (full beams)
  uint8_t* tail = nullptr;        // [nchan][tail_pitch] carried tail (compact beams)
  int64_t head = 0;               // where the next block lands
  double* run = nullptr;          // [ndm][2] running (mu, var); var < 0 = unset
  int32_t* fail = nullptr;        // waits the beam's kernels gave up (device word after run)
  uint8_t* chan = nullptr;        // float path: channel sums and (mu, w) of a primed tail [nchan] x 24 bytes
  int64_t nblocks = 0;
};

// Implemented in kernels.cu.
int tx_upload_plan(const tx_plan* plan);
// The float path (floatpath.cu): one block of a beam of a plan with a
// normalisation; arguments as tx_execute (ev: optional phase events as in
// tx_execute_timed). prime: normalise a tail of L samples into the beam.
int float_execute(const tx_plan* p, tx_beam* b, const uint8_t* d_block, void* d_out, int64_t* d_ncand,
                  void* d_workspace, void* stream, void* const* ev);
int float_prime(const tx_plan* p, tx_beam* b, const uint8_t* d_tail, void* stream);
// Waits given up by the batched kernels on the current device (batch.cu).
int batch_wait_timeouts(int64_t* n);
