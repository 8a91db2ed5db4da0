// Host side of the plan: Eq. 1 delay tables, the sub-band grouping of Sec. 2.3,
// the overlap carried between blocks, and the kernels' work lists and layouts.
//
// Compiled with -ffp-contract=off so that every delay is evaluated as
// K * DM * (1/f^2 - 1/f_ref^2) / t_samp with separately rounded IEEE double
// operations on every host architecture, then rounded half away from zero
// (llround).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "tx_internal.h"

namespace tx {

static thread_local std::string g_last_error;
static std::atomic<uint32_t> g_first_wait_polls{kWaitPolls};

uint32_t first_wait_polls() { return g_first_wait_polls.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Shared memory of the stage-1 kernel: staged words, raw prefetch buffer and
// the offset table (rows padded to a multiple of four entries).
int64_t stage1_smem_bytes(int m, int q) {
  // staged words, raw windows, offset table, P-row bases, three item
  // descriptors, two rows of delays and two sub-band offsets
  return (int64_t)m * kStage1StagedWords(q) * 4 + (int64_t)m * kStage1RawBytes(q) +
         (int64_t)kStage1MaxCoarse * ((m + 3) & ~3) * 4 + (int64_t)kStage1MaxCoarse * 4 +
         3 * (int64_t)sizeof(Stage1Item) + 2 * (int64_t)((m + 3) & ~3) * 4 + 16;
}

static int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Eq. 1 in samples: rnd(K DM (1/f^2 - 1/f_ref^2) / t_samp), rnd = llround.
static int64_t delay_samples(double dm, double f, double f_ref, double tsamp) {
  const double v = kDispersion * dm * (1.0 / (f * f) - 1.0 / (f_ref * f_ref)) / tsamp;
  return std::llround(v);
}

// Automatic coarse-grid rule (the paper leaves the coarse DM grid open): the
// largest power of two G with G <= 1 + S_full / S_sub, where S_full is the
// delay per unit DM across the whole band and S_sub the largest one inside a
// sub-band, capped by the largest power of two <= ndm. Then a coarse DM's
// residual smear inside any sub-band stays below the fine grid's half-step
// smear across the band.
static int auto_group(const std::vector<double>& f, double tsamp, int nsub, int ndm) {
  const int nchan = (int)f.size();
  const int m = nchan / nsub;
  const double f_ref = *std::max_element(f.begin(), f.end());
  const double f_min = *std::min_element(f.begin(), f.end());
  const double s_full = kDispersion * (1.0 / (f_min * f_min) - 1.0 / (f_ref * f_ref)) / tsamp;
  double s_sub = 0.0;
  for (int s = 0; s < nsub; ++s) {
    const double lo = *std::min_element(f.begin() + s * m, f.begin() + (s + 1) * m);
    const double hi = *std::max_element(f.begin() + s * m, f.begin() + (s + 1) * m);
    const double v = kDispersion * (1.0 / (lo * lo) - 1.0 / (hi * hi)) / tsamp;
    s_sub = std::max(s_sub, v);
  }
  int cap = 1;
  while ((int64_t)cap * 2 <= ndm) cap *= 2;
  if (s_sub <= 0.0) return cap;
  const double ratio = 1.0 + s_full / s_sub;
  int g = 1;
  while ((double)(g * 2) <= ratio && g * 2 <= cap) g *= 2;
  return g;
}

static int build(tx_plan* p, const tx_plan_desc* d) {
  // ---- validation ----------------------------------------------------------
  if (!d->freq_mhz || !d->dm || !d->widths) { set_error("null table pointer in plan description"); return TX_ERR_INVALID_ARG; }
  if (d->nchan < 1 || d->nsub < 1 || d->ndm < 1) { set_error("nchan, nsub and ndm must be >= 1"); return TX_ERR_INVALID_ARG; }
  if (d->nchan % d->nsub) { set_error("nchan (%d) is not a multiple of nsub (%d)", d->nchan, d->nsub); return TX_ERR_NOT_DIVISIBLE; }
  const int m = d->nchan / d->nsub;
  if (m > 257) { set_error("at most 257 channels per sub-band (uint16 stage-1 sums); got %d", m); return TX_ERR_UNSUPPORTED; }
  if (!(d->tsamp_s > 0.0) || !std::isfinite(d->tsamp_s)) { set_error("tsamp_s must be > 0"); return TX_ERR_INVALID_ARG; }
  for (int c = 0; c < d->nchan; ++c)
    if (!(d->freq_mhz[c] > 0.0) || !std::isfinite(d->freq_mhz[c])) { set_error("freq_mhz[%d] must be finite and > 0", c); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < d->ndm; ++i) {
    if (!(d->dm[i] >= 0.0) || !std::isfinite(d->dm[i])) { set_error("dm[%d] must be finite and >= 0", i); return TX_ERR_INVALID_ARG; }
    if (i && d->dm[i] < d->dm[i - 1]) { set_error("dm must be ascending (dm[%d] < dm[%d])", i, i - 1); return TX_ERR_INVALID_ARG; }
  }
  if (d->nwidth < 1 || d->nwidth > kMaxWidths) { set_error("nwidth must be in [1, %d]", kMaxWidths); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < d->nwidth; ++i) {
    if (d->widths[i] < 1 || d->widths[i] > kMaxWidth) { set_error("widths[%d] must be in [1, %d]", i, kMaxWidth); return TX_ERR_INVALID_ARG; }
    if (i && d->widths[i] <= d->widths[i - 1]) { set_error("widths must be strictly ascending"); return TX_ERR_INVALID_ARG; }
  }
  if (d->nsamp < 1) { set_error("nsamp must be >= 1"); return TX_ERR_INVALID_ARG; }
  if (d->group < 0) { set_error("group must be >= 0"); return TX_ERR_INVALID_ARG; }
  if (d->layout != TX_LAYOUT_FT && d->layout != TX_LAYOUT_TF) { set_error("bad layout"); return TX_ERR_INVALID_ARG; }
  if (d->interm != TX_INTERM_U16 && d->interm != TX_INTERM_I32 && d->interm != TX_INTERM_F16 && d->interm != TX_INTERM_F32) { set_error("bad interm"); return TX_ERR_INVALID_ARG; }
  if (d->norm != TX_NORM_NONE && d->norm != TX_NORM_UNIT && d->norm != TX_NORM_INVVAR) { set_error("bad norm"); return TX_ERR_INVALID_ARG; }
  if ((d->norm != TX_NORM_NONE) != (d->interm == TX_INTERM_F32)) {
    set_error("the float path pairs a normalisation (norm) with float32 intermediates (TX_INTERM_F32)");
    return TX_ERR_INVALID_ARG;
  }
  if (d->norm != TX_NORM_NONE && d->ndm > 65535) { set_error("the float path takes at most 65535 DM trials"); return TX_ERR_UNSUPPORTED; }
  if (d->output < TX_OUT_CANDS || d->output > TX_OUT_SERIES) { set_error("bad output mode"); return TX_ERR_INVALID_ARG; }
  if (d->stats != TX_STATS_BLOCK && d->stats != TX_STATS_RUNNING) { set_error("bad stats mode"); return TX_ERR_INVALID_ARG; }
  if (d->stats == TX_STATS_RUNNING && !(d->stats_lambda > 0.0 && d->stats_lambda <= 1.0)) { set_error("stats_lambda must be in (0, 1]"); return TX_ERR_INVALID_ARG; }
  if (d->output == TX_OUT_CANDS && d->max_cands < 1) { set_error("max_cands must be >= 1"); return TX_ERR_INVALID_ARG; }
  if (!std::isfinite(d->snr_threshold)) { set_error("snr_threshold must be finite"); return TX_ERR_INVALID_ARG; }

  p->nchan = d->nchan; p->nsub = d->nsub; p->m = m; p->ndm = d->ndm; p->nw = d->nwidth;
  p->T = d->nsamp; p->layout = d->layout; p->interm = d->interm; p->output = d->output;
  p->stats = d->stats; p->gamma = d->snr_threshold; p->max_cands = d->max_cands;
  p->norm = d->norm;
  p->lambda = d->stats == TX_STATS_RUNNING ? d->stats_lambda : 1.0;
  p->tsamp = d->tsamp_s;
  p->freq.assign(d->freq_mhz, d->freq_mhz + d->nchan);
  p->dm.assign(d->dm, d->dm + d->ndm);
  p->widths.assign(d->widths, d->widths + d->nwidth);
  p->wmax = p->widths.back();
  p->box_vec = p->nw >= 2 && p->widths[0] == 1 && p->widths[1] == 2;
  for (int w = 2; w < p->nw; ++w) p->box_vec = p->box_vec && p->widths[w] % 4 == 0;
  // window sums (<= wmax * nchan * 255) and W * mu must fit int32
  if ((double)p->wmax * p->nchan * 255.0 >= 2147483647.0) { set_error("wmax * nchan * 255 must be < 2^31"); return TX_ERR_UNSUPPORTED; }
  // exact S2 = sum D^2 in uint64
  if ((double)p->T * std::pow((double)p->nchan * 255.0, 2) >= 9.2e18) { set_error("nsamp * (nchan*255)^2 must be < 2^63"); return TX_ERR_UNSUPPORTED; }

  // ---- Eq. 1 tables, sub-band scheme of Sec. 2.3 ----------------------------
  const int nchan = p->nchan, nsub = p->nsub, ndm = p->ndm;
  p->group = d->group ? d->group : auto_group(p->freq, p->tsamp, nsub, ndm);
  const int G = p->group;
  if (G > kStage2MaxGroup) { set_error("group (%d) must be <= %d", G, kStage2MaxGroup); return TX_ERR_UNSUPPORTED; }
  p->nk = (ndm + G - 1) / G;
  const int nk = p->nk;
  p->f_ref = *std::max_element(p->freq.begin(), p->freq.end());
  p->f_ref_s.resize(nsub);
  for (int s = 0; s < nsub; ++s) p->f_ref_s[s] = *std::max_element(p->freq.begin() + s * m, p->freq.begin() + (s + 1) * m);
  {
    // DM as dispersion delay across the band (Sec. 2.5 clustering), ms
    const double f_lo = *std::min_element(p->freq.begin(), p->freq.end());
    p->delay_ms.resize(ndm);
    for (int i = 0; i < ndm; ++i)
      p->delay_ms[i] = kDispersion * p->dm[i] * (1.0 / (f_lo * f_lo) - 1.0 / (p->f_ref * p->f_ref)) * 1e3;
  }
  p->kof.resize(ndm);
  for (int i = 0; i < ndm; ++i) p->kof[i] = i / G;
  p->coarse_dm.resize(nk);
  for (int k = 0; k < nk; ++k) p->coarse_dm[k] = (p->dm[k * G] + p->dm[std::min((k + 1) * G, ndm) - 1]) / 2.0;
  p->d1.resize((size_t)nk * nchan);
  for (int k = 0; k < nk; ++k)
    for (int c = 0; c < nchan; ++c) {
      const int64_t v = delay_samples(p->coarse_dm[k], p->freq[c], p->f_ref_s[c / m], p->tsamp);
      if (v < 0 || v > (1LL << 30)) { set_error("stage-1 delay out of range"); return TX_ERR_UNSUPPORTED; }
      p->d1[(size_t)k * nchan + c] = (int32_t)v;
    }
  p->d2.resize((size_t)ndm * nsub);
  for (int i = 0; i < ndm; ++i)
    for (int s = 0; s < nsub; ++s) {
      const int64_t v = delay_samples(p->dm[i], p->f_ref_s[s], p->f_ref, p->tsamp);
      if (v < 0 || v > (1LL << 30)) { set_error("stage-2 delay out of range"); return TX_ERR_UNSUPPORTED; }
      p->d2[(size_t)i * nsub + s] = (int32_t)v;
    }
  // overlap L = max over (d, c) of d1[k(d)][c] + d2[d][s(c)] + W_max - 1
  int64_t best = 0;
  std::vector<int32_t> d2max((size_t)nk * nsub, 0), d2min((size_t)nk * nsub, 0);
  for (int k = 0; k < nk; ++k)
    for (int s = 0; s < nsub; ++s) {
      int32_t hi = 0, lo = INT32_MAX;
      for (int i = k * G; i < std::min((k + 1) * G, ndm); ++i) {
        hi = std::max(hi, p->d2[(size_t)i * nsub + s]);
        lo = std::min(lo, p->d2[(size_t)i * nsub + s]);
      }
      d2max[(size_t)k * nsub + s] = hi;
      d2min[(size_t)k * nsub + s] = lo;
      for (int c = s * m; c < (s + 1) * m; ++c) best = std::max<int64_t>(best, (int64_t)p->d1[(size_t)k * nchan + c] + hi);
    }
  p->max_delay = best;
  p->L = best + p->wmax - 1;
  if (p->T + p->L >= (1LL << 30)) { set_error("nsamp + overlap must be < 2^30"); return TX_ERR_UNSUPPORTED; }

  // ---- stage-2 layout -------------------------------------------------------
  // P row (k, s) starts at absolute time abase = min_d d2 rounded down to 16 so
  // stage-1 tiles stay aligned; e2 = d2 - abase >= 0.
  p->Td = p->T + p->wmax - 1;
  p->abase.resize((size_t)nk * nsub);
  p->e2.resize((size_t)ndm * nsub);
  int32_t span2 = 0, e2max = 0;
  for (int k = 0; k < nk; ++k)
    for (int s = 0; s < nsub; ++s) {
      const int32_t lo = d2min[(size_t)k * nsub + s];
      p->abase[(size_t)k * nsub + s] = lo & ~15;
      span2 = std::max(span2, d2max[(size_t)k * nsub + s] - lo);
    }
  for (int i = 0; i < ndm; ++i)
    for (int s = 0; s < nsub; ++s) {
      const int32_t v = p->d2[(size_t)i * nsub + s] - p->abase[(size_t)p->kof[i] * nsub + s];
      p->e2[(size_t)i * nsub + s] = v;
      e2max = std::max(e2max, v);
    }
  p->span2_max = span2;
  // Stage-2 tiles hold nw2 uint16 pairs (2 * nw2 outputs).
  // A sub-band's staged window starts at the tile start + emin rounded down to
  // 8 elements (16 bytes) and spans the tile, the group's delay spread and
  // that alignment: sww2 32-bit words.
  // 512-word tiles shared by 2-8 warps per fine DM, or 256-word tiles with one
  int split = d->tile_split2;
  if (split == 0) split = G <= 4 ? 8 : G <= 8 ? 4 : G <= 16 ? 2 : 1;
  if (split != 1 && split != 2 && split != 4 && split != 8) { set_error("tile_split2 must be 0, 1, 2, 4 or 8"); return TX_ERR_INVALID_ARG; }
  if (std::min(G, kStage2MaxGroup) * split > 32) { set_error("min(group, 32) * tile_split2 must be <= 32 (group %d)", G); return TX_ERR_INVALID_ARG; }
  p->split2 = split;
  p->nw2 = split == 1 ? 256 : 512;
  // 16-bit intermediates with groups of up to 16 fine DMs: the pipelined stage 2,
  // 1024-output tiles, consumer warps per fine DM the largest of 4, 2, 1 that
  // keeps group x warps + producer warps <= 32 (the desc's tile_split2 applies
  // to the other kernel)
  const bool is16 = d->interm == TX_INTERM_U16 || d->interm == TX_INTERM_F16;
  const int32_t sww_pipe = (int32_t)round_up(512 + (span2 + 7 + 2) / 2 + 6, 4);
  p->pipe2 = is16 && G <= kPipeMaxGroup2 && stage2_pipe_smem(1, sww_pipe) <= kSmemMax - 1024;
  if (p->pipe2) {
    const int cmax = 32 - kPipeProd2;   // consumer warps beside the producer warps
    p->split2 = G * 4 <= cmax ? 4 : G * 2 <= cmax ? 2 : 1;
    p->nw2 = 512;
  }
  const int64_t tt2 = 2 * (int64_t)p->nw2;
  p->ntile2 = (int32_t)((p->Td + tt2 - 1) / tt2);
  p->sww2 = (int32_t)round_up(p->nw2 + (span2 + 7 + 2) / 2 + 6, 4);
  const int64_t last_t0 = (int64_t)(p->ntile2 - 1) * tt2;
  // uint16 path reads [base, base + 2 sww2) with base <= t0 + 15; int32 path
  // reads [t0 + emin, + tt2 + span2 + 16)
  p->Pp = round_up(std::max<int64_t>(last_t0 + 16 + 2 * (int64_t)p->sww2, last_t0 + 16 + tt2 + span2 + 16) + 16, 64);
  if (p->pipe2) {
    // per stage: even and odd slots of sww2 words per sub-band, and the address table
    int32_t sc = nsub;
    while (sc > 1 && stage2_pipe_smem(sc, p->sww2) > kSmemMax - 1024) --sc;
    p->nsub_chunk2 = stage2_pipe_smem(sc, p->sww2) <= kSmemMax - 1024 ? sc : 0;
  } else if (p->interm == TX_INTERM_U16 || p->interm == TX_INTERM_F16) {
    // two buffers of a group's delays, double-buffered even copy + odd copy + address table
    p->e2w2 = (int32_t)round_up((int64_t)G * nsub, 4);
    const int64_t per_sub = 3 * (int64_t)p->sww2 * 4 + (int64_t)kStage2MaxGroup * 4 + 8;
    p->nsub_chunk2 = (int32_t)std::min<int64_t>(nsub, (kSmemMax - 1024 - 8 * (int64_t)p->e2w2) / per_sub);
  } else {
    p->sw2_i32 = (int32_t)(tt2 + span2 + 16);
    const int64_t per_sub = (int64_t)p->sw2_i32 * 4 + (int64_t)kStage2MaxGroup * 4 + 8;
    p->nsub_chunk2 = (int32_t)std::min<int64_t>(nsub, (kSmemMax - 1024) / per_sub);
  }
  if (p->nsub_chunk2 < 1) { set_error("stage-2 delay spread within a DM group (%d samples) too large; use a smaller group", span2); return TX_ERR_UNSUPPORTED; }
  if (p->pipe2) {
    // offsets of every (fine DM, sub-band) from its sub-band's staged row start,
    // which is the tile start plus the group's first (smallest) delay rounded
    // down to 8 elements; tiles start at multiples of 1024
    const int SC = p->nsub_chunk2, SCq = (SC + 3) & ~3, nch = (nsub + SC - 1) / SC;
    p->tab2.assign((size_t)nk * nch * (G + 1) * SCq, 0);
    for (int k = 0; k < nk; ++k)
      for (int ch = 0; ch < nch; ++ch) {
        int32_t* blk = p->tab2.data() + ((size_t)k * nch + ch) * (G + 1) * SCq;
        for (int ss = 0; ss < SC && ch * SC + ss < nsub; ++ss) {
          const int s = ch * SC + ss;
          const int32_t start = p->e2[(size_t)k * G * nsub + s] & ~7;
          blk[(size_t)G * SCq + ss] = start;
          for (int g = 0; g < G && k * G + g < ndm; ++g)
            blk[(size_t)g * SCq + ss] = p->e2[(size_t)(k * G + g) * nsub + s] - start;
        }
      }
  }
  p->Dp = round_up(p->Td + 8, 8);
  // boxcar units: the longest of 4, 2 or 1 kBoxTile sub-tiles that still gives
  // every resident block of a full GPU several units (longer units spend less
  // on the scan's barriers, the copy hand-off and the look-ahead)
  p->box_tile = kBoxTile;
  if (d->tile_box) {
    if (d->tile_box != kBoxTile && d->tile_box != 2 * kBoxTile && d->tile_box != 4 * kBoxTile) {
      set_error("tile_box must be 0, %d, %d or %d", kBoxTile, 2 * kBoxTile, 4 * kBoxTile);
      return TX_ERR_INVALID_ARG;
    }
    p->box_tile = d->tile_box;
  }
  for (int f = 4; f > 1 && !d->tile_box; f /= 2) {
    const int64_t units = (int64_t)p->ndm * ((p->T + (int64_t)f * kBoxTile - 1) / ((int64_t)f * kBoxTile));
    if (units >= kBoxMinUnits) { p->box_tile = f * kBoxTile; break; }
  }
  p->ntile3 = (int32_t)((p->T + p->box_tile - 1) / p->box_tile);
  p->ntile2f = p->ntile2;   // the float path's stage 2 uses the same tiles (2 nw2 outputs)

  // ---- stage-1 work list ----------------------------------------------------
  // quarter length q1: the largest of 256/128/64/32 whose staged words, raw
  // prefetch buffer and address table fit in shared memory
  int q1 = 256;
  if (d->tile_q1) {
    if (d->tile_q1 != 32 && d->tile_q1 != 64 && d->tile_q1 != 128 && d->tile_q1 != 256) { set_error("tile_q1 must be 0, 32, 64, 128 or 256"); return TX_ERR_INVALID_ARG; }
    q1 = d->tile_q1;
    if (stage1_smem_bytes(m, q1) > kSmemMax) { set_error("tile_q1 %d does not fit shared memory with %d channels per sub-band", q1, m); return TX_ERR_UNSUPPORTED; }
  }
  while (q1 > 32 && stage1_smem_bytes(m, q1) > kSmemMax) q1 /= 2;
  if (stage1_smem_bytes(m, q1) > kSmemMax) { set_error("too many channels per sub-band for stage 1 (%d)", m); return TX_ERR_UNSUPPORTED; }
  p->q1 = q1;
  p->span1_max = q1 - 16;
  const int64_t tt1 = 4 * (int64_t)q1;
  // every window start of an execute is (head - L) mod R with head a multiple
  // of 64 plus a multiple of T, and R a multiple of 64
  p->tab1_phase = (int32_t)((16 - p->L % 16) % 16);
  const int TS1 = (m + 3) & ~3, SW1 = kStage1StagedWords(q1);
  p->tab1.clear();
  for (int s = 0; s < nsub; ++s) {
    int kb = 0;
    while (kb < nk) {
      auto spread = [&](int k0, int k1) {  // max_c d1[k1-1][c] - d1[k0][c]
        int32_t v = 0;
        for (int c = s * m; c < (s + 1) * m; ++c)
          v = std::max(v, p->d1[(size_t)(k1 - 1) * nchan + c] - p->d1[(size_t)k0 * nchan + c]);
        return v;
      };
      int ke = kb + 1;
      while (ke < nk && ke - kb < kStage1MaxCoarse && spread(kb, ke + 1) <= p->span1_max) ++ke;
      // 16, 32 or 64 coarse DMs keep the 32 warps evenly busy (two, one or half a warp per DM)
      if (ke - kb >= 32) ke = kb + (ke - kb) / 32 * 32;
      else if (ke - kb >= 16) ke = kb + 16;
      const int32_t span = spread(kb, ke);
      int64_t lo = INT64_MAX, hi = 0;
      for (int k = kb; k < ke; ++k) {
        lo = std::min<int64_t>(lo, p->abase[(size_t)k * nsub + s]);
        hi = std::max<int64_t>(hi, (int64_t)p->abase[(size_t)k * nsub + s] + p->Pp);
      }
      const int32_t toff = (int32_t)p->tab1.size();
      for (int kk = 0; kk < ke - kb; ++kk)
        for (int c = 0; c < TS1; ++c) {
          if (c >= m) { p->tab1.push_back(0); continue; }
          const int32_t d0 = p->d1[(size_t)kb * nchan + s * m + c];
          p->tab1.push_back(c * SW1 + ((p->tab1_phase + d0) & 15) + p->d1[(size_t)(kb + kk) * nchan + s * m + c] - d0);
        }
      for (int kk = 0; kk < ((ke - kb + 3) & ~3); ++kk)   // the coarse DMs' P-row bases
        p->tab1.push_back(kk < ke - kb ? p->abase[(size_t)(kb + kk) * nsub + s] : 0);
      for (int64_t t0 = floor_div(lo, tt1) * tt1; t0 < hi; t0 += tt1)
        p->items1.push_back(Stage1Item{s, kb, ke, (int32_t)t0, span, toff, 0, 0});
      kb = ke;
    }
  }
  // Time-major order: blocks working at the same time read overlapping input
  // windows of every sub-band, which keeps the ring's working set in L2.
  std::stable_sort(p->items1.begin(), p->items1.end(), [](const Stage1Item& a, const Stage1Item& b) {
    return a.tau0 != b.tau0 ? a.tau0 < b.tau0 : (a.s != b.s ? a.s < b.s : a.kb < b.kb);
  });
  if (p->interm == TX_INTERM_F32) {
    // float path stage 1: items of `tile_f` times whose coarse DMs' delay spread in
    // the sub-band is at most span_f, the largest of four shapes whose staged
    // float windows (tile + spread + 4 per channel) fit shared memory
    const int shapes[4][2] = {{256, 240}, {128, 112}, {64, 48}, {32, 16}};
    int si = 0;
    while (si < 3 && (int64_t)m * (shapes[si][0] + shapes[si][1] + 4) * 4 > kSmemMax - 2048) ++si;
    p->tile_f = shapes[si][0];
    p->span_f = shapes[si][1];
    for (int s = 0; s < nsub; ++s) {
      int kb = 0;
      while (kb < nk) {
        auto spread = [&](int k0, int k1) {
          int32_t v = 0;
          for (int c = s * m; c < (s + 1) * m; ++c)
            v = std::max(v, p->d1[(size_t)(k1 - 1) * nchan + c] - p->d1[(size_t)k0 * nchan + c]);
          return v;
        };
        int ke = kb + 1;
        while (ke < nk && ke - kb < kStage1MaxCoarse && spread(kb, ke + 1) <= p->span_f) ++ke;
        int64_t lo = INT64_MAX, hi = 0;
        for (int k = kb; k < ke; ++k) {
          lo = std::min<int64_t>(lo, p->abase[(size_t)k * nsub + s]);
          hi = std::max<int64_t>(hi, (int64_t)p->abase[(size_t)k * nsub + s] + p->Pp);
        }
        const int32_t span = spread(kb, ke);
        for (int64_t t0 = floor_div(lo, p->tile_f) * p->tile_f; t0 < hi; t0 += p->tile_f)
          p->items_f.push_back(Stage1Item{s, kb, ke, (int32_t)t0, span, 0, 0, 0});
        kb = ke;
      }
    }
    std::stable_sort(p->items_f.begin(), p->items_f.end(), [](const Stage1Item& a, const Stage1Item& b) {
      return a.tau0 != b.tau0 ? a.tau0 < b.tau0 : (a.s != b.s ? a.s < b.s : a.kb < b.kb);
    });
  }

  // ---- ring ----------------------------------------------------------------------
  // Each channel is a circular buffer of R bytes; the next block lands at
  // `head` and the samples of an execute's buffer are the L before it and the
  // T of the block. R and the first head are multiples of 64 so a block of a
  // multiple of 64 samples always lands 64-byte aligned. Stage 1's reads past
  // the buffer (tile rounding) wrap onto older samples and only feed sums that
  // stage 2 never reads.
  p->R = round_up(p->L + p->T + 64, 64);
  p->head0 = round_up(p->L, 64) % p->R;

  // ---- sizes ---------------------------------------------------------------------
  const bool fpath = p->interm == TX_INTERM_F32;
  const int64_t psz = p->interm == TX_INTERM_I32 || fpath ? 4 : 2;
  int64_t off = 0;
  p->ws_P = off; off = round_up(off + (int64_t)nk * nsub * p->Pp * psz, 256);
  p->ws_D = off; off = round_up(off + (p->output == TX_OUT_SERIES ? 0 : (int64_t)ndm * p->Dp * 4), 256);
  const int64_t parts = fpath ? (int64_t)p->ntile2f : (int64_t)p->ntile2 * (p->pipe2 ? p->split2 : 1);
  p->ws_part = off; off = round_up(off + (int64_t)ndm * parts * 16, 256);
  // S/N constants per (DM, width); the float path keeps (mu, sigma) per DM in double
  p->ws_const = off; off = round_up(off + std::max<int64_t>((int64_t)ndm * p->nw * (int64_t)sizeof(SnrConst), fpath ? (int64_t)ndm * 16 : 0), 256);
  // half intermediates: per-sub-band offsets; float path: per-channel sums (2 x u64), then (mu, w) as float pairs
  p->ws_hoff = off; off = round_up(off + (p->interm == TX_INTERM_F16 ? (int64_t)(nsub + 1) * 4 : fpath ? (int64_t)nchan * 24 : 0), 256);
  // the stage-1 item counter of an execute
  p->ws_ctr = off; off = round_up(off + 4, 256);
  p->ws_bytes = off;
  switch (p->output) {
    case TX_OUT_CANDS: p->out_bytes = p->max_cands * (int64_t)sizeof(tx_cand); break;
    case TX_OUT_PLANE: p->out_bytes = (int64_t)ndm * p->T * 5; break;
    case TX_OUT_CUBE: p->out_bytes = (int64_t)ndm * p->nw * p->T * 4; break;
    default: p->out_bytes = (int64_t)ndm * p->Td * 4; break;
  }
  p->esz = fpath ? 4 : 1;   // the beam's buffer holds normalised float32 samples on the float path
  p->beam_bytes = (int64_t)nchan * p->R * p->esz + (int64_t)ndm * 16 + 16;
  p->tail_pad = (16 - p->L % 16) % 16;
  p->tail_pitch = p->L + p->tail_pad;
  p->ws_ring = p->ws_bytes;
  p->ws_bytes_compact = round_up(p->ws_ring + (int64_t)nchan * p->R, 256);
  p->compact_beam_bytes = (int64_t)nchan * p->tail_pitch + (int64_t)ndm * 16 + 16;
  p->export_bytes = 64 + (int64_t)nchan * p->L * p->esz + (int64_t)ndm * 16;
  return TX_OK;
}

}  // namespace tx

using namespace tx;

extern "C" {

int32_t tx_version(void) { return 300; }

int32_t tx_set_wait_polls(int64_t polls, int64_t* previous) {
  if (polls < 0 || polls > (int64_t)kWaitPolls) { set_error("polls must be in [0, %u]", kWaitPolls); return TX_ERR_INVALID_ARG; }
  const uint32_t old = g_first_wait_polls.exchange((uint32_t)polls);
  if (previous) *previous = old;
  return TX_OK;
}

int32_t tx_last_error(char* buf, size_t size) {
  const std::string& e = g_last_error;
  if (buf && size) {
    const size_t n = std::min(size - 1, e.size());
    std::memcpy(buf, e.data(), n);
    buf[n] = 0;
  }
  return (int32_t)e.size();
}

int32_t tx_plan_create(const tx_plan_desc* desc, tx_plan** out) {
  if (!desc || !out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  tx_plan* p = new (std::nothrow) tx_plan();
  if (!p) { set_error("out of host memory"); return TX_ERR_OOM; }
  int rc;
  try {
    rc = build(p, desc);
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    rc = TX_ERR_OOM;
  }
  if (rc != TX_OK) { delete p; return rc; }
  *out = p;
  return TX_OK;
}

int32_t tx_plan_get_info(const tx_plan* p, tx_plan_info* info) {
  if (!p || !info) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  std::memset(info, 0, sizeof(*info));
  info->nchan = p->nchan; info->nsub = p->nsub; info->ndm = p->ndm; info->ncoarse = p->nk;
  info->group = p->group; info->nwidth = p->nw; info->wmax = p->wmax;
  info->nsamp = p->T; info->overlap = p->L; info->max_delay = p->max_delay; info->series_len = p->Td;
  info->workspace_bytes = p->ws_bytes; info->beam_state_bytes = p->beam_bytes;
  info->out_bytes = p->out_bytes; info->export_bytes = p->export_bytes;
  info->block_bytes = (int64_t)p->nchan * p->T;
  info->ring_len = p->R;
  info->ring_head0 = p->head0;
  info->tile_q1 = p->q1;
  info->tile_split2 = p->split2;
  info->tile_box = p->box_tile;
  info->workspace_bytes_compact = p->ws_bytes_compact;
  info->compact_beam_state_bytes = p->compact_beam_bytes;
  return TX_OK;
}

int32_t tx_plan_tables(const tx_plan* p, int32_t* d1, int32_t* d2, int32_t* coarse_of_fine, double* coarse_dm) {
  if (!p) { set_error("null plan"); return TX_ERR_INVALID_ARG; }
  if (d1) std::memcpy(d1, p->d1.data(), p->d1.size() * 4);
  if (d2) std::memcpy(d2, p->d2.data(), p->d2.size() * 4);
  if (coarse_of_fine) std::memcpy(coarse_of_fine, p->kof.data(), p->kof.size() * 4);
  if (coarse_dm) std::memcpy(coarse_dm, p->coarse_dm.data(), p->coarse_dm.size() * 8);
  return TX_OK;
}

int32_t tx_geometric_widths(double ratio, int32_t wmax, int32_t* h_widths, int32_t cap) {
  if (!(ratio > 1.0) || wmax < 1 || cap < 0 || (cap > 0 && !h_widths)) { set_error("need ratio > 1, wmax >= 1"); return TX_ERR_INVALID_ARG; }
  int32_t n = 0, last = 0;
  double w = 1.0;
  while (true) {
    const int32_t iw = (int32_t)std::floor(w + 0.5);
    if (iw > wmax) break;
    if (iw != last) {
      if (n < cap) h_widths[n] = iw;
      ++n;
      last = iw;
    }
    w *= ratio;
  }
  return n;
}

int32_t tx_plan_segments(int32_t nchan, const double* freq_mhz, double tsamp_s, int32_t ndm, const double* dm,
                         int32_t f_max, int32_t* h_factor) {
  if (nchan < 2 || !freq_mhz || !(tsamp_s > 0.0) || ndm < 1 || !dm || f_max < 1 || !h_factor) {
    set_error("need >= 2 channels, tsamp > 0, >= 1 DM, f_max >= 1 and an output array");
    return TX_ERR_INVALID_ARG;
  }
  // lowest channel: its centre and the spacing to the next one give its edges
  std::vector<double> f(freq_mhz, freq_mhz + nchan);
  std::sort(f.begin(), f.end());
  const double width = f[1] - f[0];
  const double lo = f[0] - width / 2.0, hi = f[0] + width / 2.0;
  if (!(lo > 0.0) || !(width > 0.0)) { set_error("channel frequencies must be distinct and positive"); return TX_ERR_INVALID_ARG; }
  for (int i = 0; i < ndm; ++i) {
    // Eq. 1 across the channel, in samples; the largest power of two not above it
    const double smear = kDispersion * dm[i] * (1.0 / (lo * lo) - 1.0 / (hi * hi)) / tsamp_s;
    int32_t fac = 1;
    while ((double)(fac * 2) <= smear && fac * 2 <= f_max) fac *= 2;
    h_factor[i] = fac;
  }
  return TX_OK;
}

}  // extern "C"

struct tx_dsplan {
  int64_t T = 0, L = 0;
  std::vector<tx_segment> seg;
  std::vector<tx_plan*> plans;
  ~tx_dsplan() {
    for (tx_plan* p : plans) tx_plan_destroy(p);
  }
};

extern "C" {

int32_t tx_dsplan_create(const tx_plan_desc* desc, int32_t f_max, tx_dsplan** out) {
  if (!desc || !out || f_max < 1) { set_error("need a plan description, f_max >= 1 and an output handle"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  if (desc->nsamp < 1 || desc->ndm < 1 || !desc->dm || !desc->widths || desc->nwidth < 1) {
    set_error("need nsamp >= 1, ndm >= 1 and DM and width tables");
    return TX_ERR_INVALID_ARG;
  }
  // a factor must divide the block: f_max drops to the largest power of two dividing T
  int32_t fdiv = 1;
  while (desc->nsamp % ((int64_t)fdiv * 2) == 0 && fdiv * 2 <= f_max) fdiv *= 2;
  std::vector<int32_t> fac(desc->ndm);
  int rc = tx_plan_segments(desc->nchan, desc->freq_mhz, desc->tsamp_s, desc->ndm, desc->dm, fdiv, fac.data());
  if (rc) return rc;
  tx_dsplan* ds = new (std::nothrow) tx_dsplan();
  if (!ds) { set_error("out of host memory"); return TX_ERR_OOM; }
  ds->T = desc->nsamp;
  try {
    int a = 0;
    for (int i = 1; i <= desc->ndm; ++i) {
      if (i < desc->ndm && fac[i] == fac[a]) continue;
      const int32_t f = fac[a];
      // widths in downsampled samples: W / f, at least 1, duplicates dropped
      std::vector<int32_t> w;
      for (int k = 0; k < desc->nwidth; ++k) w.push_back(std::max(1, desc->widths[k] / f));
      std::sort(w.begin(), w.end());
      w.erase(std::unique(w.begin(), w.end()), w.end());
      tx_plan_desc d = *desc;
      d.tsamp_s = desc->tsamp_s * f;
      d.ndm = i - a;
      d.dm = desc->dm + a;
      d.nwidth = (int32_t)w.size();
      d.widths = w.data();
      d.nsamp = desc->nsamp / f;
      tx_plan* p = nullptr;
      if ((rc = tx_plan_create(&d, &p))) break;
      ds->plans.push_back(p);
      tx_segment sg{};
      sg.dm_lo = a;
      sg.dm_hi = i;
      sg.factor = f;
      sg.nwidth = d.nwidth;
      for (int k = 0; k < d.nwidth; ++k) sg.widths[k] = w[k];
      sg.nsamp = d.nsamp;
      sg.overlap = p->L;
      ds->seg.push_back(sg);
      ds->L = std::max(ds->L, (int64_t)f * p->L);
      a = i;
    }
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    rc = TX_ERR_OOM;
  }
  if (rc) { delete ds; return rc; }
  // native window time of a segment's output t' is f t' + L - f L_j
  for (tx_segment& sg : ds->seg) sg.native_offset = ds->L - (int64_t)sg.factor * sg.overlap;
  *out = ds;
  return TX_OK;
}

int32_t tx_dsplan_get_info(const tx_dsplan* ds, int32_t* nseg, int64_t* overlap) {
  if (!ds) { set_error("null plan"); return TX_ERR_INVALID_ARG; }
  if (nseg) *nseg = (int32_t)ds->seg.size();
  if (overlap) *overlap = ds->L;
  return TX_OK;
}

int32_t tx_dsplan_segment(const tx_dsplan* ds, int32_t j, tx_segment* seg, const tx_plan** plan) {
  if (!ds || j < 0 || j >= (int32_t)ds->seg.size()) { set_error("no segment %d", j); return TX_ERR_INVALID_ARG; }
  if (seg) *seg = ds->seg[j];
  if (plan) *plan = ds->plans[j];
  return TX_OK;
}

void tx_dsplan_destroy(tx_dsplan* ds) { delete ds; }

int32_t tx_plan_delay_table(const tx_plan* p, double* h_delay_ms) {
  if (!p || !h_delay_ms) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  std::memcpy(h_delay_ms, p->delay_ms.data(), p->delay_ms.size() * sizeof(double));
  return TX_OK;
}

int32_t tx_plan_stage1_layout(const tx_plan* p, int64_t* p_offset, int64_t* p_pitch, int32_t* h_base) {
  if (!p) { set_error("null plan"); return TX_ERR_INVALID_ARG; }
  if (p_offset) *p_offset = p->ws_P;
  if (p_pitch) *p_pitch = p->Pp;
  if (h_base) std::memcpy(h_base, p->abase.data(), p->abase.size() * 4);
  return TX_OK;
}

}  // extern "C"
