"""Oracle: de-dispersion (Sec. 2.3) and boxcar matched filtering (Sec. 2.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper and its sub-band scheme:

  X[c][j]      uint8 samples of channel c, j in [0, T + L): a block of T new
               samples preceded by the overlap L carried from the previous
               block (Sec. 2.3 data flow, steps 1-4).
  D[d][t]      de-dispersed series of fine DM trial d; t is the arrival time at
               the reference frequency f_ref, t in [0, T + W_max - 1).
  P[k][s][t]   stage-1 sum of sub-band s at coarse DM k.
  S/N[d][w][t] boxcar S/N of width W_w starting at t, t in [0, T).

Readings of the paper used here (each is listed with its reason in the
design notes):
  * f_ref = the highest channel centre, so every delay is >= 0.
  * delays are rounded half away from zero (C ``llround``) after evaluating
    K * DM * (1/f^2 - 1/f_ref^2) / t_samp in that order, in IEEE double.
  * sub-band s = channels [s m, (s+1) m); its reference f_ref,s = the highest
    centre inside it; fine DMs are grouped G at a time, in order, and the
    coarse DM of a group is the midpoint of its first and last fine DM.
  * stage 2 shifts each sub-band by the delay of the *fine* DM between
    f_ref,s and f_ref.
  * a boxcar of width W covers [t, t + W) and is reported at its start t.
  * mu and sigma are the population mean and standard deviation of D[d][t]
    over this block's t in [0, T); sigma = 0 gives S/N = 0.
"""
from __future__ import annotations

import math

import numpy as np

# Eq. 1 constant e^2 / (2 pi m_e c) in s MHz^2 pc^-1 cm^3.
K_DM = 4.148808e3


# ----------------------------------------------------------------------------
# Eq. 1: cold-plasma delay in samples
# ----------------------------------------------------------------------------
def rnd(x: float) -> int:
    """Round half away from zero, like C llround (x - trunc(x) is exact)."""
    t = math.trunc(x)
    frac = x - t
    if frac >= 0.5:
        t += 1
    elif frac <= -0.5:
        t -= 1
    return int(t)


def rnd_array(x: np.ndarray) -> np.ndarray:
    """Element-wise ``rnd`` of a float64 array -> int64."""
    x = np.asarray(x, dtype=np.float64)
    t = np.trunc(x)
    frac = x - t
    t = t + (frac >= 0.5) - (frac <= -0.5)
    return t.astype(np.int64)


def delay_seconds(dm, f_mhz, f_ref_mhz):
    """Eq. 1: tau = K DM (f^-2 - f_ref^-2), seconds."""
    return K_DM * dm * (1.0 / (f_mhz * f_mhz) - 1.0 / (f_ref_mhz * f_ref_mhz))


def delay_samples(dm, f_mhz, f_ref_mhz, tsamp_s):
    """Eq. 1 in samples: rnd(K * DM * (1/f^2 - 1/f_ref^2) / t_samp)."""
    v = K_DM * np.asarray(dm, dtype=np.float64) * (
        1.0 / (np.asarray(f_mhz, dtype=np.float64) * np.asarray(f_mhz, dtype=np.float64))
        - 1.0 / (f_ref_mhz * f_ref_mhz)) / tsamp_s
    return rnd_array(v)


def _acc_dtype(X) -> type:
    """int64 sums for integer samples, float64 for float (noise-free model) input."""
    return np.int64 if np.issubdtype(np.asarray(X).dtype, np.integer) else np.float64


# ----------------------------------------------------------------------------
# Brute-force (direct) de-dispersion, Sec. 2.3, O(N_DM N_t N_f)
# ----------------------------------------------------------------------------
def direct_delays(freqs, tsamp, dms) -> np.ndarray:
    """dd[d][c] = rnd(K DM_d (f_c^-2 - f_ref^-2) / t_samp), f_ref = max f."""
    freqs = np.asarray(freqs, dtype=np.float64)
    f_ref = float(freqs.max())
    return np.stack([delay_samples(float(dm), freqs, f_ref, tsamp) for dm in dms])


def direct_dedisperse(X: np.ndarray, freqs, tsamp, dms, nout: int) -> np.ndarray:
    """D[d][t] = sum_c X[c][t + dd[d][c]] for t in [0, nout), int64."""
    dd = direct_delays(freqs, tsamp, dms)
    nchan = X.shape[0]
    D = np.zeros((len(dms), nout), dtype=_acc_dtype(X))
    for d in range(len(dms)):
        for c in range(nchan):
            o = int(dd[d, c])
            D[d] += X[c, o:o + nout]
    return D


# ----------------------------------------------------------------------------
# Sub-band de-dispersion plan, Sec. 2.3 and Fig. 3
# ----------------------------------------------------------------------------
def auto_group(freqs, tsamp, nsub, ndm) -> int:
    """Fine DMs per coarse DM when the caller asks for the automatic rule.

    The paper leaves the coarse grid open. Reading: take the largest power of
    two G with G <= 1 + S_full / S_sub, where S_full is the whole-band delay per
    unit DM (f_min to f_ref) and S_sub the largest within-sub-band delay per
    unit DM (lowest to highest centre of a sub-band). Then the smear a coarse
    DM leaves inside a sub-band, (G - 1) / 2 fine steps across S_sub, stays
    below the half-step smear of the fine grid across the whole band. G is also
    capped by the largest power of two <= ndm.
    """
    freqs = np.asarray(freqs, dtype=np.float64)
    nchan = freqs.size
    m = nchan // nsub
    f_ref = float(freqs.max())
    f_min = float(freqs.min())
    s_full = K_DM * (1.0 / (f_min * f_min) - 1.0 / (f_ref * f_ref)) / tsamp
    s_sub = 0.0
    for s in range(nsub):
        fs = freqs[s * m:(s + 1) * m]
        lo, hi = float(fs.min()), float(fs.max())
        v = K_DM * (1.0 / (lo * lo) - 1.0 / (hi * hi)) / tsamp
        s_sub = max(s_sub, v)
    cap = 1
    while cap * 2 <= ndm:
        cap *= 2
    if s_sub <= 0.0:
        return cap
    ratio = 1.0 + s_full / s_sub
    g = 1
    while g * 2 <= ratio and g * 2 <= cap:
        g *= 2
    return g


class SubbandPlan:
    """Tables of the two-stage sub-band scheme (Sec. 2.3, Fig. 3)."""

    def __init__(self, freqs, tsamp, dms, nsub, group=0, widths=(1,)):
        self.freqs = np.asarray(freqs, dtype=np.float64)
        self.tsamp = float(tsamp)
        self.dms = np.asarray(dms, dtype=np.float64)
        self.nchan = self.freqs.size
        self.nsub = int(nsub)
        if self.nchan % self.nsub:
            raise ValueError("nchan must be a multiple of nsub")
        self.m = self.nchan // self.nsub
        self.ndm = self.dms.size
        self.widths = np.asarray(widths, dtype=np.int64)
        self.wmax = int(self.widths.max())
        self.group = int(group) if group else auto_group(self.freqs, self.tsamp, self.nsub, self.ndm)
        G = self.group
        self.nk = (self.ndm + G - 1) // G
        self.f_ref = float(self.freqs.max())
        self.f_ref_s = np.array([self.freqs[s * self.m:(s + 1) * self.m].max() for s in range(self.nsub)])
        self.coarse_of_fine = np.arange(self.ndm) // G
        self.coarse_dm = np.array([
            (self.dms[k * G] + self.dms[min((k + 1) * G, self.ndm) - 1]) / 2.0 for k in range(self.nk)])
        sub_of_chan = np.arange(self.nchan) // self.m
        f_ref_c = self.f_ref_s[sub_of_chan]
        # stage 1: channels -> sub-band reference at the coarse DM
        self.d1 = np.stack([delay_samples(float(dmk), self.freqs, f_ref_c, self.tsamp)
                            for dmk in self.coarse_dm])               # [nk][nchan]
        # stage 2: sub-band reference -> f_ref at the fine DM
        self.d2 = np.stack([delay_samples(float(dm), self.f_ref_s, self.f_ref, self.tsamp)
                            for dm in self.dms])                        # [ndm][nsub]
        # overlap L = max over (d, c) of d1 + d2 + W_max - 1
        best = 0
        for k in range(self.nk):
            ds = slice(k * G, min((k + 1) * G, self.ndm))
            d2max = self.d2[ds].max(axis=0)                              # [nsub]
            best = max(best, int((self.d1[k] + d2max[sub_of_chan]).max()))
        self.max_delay = best
        self.overlap = best + self.wmax - 1

    def fine_dms_of(self, k):
        return range(k * self.group, min((k + 1) * self.group, self.ndm))


def stage1(X: np.ndarray, plan: SubbandPlan, k: int, s: int, n: int) -> np.ndarray:
    """P[k][s][t] = sum_{c in s} X[c][t + d1[k][c]] for t in [0, n), int64."""
    P = np.zeros(n, dtype=_acc_dtype(X))
    for c in range(s * plan.m, (s + 1) * plan.m):
        o = int(plan.d1[k, c])
        P += X[c, o:o + n]
    return P


def subband_dedisperse(X: np.ndarray, plan: SubbandPlan, nout: int, dm_indices=None) -> np.ndarray:
    """Two-stage sub-band de-dispersion (Sec. 2.3):

    (1) each sub-band summed at the coarse DM of the trial's group;
    (2) the sub-band sums shifted by the fine DM's delay and summed.
    Returns D[i][t] for the requested fine DMs (all by default), int64.
    """
    if dm_indices is None:
        dm_indices = range(plan.ndm)
    dm_indices = list(dm_indices)
    D = np.zeros((len(dm_indices), nout), dtype=_acc_dtype(X))
    cache = {}
    for i, d in enumerate(dm_indices):
        k = int(plan.coarse_of_fine[d])
        if k not in cache:
            ds = list(plan.fine_dms_of(k))
            cache.clear()
            cache[k] = [stage1(X, plan, k, s, nout + int(plan.d2[ds, s].max())) for s in range(plan.nsub)]
        P = cache[k]
        for s in range(plan.nsub):
            o = int(plan.d2[d, s])
            D[i] += P[s][o:o + nout]
    return D


def half_offsets(X: np.ndarray, plan: SubbandPlan, block: slice) -> np.ndarray:
    """Integer offset per sub-band for half-precision stage-1 storage:
    o_s = sum over the channels c of s of rnd(mean of X[c] over the block's
    samples), each mean rounded half up (an integer, so subtracting it and
    adding it back is exact). Returns int64 [nsub]."""
    Xb = np.asarray(X[:, block], dtype=np.int64)
    T = Xb.shape[1]
    sums = Xb.sum(axis=1)
    means = (2 * sums + T) // (2 * T)           # rnd(sum / T), half up, for sum >= 0
    return means.reshape(plan.nsub, plan.m).sum(axis=1)


def subband_dedisperse_f16(X: np.ndarray, plan: SubbandPlan, nout: int, block: slice, dm_indices=None):
    """The sub-band scheme of Sec. 2.3 with the stage-1 sums kept at half
    precision (the FP16 form): P'[k][s] = P[k][s] - o_s (o_s from
    half_offsets over `block`) rounded to the nearest FP16 (ties to even),
    saturated at +-65504; stage 2 adds the halves in float64 and then the
    offsets back: D = sum_s (half(P') + o_s). Returns float64 [len(dm)][nout]
    (integer-valued: every FP16 value of an integer is an integer)."""
    if dm_indices is None:
        dm_indices = range(plan.ndm)
    dm_indices = list(dm_indices)
    off = half_offsets(X, plan, block)
    D = np.zeros((len(dm_indices), nout), dtype=np.float64)
    cache = {}
    for i, d in enumerate(dm_indices):
        k = int(plan.coarse_of_fine[d])
        if k not in cache:
            ds = list(plan.fine_dms_of(k))
            cache.clear()
            cache[k] = []
            for s in range(plan.nsub):
                P = stage1(X, plan, k, s, nout + int(plan.d2[ds, s].max())).astype(np.float64)
                h = np.clip(P - float(off[s]), -65504.0, 65504.0).astype(np.float16)
                cache[k].append(h.astype(np.float64))
        for s in range(plan.nsub):
            o = int(plan.d2[d, s])
            D[i] += cache[k][s][o:o + nout]
        D[i] += float(off.sum())
    return D


# ----------------------------------------------------------------------------
# Boxcar matched filter, Sec. 2.4 and Eq. 5
# ----------------------------------------------------------------------------
def block_stats(D: np.ndarray, T: int):
    """Exact S1 = sum D, S2 = sum D^2 over t in [0, T); mean and population std.

    var = (T S2 - S1^2) / T^2 with the numerator an exact integer.
    Returns (S1, S2, mu, sigma) as lists (Python ints / floats).
    """
    S1, S2, mu, sg = [], [], [], []
    D = np.asarray(D)
    if not np.issubdtype(D.dtype, np.integer):
        for row in D[:, :T].astype(np.float64):
            s1, s2 = float(row.sum()), float((row * row).sum())
            S1.append(s1)
            S2.append(s2)
            mu.append(s1 / T)
            sg.append(math.sqrt(max(s2 / T - (s1 / T) ** 2, 0.0)))
        return S1, S2, mu, sg
    for row in D[:, :T]:
        row = row.astype(np.int64)
        peak = int(np.abs(row).max()) if row.size else 0
        if T * peak * peak < 2 ** 62:          # int64 cannot overflow
            s1 = int(row.sum())
            s2 = int((row * row).sum())
        else:                                    # fall back to Python integers
            r = [int(v) for v in row]
            s1 = sum(r)
            s2 = sum(v * v for v in r)
        S1.append(s1)
        S2.append(s2)
        mu.append(s1 / T)
        var = float(T * s2 - s1 * s1) / float(T * T)
        sg.append(math.sqrt(var))
    return S1, S2, mu, sg


def window_sums(row: np.ndarray, W: int, T: int) -> np.ndarray:
    """B_W[t] = sum_{i=t}^{t+W-1} row[i] for t in [0, T) (plain definition)."""
    row = np.asarray(row)
    row = row.astype(_acc_dtype(row))
    B = np.zeros(T, dtype=row.dtype)
    for i in range(W):
        B += row[i:i + T]
    return B


def boxcar_snr(D: np.ndarray, widths, T: int, mu, sigma) -> np.ndarray:
    """Eq. 5: S/N[d][w][t] = (B_W[t] - W mu_d) / (sigma_d sqrt(W)), float64.

    Raw uint8 sums carry a mean of about N_c * 128, so the mean is removed
    (the paper's Eq. 5 assumes data already normalised to zero mean, Sec. 2.1).
    """
    D = np.asarray(D)
    out = np.zeros((D.shape[0], len(widths), T), dtype=np.float64)
    for d in range(D.shape[0]):
        for wi, W in enumerate(widths):
            W = int(W)
            if sigma[d] == 0.0:
                continue
            B = window_sums(D[d], W, T)
            out[d, wi] = (B - W * mu[d]) / (sigma[d] * math.sqrt(W))
    return out


def dm_time_plane(snr: np.ndarray):
    """Sec. 2.5: best S/N over width for each (DM, t); ties go to the smaller width."""
    best_w = np.argmax(snr, axis=1)
    best = np.take_along_axis(snr, best_w[:, None, :], axis=1)[:, 0, :]
    return best, best_w


def candidates(best: np.ndarray, best_w: np.ndarray, gamma: float, dm_indices=None):
    """Points of the DM-time plane with S/N >= gamma: array of (d, t, w, snr)."""
    d_idx, t_idx = np.nonzero(best >= gamma)
    if dm_indices is not None:
        dm_indices = np.asarray(dm_indices)
        dd = dm_indices[d_idx]
    else:
        dd = d_idx
    out = np.zeros(d_idx.size, dtype=[("d", np.int64), ("t", np.int64), ("w", np.int64), ("snr", np.float64)])
    out["d"] = dd
    out["t"] = t_idx
    out["w"] = best_w[d_idx, t_idx]
    out["snr"] = best[d_idx, t_idx]
    return out


def running_stats(prev, mu_b, var_b, lam):
    """Exponential update of (mu, var) across blocks: the first block initialises.

    prev is None or (mu, var); returns (mu, var).
    """
    if prev is None:
        return mu_b, var_b
    mu0, var0 = prev
    return (1.0 - lam) * mu0 + lam * mu_b, (1.0 - lam) * var0 + lam * var_b


# ----------------------------------------------------------------------------
# Blocked stream, Sec. 2.3 data flow (write, transpose, de-disperse, shift)
# ----------------------------------------------------------------------------
def stream_series(stream: np.ndarray, plan: SubbandPlan, T: int, nblocks: int):
    """Run the block loop over a channel-major stream [nchan, L + nblocks*T].

    Block b sees buffer samples [b T, b T + T + L) (its first L samples are the
    previous block's undispersed tail) and yields D over [0, T + W_max - 1).
    """
    L = plan.overlap
    outs = []
    for b in range(nblocks):
        buf = stream[:, b * T:b * T + T + L]
        outs.append(subband_dedisperse(buf, plan, T + plan.wmax - 1))
    return outs
