"""Oracle for de-dispersion plans with downsampling (Sec. 2.3, last paragraph).

Test infrastructure: only tests, the smoke check and the benchmark's CPU legs
use this module; the library never does.

The paper notes that at high DM the smearing inside one channel exceeds the
sampling time, and that a de-dispersion plan may therefore downsample the
data before de-dispersing in several DM ranges. It gives no rule; the reading
used here:

* the smearing of DM d is the Eq. 1 delay across the lowest-frequency
  channel (its edges at centre -+ width / 2), in native samples;
* DM trial d is de-dispersed after downsampling by f(d), the largest power of
  two not above that smearing (at least 1, at most f_max);
* consecutive DM trials with the same factor form a segment, de-dispersed
  with sampling time f t_samp on blocks of T / f samples; a segment's widths
  are W / f (integer division, at least 1, duplicates dropped), so the
  physical widths are kept where they are resolved;
* downsampling averages f consecutive samples of each channel and rounds half
  up, so the data stay uint8: x'[t] = (sum_{i<f} x[f t + i] + f / 2) // f.
"""
from __future__ import annotations

import math

import numpy as np

K_DM = 4.148808e3   # s MHz^2 pc^-1 cm^3 (Eq. 1)


def channel_smear_samples(dms, freqs_mhz, tsamp_s) -> np.ndarray:
    """Eq. 1 delay across the lowest channel (edges centre -+ width/2), in samples."""
    f = np.sort(np.asarray(freqs_mhz, dtype=np.float64))
    width = f[1] - f[0]
    lo, hi = f[0] - width / 2.0, f[0] + width / 2.0
    return K_DM * np.asarray(dms, dtype=np.float64) * (1.0 / (lo * lo) - 1.0 / (hi * hi)) / tsamp_s


def factor_of(smear_samples: float, f_max: int) -> int:
    """Largest power of two <= smear (at least 1, at most f_max)."""
    f = 1
    while f * 2 <= smear_samples and f * 2 <= f_max:
        f *= 2
    return f


def segments(dms, freqs_mhz, tsamp_s, widths, f_max=64):
    """[(first DM index, end DM index, factor, widths of the segment)] in DM order."""
    s = channel_smear_samples(dms, freqs_mhz, tsamp_s)
    fac = [factor_of(float(v), f_max) for v in s]
    out = []
    a = 0
    for i in range(1, len(fac) + 1):
        if i == len(fac) or fac[i] != fac[a]:
            f = fac[a]
            w = sorted({max(1, int(W) // f) for W in widths})
            out.append((a, i, f, w))
            a = i
    return out


def downsample(X: np.ndarray, f: int) -> np.ndarray:
    """uint8 [nchan, n // f]: each channel's f-sample means rounded half up."""
    n = X.shape[1] // f
    s = np.asarray(X[:, :n * f], dtype=np.int64).reshape(X.shape[0], n, f).sum(axis=2)
    return ((s + f // 2) // f).astype(np.uint8)
