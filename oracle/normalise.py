"""Oracle: per-channel normalisation of each block (Sec. 2.1).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU legs
use this module; the library never does.

The paper brings every block to zero mean and unit variance in each channel
before de-dispersing it, and notes that reweighting by the reciprocal of the
variance damps channels with outliers. Readings used here (the paper gives
no formulas):

* mu_c and sigma_c are the mean and population standard deviation of channel
  c over the block's T new samples, from exact integer sums;
* unit-variance normalisation: x' = (x - mu_c) / sigma_c; inverse-variance
  weighting: x' = (x - mu_c) / sigma_c^2; a channel with sigma_c = 0 gets
  weight 0 (it carries no information);
* a block is normalised once, as it arrives: the carried overlap keeps the
  normalisation of the block it came with (the primed first overlap is a
  block of its own);
* x' is formed in float32 exactly as the library stores it,
  x' = (float32(x) - float32(mu_c)) * float32(w_c), w_c = 1 / sigma_c or
  1 / sigma_c^2 rounded from double; each float32 operation rounds to
  nearest, so this is a definition, not an approximation of one.

De-dispersion and the boxcar then follow oracle.dedisp on the float32
values, summed in float64.
"""
from __future__ import annotations

import math

import numpy as np

NORMS = ("unit", "invvar")


def channel_moments(Xb: np.ndarray):
    """Mean and population variance of each channel (rows of Xb) from exact
    integer sums: mu = S1 / T, var = (T S2 - S1^2) / T^2."""
    T = Xb.shape[1]
    x = np.asarray(Xb, dtype=np.int64)
    S1 = x.sum(axis=1)                       # exact: T * 255 < 2^63
    S2 = (x * x).sum(axis=1)                 # exact: T * 255^2 < 2^63
    mu = np.zeros(Xb.shape[0], dtype=np.float64)
    var = np.zeros(Xb.shape[0], dtype=np.float64)
    for c in range(Xb.shape[0]):
        s1, s2 = int(S1[c]), int(S2[c])
        mu[c] = s1 / T                       # Python ints: correctly rounded
        var[c] = (T * s2 - s1 * s1) / (T * T)
    return mu, var


def weights(var: np.ndarray, norm: str) -> np.ndarray:
    """w_c = 1 / sigma_c (unit variance) or 1 / sigma_c^2 (inverse variance); 0 where sigma_c = 0."""
    w = np.zeros_like(var)
    pos = var > 0.0
    if norm == "unit":
        w[pos] = 1.0 / np.sqrt(var[pos])
    elif norm == "invvar":
        w[pos] = 1.0 / var[pos]
    else:
        raise ValueError(norm)
    return w


def normalise_block(Xb: np.ndarray, norm: str) -> np.ndarray:
    """x' of one block (uint8 [nchan, T]) with its own statistics, float32."""
    mu, var = channel_moments(Xb)
    mu32 = mu.astype(np.float32)[:, None]
    w32 = weights(var, norm).astype(np.float32)[:, None]
    return (Xb.astype(np.float32) - mu32) * w32


def normalised_stream(X: np.ndarray, L: int, T: int, nblocks: int, norm: str) -> np.ndarray:
    """The float32 data a beam holds: the first L samples normalised as a block
    of their own, then every block of T samples with its own statistics."""
    out = np.zeros((X.shape[0], L + nblocks * T), dtype=np.float32)
    if L:
        out[:, :L] = normalise_block(X[:, :L], norm)
    for b in range(nblocks):
        a = L + b * T
        out[:, a:a + T] = normalise_block(X[:, a:a + T], norm)
    return out


def sum_error_bound(Xn_abs_sums: np.ndarray, n_terms: int) -> np.ndarray:
    """First-order bound on the rounding error of a float32 sum done in any
    order as nested sums of at most n_terms terms: gamma_n * sum |terms|,
    gamma_n = n u / (1 - n u), u = 2^-24 (recursive summation)."""
    u = 2.0 ** -24
    g = n_terms * u / (1.0 - n_terms * u)
    return g * Xn_abs_sums
