"""Pins of the normalisation oracle (Sec. 2.1), CPU only.

Exact values on channels whose statistics are known by construction, the
library-free definition of the moments, unit variance on noise, and the
purpose the paper gives the reciprocal-variance weights: with channels of
unequal noise, weights 1 / sigma^2 give the textbook optimal S/N of a weighted
sum, amp * sqrt(sum 1 / sigma_c^2), which beats unit-variance weights and raw
equal weights by the Cauchy-Schwarz margins computed here from first
principles.
"""
import math

import numpy as np
import pytest

from oracle import dedisp as O
from oracle import normalise as NM


def test_two_valued_and_constant_channels_exact():
    T = 1024
    X = np.zeros((3, T), dtype=np.uint8)
    X[0, 0::2], X[0, 1::2] = 100, 132          # mean 116, sigma 16 exactly
    X[1, :] = 77                               # constant: sigma 0
    X[2, 0::2], X[2, 1::2] = 0, 255            # mean 127.5, sigma 127.5
    mu, var = NM.channel_moments(X)
    assert mu.tolist() == [116.0, 77.0, 127.5] and var.tolist() == [256.0, 0.0, 127.5 ** 2]
    u = NM.normalise_block(X, "unit")
    assert set(u[0].tolist()) == {-1.0, 1.0} and not u[1].any()
    assert np.allclose(u[2], np.where(X[2] == 0, -1.0, 1.0), atol=1e-7)
    v = NM.normalise_block(X, "invvar")
    assert set(v[0].tolist()) == {-1.0 / 16, 1.0 / 16} and not v[1].any()


def test_moments_equal_plain_definition():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 256, size=(5, 3001), dtype=np.uint8)
    mu, var = NM.channel_moments(X)
    for c in range(5):
        xs = [int(v) for v in X[c]]
        m = sum(xs) / len(xs)
        assert mu[c] == pytest.approx(m, rel=1e-15)
        assert var[c] == pytest.approx(sum((x - m) ** 2 for x in xs) / len(xs), rel=1e-12)


@pytest.mark.parametrize("norm", ["unit", "invvar"])
def test_noise_channels_zero_mean_and_their_variance(norm):
    rng = np.random.default_rng(2)
    sig = np.array([3.0, 6.0, 12.0, 24.0])
    X = np.clip(np.rint(128.0 + sig[:, None] * rng.standard_normal((4, 1 << 16))), 0, 255).astype(np.uint8)
    mu, var = NM.channel_moments(X)
    Xn = NM.normalise_block(X, norm).astype(np.float64)
    assert np.all(np.abs(Xn.mean(axis=1)) < 1e-5)
    want = np.ones(4) if norm == "unit" else 1.0 / var
    assert np.allclose(Xn.var(axis=1), want, rtol=1e-5)


def test_reciprocal_variance_weights_reach_the_matched_snr():
    """64 channels with noise sigma from 3 to 30 counts, one flat pulse of 6
    counts in every channel at t0 (DM 0): the boxcar S/N (W = 1) of the summed
    normalised channels is the weighted-sum S/N sum_c w_c a / sqrt(sum_c w_c^2
    sigma_c^2), i.e. a sqrt(sum 1/sigma_c^2) for w = 1/sigma^2, a sum(1/sigma_c)
    / sqrt(N) for w = 1/sigma and a N / sqrt(sum sigma_c^2) for raw data, within
    the noise of one sample (about 1 in S/N units)."""
    rng = np.random.default_rng(3)
    nch, T, t0, amp = 64, 1 << 16, 40000, 6.0
    sig = np.linspace(3.0, 30.0, nch)
    X = np.clip(np.rint(128.0 + sig[:, None] * rng.standard_normal((nch, T))), 0, 255)
    X[:, t0] += amp
    X = X.astype(np.uint8)
    # the textbook S/N of each weighting, from the noise levels alone
    want = {"invvar": amp * math.sqrt(float((1.0 / sig ** 2).sum())),
            "unit": amp * float((1.0 / sig).sum()) / math.sqrt(nch),
            "raw": amp * nch / math.sqrt(float((sig ** 2).sum()))}
    got = {}
    for norm in ("invvar", "unit", "raw"):
        Xn = X.astype(np.float64) if norm == "raw" else NM.normalise_block(X, norm).astype(np.float64)
        D = Xn.sum(axis=0)[None, :]
        _, _, mu, sg = O.block_stats(D, T)
        got[norm] = float(O.boxcar_snr(D, [1], T, mu, sg)[0, 0, t0])
        assert got[norm] == pytest.approx(want[norm], abs=3.0), (norm, got[norm], want[norm])
    assert want["invvar"] > 1.15 * want["unit"] > 1.15 * 1.15 * want["raw"]
    assert got["invvar"] > got["unit"] > got["raw"]


def test_stream_keeps_each_blocks_normalisation():
    rng = np.random.default_rng(4)
    L, T = 50, 200
    X = rng.integers(0, 256, size=(3, L + 2 * T), dtype=np.uint8)
    S = NM.normalised_stream(X, L, T, 2, "unit")
    assert np.array_equal(S[:, :L], NM.normalise_block(X[:, :L], "unit"))
    assert np.array_equal(S[:, L + T:], NM.normalise_block(X[:, L + T:], "unit"))
    Y = X.copy()
    Y[:, L + T:] = 255 - Y[:, L + T:]                 # a different second block leaves the first one alone
    assert np.array_equal(NM.normalised_stream(Y, L, T, 2, "unit")[:, :L + T], S[:, :L + T])


def test_sum_error_bound_covers_float32_sums():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((1000, 64)).astype(np.float32)
    exact = v.astype(np.float64).sum(axis=1)
    acc = np.zeros(1000, dtype=np.float32)
    for i in range(64):
        acc = acc + v[:, i]                      # float32 recursive summation
    bound = NM.sum_error_bound(np.abs(v.astype(np.float64)).sum(axis=1), 64)
    assert np.all(np.abs(acc.astype(np.float64) - exact) <= bound)
