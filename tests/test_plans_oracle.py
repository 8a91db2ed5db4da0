"""Pins of the downsampling de-dispersion plans' oracle (CPU).

The smearing is Eq. 1 across one channel, checked against hand values; the
factor is the largest power of two not above it; segments and their widths
follow; downsampling is the rounded mean of f samples, checked by hand.
"""
import numpy as np
import pytest

import synth
from oracle import plans as PL


def test_channel_smear_by_hand():
    # lowest channel 1000.5 MHz wide 1 MHz: edges 1000 and 1001 MHz, t_samp 1 ms
    f = np.array([1000.5, 1001.5, 1002.5])
    s = PL.channel_smear_samples([100.0], f, 1e-3)[0]
    assert s == pytest.approx(4.148808e3 * 100 * (1 / 1000.0 ** 2 - 1 / 1001.0 ** 2) / 1e-3, rel=1e-12)
    assert s == pytest.approx(0.8285, abs=1e-4)          # 4.148808e5 x 1.997004e-9 s / 1 ms


def test_factor_powers_of_two():
    assert [PL.factor_of(v, 64) for v in (0.2, 1.0, 1.99, 2.0, 3.9, 4.0, 63.0, 64.0, 1e6)] == \
        [1, 1, 1, 2, 2, 4, 32, 64, 64]
    assert PL.factor_of(1e6, 8) == 8


def test_meerkat_segments():
    wl = synth.meerkat_l_workload()
    segs = PL.segments(wl.dms, wl.freqs_mhz, wl.tsamp_s, wl.widths, f_max=64)
    # contiguous, covering, factors rising with DM
    assert segs[0][0] == 0 and segs[-1][1] == wl.ndm
    assert all(a[1] == b[0] for a, b in zip(segs, segs[1:]))
    assert [s[2] for s in segs] == sorted(s[2] for s in segs)
    # the lowest channel (0.209 MHz at 856.1 MHz) smears one 153.12-us sample at DM ~55
    s55 = PL.channel_smear_samples([55.0], wl.freqs_mhz, wl.tsamp_s)[0]
    assert 0.9 < s55 < 1.1
    # widths in downsampled samples keep the physical widths that are resolved
    for a, b, f, w in segs:
        assert w[0] == 1 and w[-1] == 256 // f


def test_downsample_by_hand():
    X = np.array([[0, 1, 2, 3, 255, 255, 254, 255, 7],
                  [1, 1, 1, 2, 10, 11, 12, 13, 99]], dtype=np.uint8)
    assert PL.downsample(X, 2).tolist() == [[1, 3, 255, 255], [1, 2, 11, 13]]     # (0+1+1)//2 = 1, (2+3+1)//2 = 3
    assert PL.downsample(X, 4).tolist() == [[2, 255], [1, 12]]                    # (6+2)//4 = 2, (1019+2)//4 = 255
