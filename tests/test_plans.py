"""De-dispersion plans with downsampling: segmentation (CPU), the downsample
kernel and every segment's series (GPU) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import dedisp as O
from oracle import plans as PL

WL = dict(nchan=64, nsub=8, ndm=60, nsamp=4096, dm_max=220.0, widths=(1, 2, 4, 8, 16, 32), f_lo=1200.0,
          f_hi=1264.0, tsamp=64e-6)


@pytest.fixture(scope="module")
def tx():
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def test_segments_equal_oracle(tx):
    from paper_2401_13834_gb300.plans import DownsampledPlan
    wl = synth.tiny_workload(**WL)
    dp = DownsampledPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, output="series")
    ref = PL.segments(wl.dms, wl.freqs_mhz, wl.tsamp_s, wl.widths, f_max=64)
    got = [(s.dm_lo, s.dm_hi, s.factor, list(s.widths)) for s in dp.segments]
    assert got == [(a, b, f, list(w)) for a, b, f, w in ref]
    assert len(got) >= 4                       # factors 1, 2, 4, 8 at least over DM 0-220
    assert dp.relative_stage1_work() < 0.6


@pytest.mark.parametrize("mk,f_max", [
    (lambda: synth.tiny_workload(**WL), 64),
    (lambda: synth.tiny_workload(**dict(WL, nsamp=6000)), 64),     # 16 is the largest power of two dividing T
    (lambda: synth.tiny_workload(**dict(WL, nsamp=4096)), 4),
    (lambda: synth.meerkat_l_workload(), 64),
])
def test_dsplan_segments_overlaps_and_offsets_equal_oracle(tx, mk, f_max):
    """The library's downsampled plan (tx_dsplan_*) against oracle/plans.py:
    segment DM ranges, factors and widths (f_max lowered to the largest power
    of two dividing T), each segment plan's overlap against the oracle's
    sub-band plan at f t_samp, the native overlap max_j f L_j, and the native
    offsets L - f L_j."""
    wl = mk()
    ds = tx._native.DsPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, f_max=f_max,
                           output="series")
    fdiv = 1
    while wl.nsamp % (2 * fdiv) == 0 and 2 * fdiv <= f_max:
        fdiv *= 2
    ref = PL.segments(wl.dms, wl.freqs_mhz, wl.tsamp_s, wl.widths, f_max=fdiv)
    got = [(s["dm_lo"], s["dm_hi"], s["factor"], list(s["widths"])) for s in ds.segments]
    assert got == [(a, b, f, list(w)) for a, b, f, w in ref]
    Ls = []
    for s, (a, b, f, w) in zip(ds.segments, ref):
        op = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s * f, wl.dms[a:b], wl.nsub, 0, w)
        assert s["overlap"] == op.overlap == s["plan"].overlap
        assert s["nsamp"] == wl.nsamp // f == s["plan"].nsamp
        Ls.append(f * op.overlap)
    assert ds.overlap == max(Ls)
    assert [s["native_offset"] for s in ds.segments] == [ds.overlap - x for x in Ls]


@pytest.mark.gpu
@pytest.mark.parametrize("layout,nchan", [("ft", 64), ("tf", 64), ("tf", 63), ("ft", 63)])
def test_downsample_kernel(tx, layout, nchan):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X = np.random.default_rng(nchan).integers(0, 256, size=(nchan, 1024), dtype=np.uint8)
    for f in (1, 2, 4, 8, 64):
        src = torch.from_numpy(np.ascontiguousarray(X.T if layout == "tf" else X)).cuda()
        got = tx.downsample(src, layout, nchan, 1024, f).cpu().numpy()
        ref = PL.downsample(X, f)
        got = got.reshape(1024 // f, nchan).T if layout == "tf" else got.reshape(nchan, 1024 // f)
        assert np.array_equal(got, ref), f


@pytest.mark.gpu
@pytest.mark.parametrize("layout", ["ft", "tf"])
def test_segment_series_equal_oracle(tx, layout):
    """Each segment's series, two blocks in a row, equal the oracle run on the
    oracle-downsampled window of that segment."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300.plans import DownsampledPlan
    wl = synth.tiny_workload(**WL)
    dp = DownsampledPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, output="series",
                         layout=layout)
    L, T = dp.overlap, dp.nsamp
    X = synth.make_spectrum(wl, L + 2 * T, synth.small_pulses(wl) if False else [], seed=8)

    def lay(a):
        return torch.from_numpy(np.ascontiguousarray(a.T if layout == "tf" else a)).cuda()

    beams = dp.beams()
    dp.prime(beams, lay(X[:, :L]))
    batch = dp.batch(beams)
    ws = batch.alloc_workspace()
    outs = batch.alloc_outs()
    staging = dp.alloc_staging()
    for b in range(2):
        dp.execute(batch, lay(X[:, L + b * T:L + (b + 1) * T]), outs, ws, staging)
        torch.cuda.synchronize()
        for j, s in enumerate(dp.segments):
            p = s.plan
            got = tx.series_view(p, outs[j][0]).cpu().numpy()
            f, Lj = s.factor, p.overlap
            win = X[:, b * T + L - f * Lj:b * T + L + T]
            Xj = PL.downsample(win, f)
            op = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s * f, wl.dms[s.dm_lo:s.dm_hi], wl.nsub, 0, s.widths)
            assert op.overlap == Lj
            ref = O.subband_dedisperse(Xj, op, p.series_len)
            assert np.array_equal(got, ref), (b, j, f)
