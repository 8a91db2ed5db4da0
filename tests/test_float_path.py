"""The float path (per-channel normalisation, Sec. 2.1) against the oracle.

Blocks of channels with unequal noise (one of them 20 times noisier, as an
RFI-like outlier) and a dispersed pulse stream through a beam whose plan
normalises each block to unit variance or weights it by the reciprocal of
the variance. The library keeps x' in float32 exactly as the oracle defines
it, sums it in FP32; the oracle sums the same float32 values in float64.
Checked block after block: the series within the first-order rounding bound
of an FP32 sum of (channels per sub-band + sub-bands + 1) terms of the
absolute values along the track (oracle.normalise.sum_error_bound); the S/N
cube, the DM-time plane and the candidates within 1e-5 relative, as the
integer path.
"""
import numpy as np
import pytest

import synth
from oracle import dedisp as O
from oracle import normalise as NM
from test_gpu_parity import RTOL, _check_cands, _check_plane, check_snr, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NBLOCKS = 3


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def _workload(nsamp=1500, **kw):
    base = dict(nchan=64, nsub=8, ndm=37, nsamp=nsamp, group=5, dm_max=120.0, widths=(1, 2, 4, 8, 16))
    base.update(kw)
    return synth.tiny_workload(**base)


def _stream(wl, L, seed):
    """uint8 [nchan, L + NBLOCKS T]: noise of a different sigma per channel (one
    channel 20x noisier), a dispersed pulse in every block."""
    rng = np.random.default_rng(seed)
    n = L + NBLOCKS * wl.nsamp
    sig = rng.uniform(2.0, 16.0, wl.nchan)
    sig[wl.nchan // 3] = 60.0
    x = 128.0 + sig[:, None] * rng.standard_normal((wl.nchan, n))
    for b in range(NBLOCKS):
        p = synth.Pulse(dm=float(wl.dms[len(wl.dms) // 2]), t_arr=float(b * wl.nsamp + wl.nsamp // 2),
                        fwhm=6.0, amp=4.0)
        c, t, v = synth.pulse_points(p, wl.freqs_mhz, wl.tsamp_s, n)
        np.add.at(x, (c, t), v)
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def _run(tx, wl, norm, output, layout="ft", stats="block", **kw):
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, norm=norm,
                   output=output, layout=layout, stats=stats, **kw)
    assert plan.interm == "f32"
    X = _stream(wl, plan.overlap, seed=11)
    L, T = plan.overlap, plan.nsamp
    beam = tx.Beam(plan)
    beam.prime(torch.from_numpy(to_layout(X[:, :L], layout)).cuda())
    ws = plan.alloc_workspace()
    outs = []
    for b in range(NBLOCKS):
        blk = torch.from_numpy(to_layout(X[:, L + b * T:L + (b + 1) * T], layout)).cuda()
        out, nc = plan.alloc_out()
        tx.execute(plan, beam, blk, out=out, ncand=nc, workspace=ws)
        torch.cuda.synchronize()
        outs.append((out, nc))
    return plan, X, outs


def _oracle(wl, X, L, T, norm, b):
    """Block b: the window of normalised data, its series in float64 and the
    rounding bound of the FP32 sums along each track."""
    op = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group, wl.widths)
    Xn = NM.normalised_stream(X, L, T, NBLOCKS, norm)
    win = Xn[:, b * T:b * T + L + T].astype(np.float64)
    D = O.subband_dedisperse(win, op, T + op.wmax - 1)
    bound = NM.sum_error_bound(O.subband_dedisperse(np.abs(win), op, T + op.wmax - 1), op.m + op.nsub + 1)
    return op, D, bound


@pytest.mark.parametrize("norm", ["unit", "invvar"])
@pytest.mark.parametrize("layout", ["ft", "tf"])
def test_float_series_within_rounding_bound(tx, norm, layout):
    wl = _workload()
    plan, X, outs = _run(tx, wl, norm, "series", layout)
    for b, (out, _) in enumerate(outs):
        _, D, bound = _oracle(wl, X, plan.overlap, plan.nsamp, norm, b)
        got = tx.series_view(plan, out).cpu().numpy().astype(np.float64)
        err = np.abs(got - D)
        assert np.all(err <= bound), (b, float(err.max()), float(bound[err > bound].min()) if (err > bound).any() else 0)


@pytest.mark.parametrize("norm", ["unit", "invvar"])
@pytest.mark.parametrize("output", ["cube", "plane", "cands"])
def test_float_snr_matches_oracle(tx, norm, output):
    wl = _workload()
    gamma = 4.0
    kw = dict(snr_threshold=gamma, max_cands=1 << 16) if output == "cands" else {}
    plan, X, outs = _run(tx, wl, norm, output, **kw)
    T = plan.nsamp
    for b, (out, nc) in enumerate(outs):
        op, D, _ = _oracle(wl, X, plan.overlap, T, norm, b)
        _, _, mu, sg = O.block_stats(D, T)
        snr = O.boxcar_snr(D, op.widths, T, mu, sg)
        if output == "cube":
            check_snr(tx.cube_view(plan, out).cpu().numpy(), snr)
        elif output == "plane":
            s, w = tx.plane_view(plan, out)
            _check_plane(s.cpu().numpy(), w.cpu().numpy(), snr)
        else:
            got, n = tx.cands_view(plan, out, nc)
            assert 0 < n < (1 << 16)
            _check_cands(got, n, snr, gamma)


@pytest.mark.parametrize("tile_box", [4096, 8192])
def test_float_boxcar_long_units(tx, tile_box):
    """Boxcar units of 4096 or 8192 outputs on the float path (a full unit and
    a ragged one at T = 9000), S/N against the oracle."""
    wl = _workload(nsamp=9000)
    plan, X, outs = _run(tx, wl, "unit", "cube", tile_box=tile_box)
    T = plan.nsamp
    for b, (out, _) in enumerate(outs):
        op, D, _ = _oracle(wl, X, plan.overlap, T, "unit", b)
        _, _, mu, sg = O.block_stats(D, T)
        check_snr(tx.cube_view(plan, out).cpu().numpy(), O.boxcar_snr(D, op.widths, T, mu, sg))


def test_float_running_statistics(tx):
    wl = _workload()
    plan, X, outs = _run(tx, wl, "unit", "cube", stats="running", stats_lambda=0.25)
    T = plan.nsamp
    prev = None
    for b, (out, _) in enumerate(outs):
        op, D, _ = _oracle(wl, X, plan.overlap, T, "unit", b)
        _, _, mu, sg = O.block_stats(D, T)
        mu, var = np.asarray(mu), np.asarray(sg) ** 2
        prev = O.running_stats(prev, mu, var, 0.25)
        snr = O.boxcar_snr(D, op.widths, T, prev[0], np.sqrt(prev[1]))
        check_snr(tx.cube_view(plan, out).cpu().numpy(), snr)


def test_float_path_damps_the_noisy_channel(tx):
    """The reason the paper gives for the weights: a channel 20x noisier than
    the rest costs the raw (equal-weight) sum most of the pulse's S/N, unit
    variance recovers it, and reciprocal-variance weights recover the most."""
    wl = _workload()
    best = {}
    for norm in ("none", "unit", "invvar"):
        kw = dict(interm="u16") if norm == "none" else dict(norm=norm)
        plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group,
                       output="plane", **kw)
        X = _stream(wl, plan.overlap, seed=11)
        beam = tx.Beam(plan)
        beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :plan.overlap])).cuda())
        out, _ = plan.alloc_out()
        tx.execute(plan, beam, torch.from_numpy(np.ascontiguousarray(X[:, plan.overlap:plan.overlap + wl.nsamp]))
                   .cuda(), out=out)
        torch.cuda.synchronize()
        s, _ = tx.plane_view(plan, out)
        best[norm] = float(s[len(wl.dms) // 2].max())
    assert best["invvar"] > best["unit"] > best["none"], best


def test_float_checkpoint_resume(tx):
    """Export after a block, import into a fresh beam: the next block's series
    equal the uninterrupted run's exactly (the float tail is carried as is)."""
    wl = _workload()
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, norm="unit",
                   output="series")
    X = _stream(wl, plan.overlap, seed=5)
    L, T = plan.overlap, plan.nsamp
    blk = [torch.from_numpy(np.ascontiguousarray(X[:, L + b * T:L + (b + 1) * T])).cuda() for b in range(2)]
    a = tx.Beam(plan)
    a.prime(torch.from_numpy(np.ascontiguousarray(X[:, :L])).cuda())
    tx.execute(plan, a, blk[0])
    state = a.export()
    ref = tx.execute(plan, a, blk[1])
    c = tx.Beam(plan)
    c.import_(state)
    got = tx.execute(plan, c, blk[1])
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_float_path_refusals(tx):
    wl = _workload()
    with pytest.raises(tx.TxError) as e:
        tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, norm="unit", interm="i32")
    assert e.value.code == -1                                   # a normalisation needs float32 intermediates
    p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, norm="unit")
    with pytest.raises(tx.TxError) as e:
        tx.Beam(p, compact=True)
    assert e.value.code == -8
    b = tx.Beam(p)
    with pytest.raises(tx.TxError) as e:
        tx.Batch([p], [b])
    assert e.value.code == -8
