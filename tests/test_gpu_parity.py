"""GPU kernels vs the CPU oracle, through the C ABI.

Integer work (stage-1 sums, de-dispersed series, candidate indices) must match
bit for bit. Float S/N must agree within |dS/N| <= 1e-5 * max(1, |S/N|). Where
float decides an integer (best width, threshold), points whose decision is
within that tolerance of a tie are checked for validity instead of equality.
"""
import math
import zlib

import numpy as np
import pytest

import synth
from oracle import dedisp as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def make_plan(tx, wl, **kw):
    return tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, **kw)


def oracle_plan(wl, group=None):
    return O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group if group is None else group, wl.widths)


def rand_stream(nchan, nsamp, seed, lo=0, hi=256):
    return np.random.default_rng(seed).integers(lo, hi, size=(nchan, nsamp), dtype=np.uint8)


def to_layout(X, layout):
    return np.ascontiguousarray(X.T if layout == "tf" else X)


def run_blocks(tx, plan, X, nblocks=1, layout="ft", interm_ws=None):
    """Prime with X[:, :L], then execute blocks of T samples; returns host outputs per block."""
    L, T = plan.overlap, plan.nsamp
    beam = tx.Beam(plan)
    if L:
        beam.prime(torch.from_numpy(to_layout(X[:, :L], layout)).cuda())
    ws = plan.alloc_workspace()
    outs = []
    for b in range(nblocks):
        blk = torch.from_numpy(to_layout(X[:, L + b * T:L + (b + 1) * T], layout)).cuda()
        out, nc = plan.alloc_out()
        res = tx.execute(plan, beam, blk, out=out, ncand=nc, workspace=ws)
        torch.cuda.synchronize()
        outs.append((out, nc, ws.clone() if interm_ws else None))
    return outs, beam


def check_snr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= RTOL, (err.max(), np.unravel_index(np.argmax(err), err.shape))


TINY = [
    dict(nchan=32, nsub=4, ndm=12, nsamp=300),
    dict(nchan=32, nsub=4, ndm=12, nsamp=300, descending=True),
    dict(nchan=64, nsub=8, ndm=37, nsamp=1500, group=5),        # ragged last group, ragged tiles
    dict(nchan=48, nsub=48, ndm=9, nsamp=777, group=4),         # one channel per sub-band
    dict(nchan=40, nsub=1, ndm=7, nsamp=2100, group=1),         # one sub-band, unit groups
    dict(nchan=16, nsub=2, ndm=1, nsamp=1, widths=(1,)),        # T = 1, one DM
    dict(nchan=257, nsub=1, ndm=20, nsamp=4099, group=32),      # max channels per sub-band, max group
    dict(nchan=128, nsub=16, ndm=64, nsamp=5000, dm_max=400.0, tsamp=128e-6),
]


@pytest.mark.parametrize("interm", ["u16", "i32"])
@pytest.mark.parametrize("cfg", TINY)
def test_series_bit_exact(tx, cfg, interm):
    wl = synth.tiny_workload(**cfg)
    plan = make_plan(tx, wl, output="series", interm=interm)
    op = oracle_plan(wl)
    assert plan.overlap == op.overlap
    X = rand_stream(wl.nchan, plan.overlap + wl.nsamp, seed=zlib.crc32(str(cfg).encode()) % 1000)
    (out, _, _), = run_blocks(tx, plan, X)[0]
    got = tx.series_view(plan, out).cpu().numpy()
    ref = O.subband_dedisperse(X, op, plan.series_len)
    assert np.array_equal(got, ref)


def test_stage1_intermediate_bit_exact(tx):
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=40, nsamp=3000, dm_max=120.0)
    plan = make_plan(tx, wl, output="series")
    op = oracle_plan(wl)
    X = rand_stream(wl.nchan, plan.overlap + wl.nsamp, seed=5)
    (out, _, ws), = run_blocks(tx, plan, X, interm_ws=True)[0]
    off, pitch, base = plan.stage1_layout()
    P = ws[off:off + plan.ncoarse * plan.nsub * pitch * 2].view(torch.int16).cpu().numpy().view(np.uint16)
    P = P.reshape(plan.ncoarse, plan.nsub, pitch)
    for k in range(plan.ncoarse):
        ds = list(op.fine_dms_of(k))
        for s in range(plan.nsub):
            need = plan.series_len + int(op.d2[ds, s].max()) - int(base[k, s])
            full = O.stage1(X, op, k, s, int(base[k, s]) + need)
            assert np.array_equal(P[k, s, :need].astype(np.int64), full[base[k, s]:])


def test_tf_layout_matches_ft(tx):
    wl = synth.tiny_workload(nchan=96, nsub=8, ndm=24, nsamp=2000)
    X = rand_stream(wl.nchan, 0 + 10 ** 5, seed=6)
    res = []
    for layout in ("ft", "tf"):
        plan = make_plan(tx, wl, output="series", layout=layout)
        Xs = X[:, :plan.overlap + wl.nsamp]
        (out, _, _), = run_blocks(tx, plan, Xs, layout=layout)[0]
        res.append(tx.series_view(plan, out).cpu().numpy())
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("output", ["series", "cands"])
def test_beams_on_two_streams(tx, output):
    """Two beams of one plan, each with its own workspace and outputs, whose
    blocks are launched alternately on two CUDA streams: every block's result
    equals the oracle's (series bit for bit; candidates as in the other
    tests), so nothing an execute keeps in its workspace (the stage-1 item
    counter, the sums) or in the plan's tables is shared between concurrent
    executes."""
    wl = synth.tiny_workload(nchan=128, nsub=16, ndm=48, nsamp=4096, dm_max=300.0, tsamp=128e-6)
    gamma = 4.0
    kw = dict(snr_threshold=gamma, max_cands=1 << 18) if output == "cands" else {}
    plan = make_plan(tx, wl, output=output, **kw)
    op = oracle_plan(wl)
    L, T, nb = plan.overlap, plan.nsamp, 3
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    Xs = [rand_stream(wl.nchan, L + nb * T, seed=40 + i) for i in range(2)]
    beams, outs = [], [[], []]
    for i in range(2):
        b = tx.Beam(plan)
        b.prime(torch.from_numpy(np.ascontiguousarray(Xs[i][:, :L])).cuda())
        beams.append(b)
    torch.cuda.synchronize()
    ws = [plan.alloc_workspace() for _ in range(2)]
    blocks = [[torch.from_numpy(np.ascontiguousarray(Xs[i][:, L + b * T:L + (b + 1) * T])).cuda() for b in range(nb)]
              for i in range(2)]
    for b in range(nb):
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                o, nc = plan.alloc_out()
                tx.execute(plan, beams[i], blocks[i][b], out=o, ncand=nc, workspace=ws[i], stream=streams[i])
                outs[i].append((o, nc))
    torch.cuda.synchronize()
    for i in range(2):
        ref = O.stream_series(Xs[i], op, T, nb)
        for b in range(nb):
            o, nc = outs[i][b]
            if output == "series":
                assert np.array_equal(tx.series_view(plan, o).cpu().numpy(), ref[b]), (i, b)
            else:
                D = ref[b]
                _, _, mu, sg = O.block_stats(D, T)
                snr = O.boxcar_snr(D, op.widths, T, mu, sg)
                got, n = tx.cands_view(plan, o, nc)
                _check_cands(got, n, snr, gamma)


@pytest.mark.parametrize("layout", ["ft", "tf"])
def test_streaming_blocks_and_checkpoint(tx, layout):
    """Four blocks of one stream and a checkpoint/resume, bit-exact against the oracle.
    T = 1000 is not a multiple of 16, so the window start's residue mod 16
    alternates between blocks: blocks 0 and 2 use the plan's precomputed
    stage-1 offset tables, blocks 1 and 3 the tables built in the kernel."""
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=16, nsamp=1000, dm_max=80.0)
    plan = make_plan(tx, wl, output="series", layout=layout)
    op = oracle_plan(wl)
    nb = 4
    X = rand_stream(wl.nchan, plan.overlap + nb * wl.nsamp, seed=7)
    outs, beam = run_blocks(tx, plan, X, nblocks=nb, layout=layout)
    ref = O.stream_series(X, op, wl.nsamp, nb)
    for b in range(nb):
        assert np.array_equal(tx.series_view(plan, outs[b][0]).cpu().numpy(), ref[b])
    assert beam.nblocks == nb
    # checkpoint after two blocks, resume in a fresh beam
    outs2, beam2 = run_blocks(tx, plan, X[:, :plan.overlap + 2 * wl.nsamp], nblocks=2, layout=layout)
    state = beam2.export()
    beam3 = tx.Beam(plan)
    beam3.import_(state)
    assert beam3.nblocks == 2
    ws = plan.alloc_workspace()
    for b in (2, 3):
        blk = torch.from_numpy(to_layout(X[:, plan.overlap + b * wl.nsamp:plan.overlap + (b + 1) * wl.nsamp], layout)).cuda()
        out = tx.execute(plan, beam3, blk, workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(tx.series_view(plan, out).cpu().numpy(), ref[b])


def _oracle_snr(X, op, T, dm_indices=None):
    D = O.subband_dedisperse(X, op, T + op.wmax - 1, dm_indices)
    _, _, mu, sg = O.block_stats(D, T)
    return O.boxcar_snr(D, op.widths, T, mu, sg), D


@pytest.fixture(scope="module")
def small_case():
    wl = synth.small_workload()
    op = oracle_plan(wl)
    X = synth.make_spectrum(wl, op.overlap + wl.nsamp, synth.small_pulses(wl), seed=0)
    snr, D = _oracle_snr(X, op, wl.nsamp)
    return wl, op, X, snr, D


def test_small_cube(tx, small_case):
    wl, op, X, snr, D = small_case
    plan = make_plan(tx, wl, output="cube")
    (out, _, _), = run_blocks(tx, plan, X)[0]
    got = tx.cube_view(plan, out).cpu().numpy()
    check_snr(got, snr)
    # the injected pulse is found near DM 100 with S/N close to 20
    d, w, t = np.unravel_index(np.argmax(got), got.shape)
    assert abs(wl.dms[d] - 100.0) < 4.0 and got[d, w, t] > 15.0


def _check_plane(best_g, w_g, snr_ref):
    best_ref, w_ref = O.dm_time_plane(snr_ref)
    check_snr(best_g, best_ref)
    srt = np.sort(snr_ref, axis=1)
    gap = (srt[:, -1, :] - srt[:, -2, :]) if snr_ref.shape[1] > 1 else np.full(best_ref.shape, np.inf)
    tol = 2 * RTOL * np.maximum(1.0, np.abs(best_ref))
    clear = gap > tol
    assert np.array_equal(w_g[clear], w_ref[clear])
    # near-ties: the chosen width's S/N is (within tolerance) the best
    chosen = np.take_along_axis(snr_ref, w_g[:, None, :].astype(np.int64), axis=1)[:, 0, :]
    assert np.all(np.abs(chosen - best_ref)[~clear] <= tol[~clear])


def test_small_plane(tx, small_case):
    wl, op, X, snr, D = small_case
    plan = make_plan(tx, wl, output="plane")
    (out, _, _), = run_blocks(tx, plan, X)[0]
    s, w = tx.plane_view(plan, out)
    _check_plane(s.cpu().numpy(), w.cpu().numpy(), snr)


def _check_cands(got, n, snr_ref, gamma, dm_indices=None):
    best_ref, w_ref = O.dm_time_plane(snr_ref)
    ref = O.candidates(best_ref, w_ref, gamma, dm_indices)
    tol = RTOL * max(1.0, abs(gamma))
    assert n == got.size
    g = {(int(r["dm_index"]), int(r["t"])): r for r in got}
    r_ = {(int(r["d"]), int(r["t"])): r for r in ref}
    assert len(g) == got.size  # no duplicates
    for key in set(g) ^ set(r_):  # disagreements only at the threshold
        row = dm_indices.index(key[0]) if dm_indices is not None else key[0]
        assert abs(best_ref[row, key[1]] - gamma) <= tol, key
    for key in set(g) & set(r_):
        a, b = g[key], r_[key]
        assert abs(float(a["snr"]) - b["snr"]) <= RTOL * max(1.0, abs(b["snr"]))


def test_small_candidates(tx, small_case):
    wl, op, X, snr, D = small_case
    gamma = 6.0
    plan = make_plan(tx, wl, output="cands", snr_threshold=gamma, max_cands=1 << 16)
    (out, nc, _), = run_blocks(tx, plan, X)[0]
    got, n = tx.cands_view(plan, out, nc)
    assert 0 < n < (1 << 16)
    _check_cands(got, n, snr, gamma)


def test_candidate_overflow_keeps_valid_records(tx, small_case):
    wl, op, X, snr, D = small_case
    plan = make_plan(tx, wl, output="cands", snr_threshold=2.0, max_cands=100)
    (out, nc, _), = run_blocks(tx, plan, X)[0]
    n = int(nc.item())
    assert n > 100
    got = out[:100].cpu().numpy().view(tx.CAND_DTYPE).reshape(-1)
    best_ref, _ = O.dm_time_plane(snr)
    for r in got:
        assert abs(float(r["snr"]) - best_ref[r["dm_index"], r["t"]]) <= RTOL * max(1, abs(float(r["snr"])))
        assert float(r["snr"]) >= 2.0 - RTOL * 2.0  # the threshold decision is exact; the float S/N rounds


def test_running_statistics(tx):
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=10, nsamp=2000, dm_max=50.0)
    plan = make_plan(tx, wl, output="cube", stats="running", stats_lambda=0.25)
    op = oracle_plan(wl)
    nb = 3
    X = rand_stream(wl.nchan, plan.overlap + nb * wl.nsamp, seed=9)
    outs, _ = run_blocks(tx, plan, X, nblocks=nb)
    series = O.stream_series(X, op, wl.nsamp, nb)
    st = None
    for b in range(nb):
        _, _, mu, sg = O.block_stats(series[b], wl.nsamp)
        new = []
        for i in range(len(mu)):
            prev = None if st is None else st[i]
            new.append(O.running_stats(prev, mu[i], sg[i] ** 2, 0.25))
        st = new
        ref = O.boxcar_snr(series[b], op.widths, wl.nsamp, [s[0] for s in st], [math.sqrt(s[1]) for s in st])
        check_snr(tx.cube_view(plan, outs[b][0]).cpu().numpy(), ref)


def test_constant_input_gives_zero_snr(tx):
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=6, nsamp=900)
    plan = make_plan(tx, wl, output="cube")
    X = np.full((wl.nchan, plan.overlap + wl.nsamp), 77, dtype=np.uint8)
    (out, _, _), = run_blocks(tx, plan, X)[0]
    assert torch.count_nonzero(tx.cube_view(plan, out)).item() == 0


def test_execute_host_matches_device(tx, small_case):
    wl, op, X, snr, D = small_case
    gamma = 7.0
    plan = make_plan(tx, wl, output="cands", snr_threshold=gamma, max_cands=4096)
    (out, nc, _), = run_blocks(tx, plan, X)[0]
    dev, n = tx.cands_view(plan, out, nc)
    beam = tx.Beam(plan)
    beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :plan.overlap])).cuda())
    staging = torch.empty(plan.block_bytes, dtype=torch.uint8, device="cuda")
    dout, dnc = plan.alloc_out()
    ws = plan.alloc_workspace()
    h_out = np.zeros(4096, dtype=tx.CAND_DTYPE)
    nh = tx.execute_host(plan, beam, np.ascontiguousarray(X[:, plan.overlap:]), h_out, staging, dout, dnc, ws)
    assert nh == n
    key = lambda a: sorted((int(r["dm_index"]), int(r["t"]), int(r["w_index"]), float(r["snr"])) for r in a)
    assert key(h_out[:nh]) == key(dev)


@pytest.fixture(scope="module")
def meerkat_case():
    wl = synth.meerkat_l_workload()
    op = oracle_plan(wl)
    pulses = synth.meerkat_pulses(wl)
    X = synth.make_spectrum(wl, op.overlap + wl.nsamp, pulses, seed=1)
    return wl, op, X, pulses


def test_meerkat_full_size_sampled(tx, meerkat_case):
    """Full 4096-channel x 4096-DM block in the benchmark's launch configuration,
    checked on sampled DM trials (first/last groups, segment edges, pulses)."""
    wl, op, X, pulses = meerkat_case
    gamma = 7.0
    sample = sorted({0, 1, 15, 16, 1023, 1024, 2047, 2048, 3071, 3072, 4094, 4095}
                    | {int(np.argmin(np.abs(wl.dms - p.dm))) for p in pulses[:4]})
    plan_s = make_plan(tx, wl, output="series")
    (out, _, _), = run_blocks(tx, plan_s, X)[0]
    series = tx.series_view(plan_s, out)[sample].cpu().numpy()
    D = O.subband_dedisperse(X, op, plan_s.series_len, sample)
    assert np.array_equal(series, D)
    del out
    torch.cuda.empty_cache()
    _, _, mu, sg = O.block_stats(D, wl.nsamp)
    snr = O.boxcar_snr(D, op.widths, wl.nsamp, mu, sg)
    plan_p = make_plan(tx, wl, output="plane")
    (out, _, _), = run_blocks(tx, plan_p, X)[0]
    s, w = tx.plane_view(plan_p, out)
    _check_plane(s[sample].cpu().numpy(), w[sample].cpu().numpy(), snr)
    del out
    torch.cuda.empty_cache()
    plan_c = make_plan(tx, wl, output="cands", snr_threshold=gamma, max_cands=1 << 24)
    (out, nc, _), = run_blocks(tx, plan_c, X)[0]
    got, n = tx.cands_view(plan_c, out, nc)
    assert n < (1 << 24)
    sub = got[np.isin(got["dm_index"], sample)]
    _check_cands(sub, sub.size, snr, gamma, dm_indices=sample)


@pytest.mark.parametrize("widths", [(1,), (3, 7), tuple(range(1, 17)), tuple(range(1, 21)), (1, 2, 4, 8, 16, 32, 64, 100, 200, 400, 800, 1000),
                                    (1, 2), (1, 2, 8, 20, 64, 252), (2, 4, 8)])
@pytest.mark.parametrize("output", ["cube", "plane", "cands"])
def test_boxcar_width_sets(tx, widths, output):
    """Every width-count code path (exact counts and the generic one; for candidates
    also the four-output test of widths 1, 2 and multiples of 4) against the oracle,
    on one full 2048-output tile and a ragged one."""
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=6, nsamp=3000, widths=widths)
    gamma = 3.0
    kw = dict(snr_threshold=gamma, max_cands=1 << 16) if output == "cands" else {}
    plan = make_plan(tx, wl, output=output, **kw)
    op = oracle_plan(wl)
    X = synth.make_spectrum(wl, plan.overlap + wl.nsamp,
                            [synth.Pulse(dm=30.0, t_arr=1200.0, fwhm=12.0, amp=9.0)], seed=11)
    (out, nc, _), = run_blocks(tx, plan, X)[0]
    snr, _ = _oracle_snr(X, op, wl.nsamp)
    if output == "cube":
        check_snr(tx.cube_view(plan, out).cpu().numpy(), snr)
    elif output == "plane":
        s, w = tx.plane_view(plan, out)
        _check_plane(s.cpu().numpy(), w.cpu().numpy(), snr)
    else:
        got, n = tx.cands_view(plan, out, nc)
        assert 0 < n < (1 << 16)
        assert (got["t"] < 2048).any() and (got["t"] >= 2048).any()   # hits in the full tile and the ragged one
        _check_cands(got, n, snr, gamma)


@pytest.mark.parametrize("tile_box", [4096, 8192])
@pytest.mark.parametrize("widths", [(1, 2, 4, 8, 16, 32, 64), (1, 2, 3, 5, 8, 13, 21, 34, 55, 89)])
@pytest.mark.parametrize("output", ["cube", "plane", "cands"])
def test_boxcar_long_units(tx, tile_box, widths, output):
    """Boxcar units of 2 or 4 sub-tiles of 2048 outputs: T = 11192 gives full
    units and a last one of 3000 outputs (one full sub-tile and a ragged one);
    widths 1, 2 and multiples of 4 take the four-output test, the Fibonacci set
    the one-output test of full sub-tiles."""
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=5, nsamp=11192, widths=widths)
    gamma = 3.0
    kw = dict(snr_threshold=gamma, max_cands=1 << 17) if output == "cands" else {}
    plan = make_plan(tx, wl, output=output, tile_box=tile_box, **kw)
    assert plan.tile_box == tile_box
    op = oracle_plan(wl)
    pulses = [synth.Pulse(dm=30.0, t_arr=float(t), fwhm=12.0, amp=9.0) for t in (1500, 5000, 9000, 10800)]
    X = synth.make_spectrum(wl, plan.overlap + wl.nsamp, pulses, seed=12)
    (out, nc, _), = run_blocks(tx, plan, X)[0]
    snr, _ = _oracle_snr(X, op, wl.nsamp)
    if output == "cube":
        check_snr(tx.cube_view(plan, out).cpu().numpy(), snr)
    elif output == "plane":
        s, w = tx.plane_view(plan, out)
        _check_plane(s.cpu().numpy(), w.cpu().numpy(), snr)
    else:
        got, n = tx.cands_view(plan, out, nc)
        assert 0 < n < (1 << 17)
        t = got["t"][:n]
        assert (t < 2048).any() and ((t >= 2048) & (t < tile_box)).any() and (t >= 10240).any()
        _check_cands(got, n, snr, gamma)


@pytest.mark.parametrize("q1", [32, 64, 128, 256])
@pytest.mark.parametrize("group,split,want", [
    (4, 0, 4), (8, 0, 2), (16, 0, 1),          # the pipelined stage 2: 4, 2, 1 consumer warps per DM
    (17, 1, 1), (32, 1, 1),                    # larger groups: the other kernel, split as asked
])
def test_tile_shapes_do_not_change_results(tx, q1, group, split, want):
    """Every stage-1 tile length, both stage-2 kernels and each of their warp
    splits give the oracle's series."""
    wl = synth.tiny_workload(nchan=128, nsub=16, ndm=64, nsamp=5000, dm_max=400.0, tsamp=128e-6, group=group)
    plan = make_plan(tx, wl, output="series", tile_q1=q1, tile_split2=split)
    assert (plan.tile_q1, plan.tile_split2) == (q1, want)
    op = oracle_plan(wl)
    X = rand_stream(wl.nchan, plan.overlap + wl.nsamp, seed=77)
    (out, _, _), = run_blocks(tx, plan, X)[0]
    got = tx.series_view(plan, out).cpu().numpy()
    assert np.array_equal(got, O.subband_dedisperse(X, op, plan.series_len))


@pytest.mark.parametrize("layout", ["ft", "tf"])
@pytest.mark.parametrize("cfg", [TINY[2], TINY[3], TINY[7], dict(nchan=64, nsub=8, ndm=20, nsamp=4096, dm_max=90.0)])
def test_compact_beam_equals_full_beam(tx, cfg, layout):
    """A compact beam (tail resident, buffer borrowed from the workspace) gives
    exactly the full beam's outputs, block after block; odd L and T exercise
    the tail store's padding and its byte-wise copy."""
    wl = synth.tiny_workload(**cfg)
    for output in ("series", "cands"):
        plan = make_plan(tx, wl, output=output, layout=layout, snr_threshold=3.0)
        L, T = plan.overlap, plan.nsamp
        X = rand_stream(wl.nchan, L + 3 * T, seed=91)
        full, comp = tx.Beam(plan), tx.Beam(plan, compact=True)
        tail = torch.from_numpy(to_layout(X[:, :L], layout)).cuda()
        full.prime(tail)
        comp.prime(tail)
        wsf, wsc = plan.alloc_workspace(), plan.alloc_workspace(compact=True)
        for b in range(3):
            blk = torch.from_numpy(to_layout(X[:, L + b * T:L + (b + 1) * T], layout)).cuda()
            res = []
            for beam, ws in ((full, wsf), (comp, wsc)):
                out, nc = plan.alloc_out()
                tx.execute(plan, beam, blk, out=out, ncand=nc, workspace=ws)
                torch.cuda.synchronize()
                if output == "cands":
                    rec, n = tx.cands_view(plan, out, nc)
                    res.append((n, np.sort(rec, order=("dm_index", "t"))))
                else:
                    res.append(out.cpu().numpy())
            if output == "cands":
                assert res[0][0] == res[1][0] and np.array_equal(res[0][1], res[1][1]), f"block {b}"
            else:
                assert np.array_equal(res[0], res[1]), f"block {b}"
        # the checkpoint of a compact beam is the full beam's
        assert full.export() == comp.export()


def test_compact_beam_checkpoint_restore(tx):
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=20, nsamp=1000, dm_max=90.0)
    plan = make_plan(tx, wl, output="series")
    L, T = plan.overlap, plan.nsamp
    X = rand_stream(wl.nchan, L + 3 * T, seed=92)
    a = tx.Beam(plan, compact=True)
    a.prime(torch.from_numpy(np.ascontiguousarray(X[:, :L])).cuda())
    ws = plan.alloc_workspace(compact=True)
    blk = [torch.from_numpy(np.ascontiguousarray(X[:, L + i * T:L + (i + 1) * T])).cuda() for i in range(3)]
    tx.execute(plan, a, blk[0], workspace=ws)
    state = a.export()
    ref = [tx.execute(plan, a, blk[i], workspace=ws).cpu().numpy() for i in (1, 2)]
    b = tx.Beam(plan, compact=True)
    b.import_(state)
    got = [tx.execute(plan, b, blk[i], workspace=ws).cpu().numpy() for i in (1, 2)]
    assert all(np.array_equal(x, y) for x, y in zip(ref, got))
    assert b.nblocks == 3


@pytest.mark.parametrize("cfg", TINY)
def test_f16_series_bit_exact(tx, cfg):
    """FP16 stage-1 storage: the series equal the oracle's emulation of the
    FP16 form exactly (uniform data drives the sums far past 2048, so
    rounding and, at 257 channels per sub-band, saturation both occur)."""
    wl = synth.tiny_workload(**cfg)
    plan = make_plan(tx, wl, output="series", interm="f16")
    op = oracle_plan(wl)
    X = rand_stream(wl.nchan, plan.overlap + wl.nsamp, seed=zlib.crc32(str(cfg).encode()) % 997)
    (out, _, _), = run_blocks(tx, plan, X)[0]
    got = tx.series_view(plan, out).cpu().numpy()
    ref = O.subband_dedisperse_f16(X, op, plan.series_len, slice(plan.overlap, plan.overlap + wl.nsamp))
    assert np.array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("compact", [False, True])
def test_f16_with_rfi_over_blocks(tx, compact):
    """64 channels per sub-band with narrow-band RFI and zero-DM bursts (sums
    beyond 2048 where the bursts are), three blocks through one beam."""
    wl = synth.tiny_workload(nchan=256, nsub=4, ndm=48, nsamp=3000, dm_max=150.0, tsamp=128e-6)
    plan = make_plan(tx, wl, output="series", interm="f16")
    op = oracle_plan(wl)
    L, T = plan.overlap, plan.nsamp
    rfi = synth.make_rfi(wl, L + 3 * T, seed=4)
    X = synth.make_spectrum(wl, L + 3 * T, [], seed=5, rfi=rfi)
    beam = tx.Beam(plan, compact=compact)
    beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :L])).cuda())
    ws = plan.alloc_workspace(compact=compact)
    rounded = 0
    for b in range(3):
        blk = torch.from_numpy(np.ascontiguousarray(X[:, L + b * T:L + (b + 1) * T])).cuda()
        got = tx.series_view(plan, tx.execute(plan, beam, blk, workspace=ws)).cpu().numpy()
        win = X[:, b * T:b * T + L + T]
        ref = O.subband_dedisperse_f16(win, op, plan.series_len, slice(L, L + T))
        assert np.array_equal(got.astype(np.float64), ref), f"block {b}"
        rounded += int((ref != O.subband_dedisperse(win, op, plan.series_len)).sum())
    assert rounded > 0          # the bursts did push sums past 2048


def test_misaligned_buffers_are_refused_before_any_launch(tx):
    """A series buffer that is 4- but not 8-byte aligned (the kernel stores
    two outputs at a time) and a workspace that is not 16-byte aligned (bulk
    copies) are refused with TX_ERR_INVALID_ARG, and nothing runs: the beam
    still gives the right series afterwards."""
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=12, nsamp=300)
    plan = make_plan(tx, wl, output="series")
    X = rand_stream(plan.nchan, plan.overlap + plan.nsamp, 3)
    beam = tx.Beam(plan)
    beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :plan.overlap])).cuda())
    blk = torch.from_numpy(np.ascontiguousarray(X[:, plan.overlap:])).cuda()
    big = torch.zeros(plan.ndm * plan.series_len + 2, dtype=torch.int32, device="cuda")
    ws = plan.alloc_workspace()
    wsb = torch.zeros(plan.workspace_bytes + 16, dtype=torch.uint8, device="cuda")
    for out, w in ((big[1:], ws), (big[:-2], wsb[4:])):
        with pytest.raises(tx.TxError) as e:
            tx.execute(plan, beam, blk, out=out, workspace=w)
        assert e.value.code == -1
    assert beam.nblocks == 0
    out = big[:-2]
    tx.execute(plan, beam, blk, out=out, workspace=ws)
    torch.cuda.synchronize()
    D = O.subband_dedisperse(X, oracle_plan(wl), plan.series_len)
    assert np.array_equal(tx.series_view(plan, out).cpu().numpy(), D)
