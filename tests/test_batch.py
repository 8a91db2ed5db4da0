"""Batched execute (tx_execute_batch) against the single-beam execute.

Every beam of a batch of uneven shapes must get exactly the results that
tx_execute gives for the same blocks, step after step: the same kernels do
the same integer and float arithmetic, so series, planes and cubes compare bit
for bit and candidate lists compare as sorted sets. Covered: channel counts,
sub-bands, DM grids, group sizes, block lengths, width ladders (exact-count
and generic boxcar), layouts, statistics and output modes mixed in one batch;
CUDA-graph replay and direct launches; one wave and several waves under a
workspace budget; enough steps for every beam's ring to wrap.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS = 3


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


FIB = (1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377)  # 13 widths: the generic boxcar

BEAMS = [
    dict(wl=dict(nchan=32, nsub=4, ndm=12, nsamp=300), output="series", layout="ft"),
    dict(wl=dict(nchan=64, nsub=8, ndm=37, nsamp=1500, group=5), output="cands", layout="tf", snr_threshold=3.0),
    dict(wl=dict(nchan=48, nsub=48, ndm=9, nsamp=777, group=4), output="plane", layout="ft", stats="running"),
    dict(wl=dict(nchan=257, nsub=1, ndm=20, nsamp=4099, group=32), output="cube", layout="ft"),
    dict(wl=dict(nchan=128, nsub=16, ndm=64, nsamp=5000, dm_max=400.0, tsamp=128e-6, widths=FIB),
         output="cands", layout="tf", stats="running", snr_threshold=3.5, tile_box=4096),
    dict(wl=dict(nchan=96, nsub=8, ndm=24, nsamp=2048, descending=True), output="plane", layout="tf"),
    dict(wl=None, output="cands", layout="ft", snr_threshold=6.0, tile_box=8192),   # the 256-channel small workload
    dict(wl=dict(nchan=257, nsub=1, ndm=20, nsamp=2000, group=32), output="series", layout="tf", interm="f16"),
    dict(wl=dict(nchan=128, nsub=4, ndm=40, nsamp=2500, dm_max=200.0), output="plane", layout="ft", interm="f16"),
]


def make_plan(tx, spec):
    wl = synth.small_workload() if spec["wl"] is None else synth.tiny_workload(**spec["wl"])
    kw = {k: v for k, v in spec.items() if k != "wl"}
    return tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, **kw)


def to_layout(X, layout):
    return np.ascontiguousarray(X.T if layout == "tf" else X)


def decode(tx, plan, out, nc):
    torch.cuda.synchronize()
    if plan.output == "cands":
        rec, n = tx.cands_view(plan, out, nc)
        return n, np.sort(rec, order=("dm_index", "t"))
    return out.cpu().numpy().copy()


def same(a, b):
    if isinstance(a, tuple):
        return a[0] == b[0] and np.array_equal(a[1], b[1])
    return np.array_equal(a, b)


def run_pair(tx, specs, graph, budget, profile=False, compact=()):
    """Beams in the batch (compact ones at the indices in `compact`) against
    full beams run alone, block by block."""
    plans = [make_plan(tx, s) for s in specs]
    rng = np.random.default_rng(11)
    streams = [rng.integers(0, 256, size=(p.nchan, p.overlap + NSTEPS * p.nsamp), dtype=np.uint8) for p in plans]
    solo = [tx.Beam(p) for p in plans]
    mixed = [tx.Beam(p, compact=i in compact) for i, p in enumerate(plans)]
    for p, X, b1, b2 in zip(plans, streams, solo, mixed):
        tail = torch.from_numpy(to_layout(X[:, :p.overlap], p.layout)).cuda()
        b1.prime(tail)
        b2.prime(tail)
    batch = tx.Batch(plans, mixed, workspace_budget=budget, graph=graph, profile=profile)
    ws = batch.alloc_workspace()
    outs = batch.alloc_outs()
    solo_ws = [p.alloc_workspace() for p in plans]
    for step in range(NSTEPS):
        blocks = [torch.from_numpy(to_layout(X[:, p.overlap + step * p.nsamp:p.overlap + (step + 1) * p.nsamp],
                                             p.layout)).cuda() for p, X in zip(plans, streams)]
        for o, nc in outs:  # stale values must not survive into the step's results
            o.fill_(0x5A) if o.dtype == torch.uint8 else o.fill_(-7)
            if nc is not None:
                nc.fill_(-1)
        batch.execute(blocks, outs, ws)
        got = [decode(tx, p, o, nc) for p, (o, nc) in zip(plans, outs)]
        for i, (p, b1) in enumerate(zip(plans, solo)):
            o, nc = p.alloc_out()
            tx.execute(p, b1, blocks[i], out=o, ncand=nc, workspace=solo_ws[i])
            ref = decode(tx, p, o, nc)
            assert same(got[i], ref), f"beam {i} ({p.output}, {p.nchan} ch) differs at step {step}"
    assert all(b.nblocks == NSTEPS for b in mixed)
    return batch, plans


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_beam(tx, graph):
    batch, plans = run_pair(tx, BEAMS, graph, budget=0)
    assert batch.nwaves == 1 and batch.nbeams == len(BEAMS)
    assert batch.dm_trial_samples == sum(p.ndm * p.nsamp for p in plans)


def test_batch_in_waves_under_budget(tx):
    plans = [make_plan(tx, s) for s in BEAMS]
    budget = max(p.workspace_bytes for p in plans)
    batch, _ = run_pair(tx, BEAMS, graph=True, budget=budget)
    assert batch.nwaves > 1
    assert batch.workspace_bytes <= budget


@pytest.mark.parametrize("graph", [True, False])
def test_batch_with_compact_beams(tx, graph):
    """Compact beams (tail resident, buffer borrowed from the batch workspace)
    mixed with full ones give the full beams' results."""
    run_pair(tx, BEAMS, graph, budget=0, compact=(1, 2, 4, 6))


def test_batch_profile_times_every_phase(tx):
    batch, _ = run_pair(tx, BEAMS, graph=False, budget=0, profile=True)
    ms, n = batch.read_profile()
    assert n == NSTEPS
    assert all(v > 0.0 for v in ms.values()), ms


def test_batch_rejects_what_it_cannot_run(tx):
    p16 = make_plan(tx, BEAMS[0])
    spec = dict(BEAMS[0], interm="i32")
    p32 = make_plan(tx, spec)
    b16, b32 = tx.Beam(p16), tx.Beam(p32)
    with pytest.raises(tx.TxError) as e:
        tx.Batch([p16, p32], [b16, b32])
    assert e.value.code == -8                        # int32 intermediates: unsupported
    with pytest.raises(tx.TxError) as e:
        tx.Batch([p16, p16], [b16, b16])
    assert e.value.code == -1                        # the same beam twice
    with pytest.raises(tx.TxError) as e:
        tx.Batch([p16], [b16], workspace_budget=max(1, p16.workspace_bytes // 2))
    assert e.value.code == -7                        # one beam over the budget
    with pytest.raises(tx.TxError) as e:
        tx.Batch([p16], [b16], graph=True, profile=True)
    assert e.value.code == -1                        # profiling needs direct launches


def test_batch_wait_times_out_then_completes(tx):
    """A bounded wait on a step that cannot have finished returns a timeout
    (the step is held back by a fixed-length spin enqueued before it: nothing
    hangs), and an unbounded wait then sees it complete with correct results."""
    plans = [make_plan(tx, BEAMS[0])]
    p = plans[0]
    X = np.random.default_rng(2).integers(0, 256, size=(p.nchan, p.overlap + p.nsamp), dtype=np.uint8)
    beams = [tx.Beam(p)]
    beams[0].prime(torch.from_numpy(np.ascontiguousarray(X[:, :p.overlap])).cuda())
    batch = tx.Batch(plans, beams, graph=False)
    ws, outs = batch.alloc_workspace(), batch.alloc_outs()
    blk = torch.from_numpy(np.ascontiguousarray(X[:, p.overlap:])).cuda()
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2e9))              # ~1 s of spinning on this stream, then the step
    batch.execute([blk], outs, ws)
    assert batch.wait(timeout_s=0.05) is False
    assert batch.wait() is True
    ref_beam = tx.Beam(p)
    ref_beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :p.overlap])).cuda())
    ref = tx.execute(p, ref_beam, blk)
    torch.cuda.synchronize()
    assert np.array_equal(outs[0][0].cpu().numpy(), ref.cpu().numpy())
