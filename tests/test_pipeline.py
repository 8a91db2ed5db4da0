"""Pipelined host execution (tx_pipeline_*) against block-by-block device execution.

The pipeline only orchestrates copies and the same tx_execute kernels (whose
results are checked against the oracle in test_gpu_parity.py), so a stream of
blocks pushed through it must give bit-identical results to executing the same
blocks one by one on another beam primed with the same tail.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NBLOCKS = 6


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def stream_case(tx, output, **kw):
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=24, nsamp=2500, dm_max=80.0)
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, output=output, **kw)
    L, T = plan.overlap, plan.nsamp
    pulses = [synth.Pulse(dm=20.0 + 9.0 * b, t_arr=L + b * T + 700.0, fwhm=6.0, amp=6.0) for b in range(NBLOCKS)]
    X = synth.make_spectrum(wl, L + NBLOCKS * T, pulses, seed=5)
    tail = torch.from_numpy(np.ascontiguousarray(X[:, :L])).cuda()
    blocks = [np.ascontiguousarray(X[:, L + b * T:L + (b + 1) * T]) for b in range(NBLOCKS)]
    return plan, tail, blocks


def reference(tx, plan, tail, blocks):
    beam = tx.Beam(plan)
    beam.prime(tail)
    ws = plan.alloc_workspace()
    res = []
    for blk in blocks:
        out, nc = plan.alloc_out()
        tx.execute(plan, beam, torch.from_numpy(blk).cuda(), out=out, ncand=nc, workspace=ws)
        torch.cuda.synchronize()
        if plan.output == "cands":
            res.append(tx.cands_view(plan, out, nc))
        else:
            res.append(out.cpu().numpy())
    return res


def key(rec):
    return sorted((int(r["dm_index"]), int(r["t"]), int(r["w_index"]), float(r["snr"])) for r in rec)


def pinned(blocks):
    return [torch.from_numpy(b).pin_memory() for b in blocks]


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_candidates_match_block_by_block(tx, depth):
    plan, tail, blocks = stream_case(tx, "cands", snr_threshold=6.0, max_cands=1 << 14)
    ref = reference(tx, plan, tail, blocks)
    assert all(n > 0 for _, n in ref)
    beam = tx.Beam(plan)
    beam.prime(tail)
    pl = tx.Pipeline(plan, beam, depth=depth)
    hb = pinned(blocks)
    got = []
    for b in range(NBLOCKS):
        if b >= depth:
            got.append(pl.pop())
        pl.push(hb[b])
    while len(got) < NBLOCKS:
        got.append(pl.pop())
    pl.close()
    for (rec, n), (rrec, rn) in zip(got, ref):
        assert n == rn
        assert key(rec) == key(rrec)


@pytest.mark.parametrize("output,interm", [("plane", "u16"), ("cube", "f16"), ("series", "i32")])
def test_pipeline_outputs_match_block_by_block(tx, output, interm):
    plan, tail, blocks = stream_case(tx, output, interm=interm)
    ref = reference(tx, plan, tail, blocks)
    beam = tx.Beam(plan)
    beam.prime(tail)
    pl = tx.Pipeline(plan, beam, depth=2)
    hb = pinned(blocks)
    pl.push(hb[0])
    pl.push(hb[1])
    for b in range(NBLOCKS):
        out = pl.pop().numpy().copy()
        if b + 2 < NBLOCKS:
            pl.push(hb[b + 2])
        assert np.array_equal(out, ref[b])
    pl.close()


def test_pipeline_compact_beam(tx):
    plan, tail, blocks = stream_case(tx, "cands", snr_threshold=6.0, max_cands=1 << 14)
    ref = reference(tx, plan, tail, blocks)
    beam = tx.Beam(plan, compact=True)
    beam.prime(tail)
    pl = tx.Pipeline(plan, beam, depth=2)
    hb = pinned(blocks)
    got = []
    for b in range(NBLOCKS):
        if b >= 2:
            got.append(pl.pop())
        pl.push(hb[b])
    got += [pl.pop(), pl.pop()]
    pl.close()
    for (rec, n), (rrec, rn) in zip(got, ref):
        assert n == rn and key(rec) == key(rrec)


def test_pipeline_refuses_overfill_and_empty_pop(tx):
    plan, tail, blocks = stream_case(tx, "cands", snr_threshold=6.0, max_cands=1 << 14)
    beam = tx.Beam(plan)
    beam.prime(tail)
    pl = tx.Pipeline(plan, beam, depth=2)
    with pytest.raises(tx.TxError) as e:
        pl.pop()
    assert e.value.code == -1                       # TX_ERR_INVALID_ARG: nothing in flight
    hb = pinned(blocks)
    pl.push(hb[0])
    pl.push(hb[1])
    with pytest.raises(tx.TxError) as e:
        pl.push(hb[2])
    assert e.value.code == -7                       # TX_ERR_BUDGET: depth blocks in flight
    pl.pop()
    pl.push(hb[2])                                  # room again
    pl.pop()
    pl.pop()
    pl.close()


def test_pipeline_pop_times_out_then_completes(tx):
    """A bounded pop of a block held back by a fixed-length spin enqueued before
    it on the compute stream returns None; an unbounded pop then returns the
    block's correct results (nothing hangs, nothing is lost)."""
    plan, tail, blocks = stream_case(tx, "cands", snr_threshold=6.0, max_cands=1 << 14)
    ref = reference(tx, plan, tail, blocks[:1])
    beam = tx.Beam(plan)
    beam.prime(tail)
    pl = tx.Pipeline(plan, beam, depth=2)
    hb = pinned(blocks[:1])
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2e9))                     # ~1 s of spinning on the compute stream
    pl.push(hb[0])
    assert pl.pop(timeout_s=0.02) is None
    rec, n = pl.pop()
    assert n == ref[0][1] and key(rec) == key(ref[0][0])
    pl.close()
