"""Bounded device waits: none gave up during the suite, and the give-up path
reports itself when it is taken.

Collected after every other GPU test except the allocation-free one (which
comes last): first, no kernel of any earlier test gave up a bounded wait on a
bulk copy (tx_wait_timeouts counts them on the device). Then the failure path
is driven on purpose without any fault: a polling limit of 0
(tx_set_wait_polls) makes every kernel's first wait give up at once, after
which the kernel waits at the full limit for its copies in flight and
returns. The calls that wait on the host must then say so (TX_ERR_ABORTED),
the beam must be marked (tx_beam_failed) until it is reset, and the counter
must have grown. After the limit is restored and the beam reset, results are
exact again.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def test_no_kernel_gave_up_a_wait(tx):
    assert tx.wait_timeouts() == 0


def _setup(tx, output="cands"):
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=37, nsamp=1500, group=5)
    kw = dict(snr_threshold=3.0, max_cands=1 << 16) if output == "cands" else {}
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, output=output,
                   **kw)
    X = np.random.default_rng(5).integers(0, 256, size=(plan.nchan, plan.overlap + plan.nsamp), dtype=np.uint8)
    tail = torch.from_numpy(np.ascontiguousarray(X[:, :plan.overlap])).cuda()
    return plan, X, tail


class _Polls:
    """Polling limit 0 inside the block; the default restored on the way out."""

    def __init__(self, tx):
        self.tx = tx

    def __enter__(self):
        self.old = self.tx.set_wait_polls(0)

    def __exit__(self, *exc):
        torch.cuda.synchronize()
        self.tx.set_wait_polls(self.old)


def test_give_up_is_reported_by_execute_host_and_marks_the_beam(tx):
    plan, X, tail = _setup(tx, output="series")
    beam = tx.Beam(plan)
    beam.prime(tail)
    ws = plan.alloc_workspace()
    out, _ = plan.alloc_out()
    staging = torch.empty(plan.block_bytes, dtype=torch.uint8, device="cuda")
    h_out = np.zeros(plan.out_bytes, dtype=np.uint8)
    blk = np.ascontiguousarray(X[:, plan.overlap:])
    before = tx.wait_timeouts()
    with _Polls(tx):
        with pytest.raises(tx.TxError) as e:
            tx.execute_host(plan, beam, blk, h_out, staging, out, None, ws)
    assert e.value.code == tx.TX_ERR_ABORTED
    assert beam.failed() > 0
    assert tx.wait_timeouts() > before
    # still marked on the next call, whatever it computes, until the beam is reset
    with pytest.raises(tx.TxError) as e:
        tx.execute_host(plan, beam, blk, h_out, staging, out, None, ws)
    assert e.value.code == tx.TX_ERR_ABORTED
    beam.reset()
    beam.prime(tail)
    assert beam.failed() == 0
    tx.execute_host(plan, beam, blk, h_out, staging, out, None, ws)
    ref_beam = tx.Beam(plan)
    ref_beam.prime(tail)
    ref = tx.execute(plan, ref_beam, torch.from_numpy(blk).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(h_out, ref.cpu().numpy())


def test_give_up_is_reported_by_batch_wait_and_pipeline_pop(tx):
    plan, X, tail = _setup(tx)
    blk = np.ascontiguousarray(X[:, plan.overlap:])
    beam = tx.Beam(plan)
    beam.prime(tail)
    batch = tx.Batch([plan], [beam], graph=False)
    ws, outs = batch.alloc_workspace(), batch.alloc_outs()
    with _Polls(tx):
        batch.execute([torch.from_numpy(blk).cuda()], outs, ws)
        with pytest.raises(tx.TxError) as e:
            batch.wait()
    assert e.value.code == tx.TX_ERR_ABORTED and "beam 0" in str(e.value)
    beam2 = tx.Beam(plan)
    beam2.prime(tail)
    pl = tx.Pipeline(plan, beam2, depth=1)
    pinned = torch.from_numpy(blk).pin_memory()
    with _Polls(tx):
        pl.push(pinned)
        with pytest.raises(tx.TxError) as e:
            pl.pop()
    assert e.value.code == tx.TX_ERR_ABORTED
    assert beam2.failed() > 0
    pl.close()
