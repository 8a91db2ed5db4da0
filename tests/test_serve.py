"""The serving loop on the GPU: each result is the same alone and in the mix.

Several beams of different shapes stream blocks into one Server (compact
beams, mixed batched steps on two streams, a budget small enough that blocks
wait for memory). Every block's result must equal what the beam gives when it
runs alone, block after block, on a full beam through tx_execute: bit for bit
for the plane and series outputs, the same records for candidates.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NBLK = 3


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


SHAPES = [
    (dict(nchan=64, nsub=8, ndm=37, nsamp=1500, group=5), dict(output="cands", layout="tf", snr_threshold=3.0)),
    (dict(nchan=128, nsub=16, ndm=64, nsamp=4096, dm_max=400.0, tsamp=128e-6), dict(output="cands", layout="ft",
                                                                                 snr_threshold=3.5)),
    (dict(nchan=48, nsub=48, ndm=9, nsamp=777, group=4), dict(output="plane", layout="ft")),
    (dict(nchan=96, nsub=8, ndm=24, nsamp=2048, descending=True), dict(output="series", layout="tf")),
]


def to_layout(X, layout):
    return np.ascontiguousarray(X.T if layout == "tf" else X)


def norm(plan, res):
    if plan.output == "cands":
        n, rec = res
        rec = np.ascontiguousarray(rec).view(np.dtype([("d", "<i4"), ("t", "<i4"), ("w", "<i4"), ("s", "<f4")]))
        return n, np.sort(rec.reshape(-1), order=("d", "t"))
    return res


def test_each_result_same_alone_and_in_the_mix(tx):
    from paper_2401_13834_gb300.serve import Server, TxEngine
    plans, streams = [], []
    rng = np.random.default_rng(5)
    for wk, pk in SHAPES * 2:                      # two beams of every shape
        wl = synth.tiny_workload(**wk)
        p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group,
                    stats="running", **pk)
        plans.append(p)
        streams.append(rng.integers(0, 256, size=(p.nchan, p.overlap + NBLK * p.nsamp), dtype=np.uint8))

    def block(i, k):
        p, X = plans[i], streams[i]
        return torch.from_numpy(to_layout(X[:, p.overlap + k * p.nsamp:p.overlap + (k + 1) * p.nsamp], p.layout)).cuda()

    # alone: full beams, one tx_execute per block
    alone = []
    for i, p in enumerate(plans):
        b = tx.Beam(p)
        b.prime(torch.from_numpy(to_layout(streams[i][:, :p.overlap], p.layout)).cuda())
        ws = p.alloc_workspace()
        res = []
        for k in range(NBLK):
            out, nc = p.alloc_out()
            tx.execute(p, b, block(i, k), out=out, ncand=nc, workspace=ws)
            torch.cuda.synchronize()
            if p.output == "cands":
                n = int(nc.item())
                res.append((n, out[:n].cpu().numpy()))
            else:
                res.append(out.cpu().numpy())
        alone.append(res)

    # in the mix: compact beams in a server with a budget of about three blocks
    eng = TxEngine(tx, results="cands")
    budget = 3 * max(TxEngine.reserve_bytes(p) for p in plans)
    srv = Server(eng, budget, max_batch=6, nstreams=2)
    ids = []
    for i, p in enumerate(plans):
        bid = srv.add_beam(p)
        eng.beam(bid).prime(torch.from_numpy(to_layout(streams[i][:, :p.overlap], p.layout)).cuda())
        ids.append(bid)
    torch.cuda.synchronize()
    order = [(i, k) for k in range(NBLK) for i in range(len(plans))]
    rng.shuffle(order)
    order.sort(key=lambda ik: ik[1])               # a beam's blocks stay in order; beams interleave
    jobs = {}
    for n, (i, k) in enumerate(order):
        jobs[(i, k)] = srv.submit(ids[i], block(i, k))
        if n % 3 == 2:
            srv.pump()                             # arrivals meet steps already on the device
    srv.drain()
    assert srv.peak_reserved <= budget
    assert max(srv.batch_sizes) > 1               # blocks of several beams shared steps
    for (i, k), j in jobs.items():
        p = plans[i]
        assert j.seq == k
        got, ref = norm(p, j.result), norm(p, alone[i][k])
        if p.output == "cands":
            assert got[0] == ref[0] and np.array_equal(got[1], ref[1]), (i, k)
        else:
            assert np.array_equal(got, ref), (i, k)
