"""GPU clustering (tx_cluster_run) against the DBSCAN oracle.

Labels of every point (in canonical (DM, time) order) and the cluster records
must equal the oracle's exactly: coordinates, distances and every decision
are computed the same way in IEEE double, and the labelling rules leave no
choice (a cluster's id is its first core point; a border point joins the
smallest id). The input order of the records must not matter.
"""
import numpy as np
import pytest

import synth
from oracle import cluster as CL

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


def records(d, t, w, snr):
    r = np.zeros(len(d), dtype=[("dm_index", "<i4"), ("t", "<i4"), ("w_index", "<i4"), ("snr", "<f4")])
    r["dm_index"], r["t"], r["w_index"], r["snr"] = d, t, w, snr
    return r


def gpu_cluster(tx, plan, rec, r_ms, k):
    n = len(rec)
    dev = torch.from_numpy(np.ascontiguousarray(rec).view(np.int32).reshape(-1, 4).copy()).cuda()
    cl = tx.Clusterer(plan, r_ms, k, max(n, 1))
    labels = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    out, nc = cl.run(dev, n, labels=labels, order=order)
    torch.cuda.synchronize()
    return tx.clusters_view(out, nc), labels[:n].cpu().numpy(), order[:n].cpu().numpy()


def check(tx, plan, rec, r_ms, k):
    got, labels, order = gpu_cluster(tx, plan, rec, r_ms, k)
    o_order, o_labels, o_core, o_cl = CL.cluster_candidates(rec, plan.delay_table(), plan_tsamp(plan), r_ms, k)
    assert np.array_equal(order, o_order)
    assert np.array_equal(labels, o_labels)
    assert len(got) == len(o_cl)
    for g, c in zip(got, o_cl):
        assert (int(g["id"]), int(g["dm_index"]), int(g["t"]), int(g["w_index"]), int(g["members"]),
                int(g["dm_lo"]), int(g["dm_hi"]), int(g["t_lo"]), int(g["t_hi"])) == (
            c["id"], c["dm_index"], c["t"], c["w_index"], c["members"], c["dm_lo"], c["dm_hi"], c["t_lo"], c["t_hi"])
        assert float(g["snr"]) == np.float32(c["snr"])
    return got, labels


_TSAMP = {}


def plan_tsamp(plan):
    return _TSAMP[id(plan)]


def make_plan(tx, wl):
    p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp)
    _TSAMP[id(p)] = wl.tsamp_s
    return p


def clustered_points(rng, ndm, T, nclus, per, noise):
    d, t = [], []
    for _ in range(nclus):
        cd, ct = rng.integers(0, ndm), rng.integers(0, T)
        m = rng.integers(1, per)
        d += list(np.clip(np.round(rng.normal(cd, rng.uniform(0.5, 6), m)), 0, ndm - 1).astype(int))
        t += list(np.clip(np.round(rng.normal(ct, rng.uniform(1, 30), m)), 0, T - 1).astype(int))
    d += list(rng.integers(0, ndm, noise))
    t += list(rng.integers(0, T, noise))
    key = sorted(set(zip(d, t)))                     # a plane point appears once
    rng.shuffle(key)
    d, t = np.array(key).T
    return records(d, t, rng.integers(0, 7, len(d)), rng.uniform(6, 30, len(d)).astype(np.float32))


@pytest.mark.parametrize("r_ms,k", [(0.5, 2), (1.5, 5), (3.0, 0)])
def test_clusters_equal_oracle(tx, r_ms, k):
    wl = synth.small_workload()
    plan = make_plan(tx, wl)
    rec = clustered_points(np.random.default_rng(int(r_ms * 10) + k), wl.ndm, wl.nsamp, 40, 200, 400)
    got, labels = check(tx, plan, rec, r_ms, k)
    assert len(got) > 3 and (labels == -1).any()


def test_input_order_does_not_matter(tx):
    wl = synth.small_workload()
    plan = make_plan(tx, wl)
    rec = clustered_points(np.random.default_rng(3), wl.ndm, wl.nsamp, 20, 300, 100)
    a, la, _ = gpu_cluster(tx, plan, rec, 1.0, 3)
    b, lb, _ = gpu_cluster(tx, plan, rec[::-1].copy(), 1.0, 3)
    assert np.array_equal(a, b) and np.array_equal(la, lb)


def test_edge_cases(tx):
    wl = synth.small_workload()
    plan = make_plan(tx, wl)
    got, labels, _ = gpu_cluster(tx, plan, records([], [], [], []), 1.0, 1)
    assert len(got) == 0
    got, labels, _ = gpu_cluster(tx, plan, records([5], [7], [1], [9.0]), 1.0, 0)
    assert len(got) == 0 and list(labels) == [-1]                 # a lone point has no neighbours
    far = records(np.arange(0, 120, 10), np.arange(0, 12000, 1000), np.zeros(12), np.full(12, 8.0))
    check(tx, plan, far, 0.3, 0)                                  # all outliers
    dense = records(np.repeat(np.arange(10), 50), np.tile(np.arange(50), 10), np.zeros(500), np.linspace(6, 9, 500))
    got, _ = check(tx, plan, dense, 2.0, 3)                       # one cluster
    assert len(got) == 1 and int(got[0]["members"]) == 500


def test_candidates_of_a_block(tx):
    """The small workload's own candidates (pulse and noise points) clustered."""
    wl = synth.small_workload()
    p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, output="cands", snr_threshold=4.0,
                max_cands=1 << 20)
    _TSAMP[id(p)] = wl.tsamp_s
    X = synth.make_spectrum(wl, p.overlap + wl.nsamp, synth.small_pulses(wl), seed=0)
    beam = tx.Beam(p)
    beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :p.overlap])).cuda())
    out, nc = tx.execute(p, beam, torch.from_numpy(np.ascontiguousarray(X[:, p.overlap:])).cuda())
    rec, n = tx.cands_view(p, out, nc)
    assert n > 100
    got, labels = check(tx, p, rec, 2.0, 4)
    # the injected pulse (DM 100, t ~ 0.37 T + smear) is the brightest cluster
    best = got[np.argmax(got["snr"])]
    assert abs(wl.dms[best["dm_index"]] - 100.0) < 10.0
