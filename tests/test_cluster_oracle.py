"""Pins of the clustering oracle (Sec. 2.5 DBSCAN) on the CPU.

Hand-made point sets whose clusters follow from the definitions, and
scikit-learn's DBSCAN (an independent implementation: eps = r inclusive,
min_samples = k + 2 counting the point itself) on random clustered points:
the core points, their partition into clusters and the outliers must agree.
"""
import numpy as np
import pytest

from oracle import cluster as C


def test_chain_at_exactly_r_is_one_cluster():
    # points r apart on a line: interior points have 2 neighbours, the ends 1
    r = 1.5
    x = np.arange(6) * r
    labels, core = C.dbscan(x, np.zeros(6), r, k=1)
    assert list(core) == [False, True, True, True, True, False]
    assert list(labels) == [1, 1, 1, 1, 1, 1]      # ends are reachable; id = smallest core index


def test_chain_just_beyond_r_is_all_outliers():
    r = 1.5
    x = np.arange(6) * r * (1 + 1e-9)
    labels, core = C.dbscan(x, np.zeros(6), r, k=0)
    assert not core.any() and (labels == -1).all()


def test_k_counts_others_strictly():
    # three points within r of each other: two neighbours each
    x = np.array([0.0, 0.5, 1.0])
    assert C.dbscan(x, np.zeros(3), 1.0, k=1)[1].all()       # 2 > 1
    assert not C.dbscan(x, np.zeros(3), 1.0, k=2)[1].any()   # 2 > 2 fails


def test_border_point_joins_smallest_cluster_id():
    # two groups of four mutually close points (3 neighbours each: core for k = 2) and
    # a middle point whose only neighbours are one point of each group (2: not core)
    a = [(0.05, 0.0), (-0.4, 0.0), (-0.45, 0.05), (-0.45, -0.05)]
    b = [(1.95, 0.0), (2.4, 0.0), (2.45, 0.05), (2.45, -0.05)]
    x, y = np.array(a + b + [(1.0, 0.0)]).T
    labels, core = C.dbscan(x, y, r=1.0, k=2)
    assert list(core) == [True] * 8 + [False]
    assert list(labels) == [0] * 4 + [4] * 4 + [0]


def test_two_blobs_and_outliers():
    rng = np.random.default_rng(0)
    a = rng.normal([0, 0], 0.2, size=(40, 2))
    b = rng.normal([10, 10], 0.2, size=(30, 2))
    o = np.array([[5, 5], [20, 0], [-8, 3]])
    p = np.vstack([a, b, o])
    labels, core = C.dbscan(p[:, 0], p[:, 1], r=1.0, k=3)
    assert len(set(labels[:40])) == 1 and len(set(labels[40:70])) == 1 and labels[0] != labels[40]
    assert list(labels[70:]) == [-1, -1, -1]


def test_against_scikit_learn():
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(7)
    centres = rng.uniform(0, 50, size=(12, 2))
    p = np.vstack([rng.normal(c, rng.uniform(0.3, 1.5), size=(rng.integers(5, 60), 2)) for c in centres]
                  + [rng.uniform(0, 50, size=(80, 2))])
    for r, k in ((1.0, 2), (1.7, 4), (0.6, 0)):
        labels, core = C.dbscan(p[:, 0], p[:, 1], r, k)
        ref = sk.DBSCAN(eps=r, min_samples=k + 2).fit(p)
        ref_core = np.zeros(len(p), dtype=bool)
        ref_core[ref.core_sample_indices_] = True
        assert np.array_equal(core, ref_core)
        assert np.array_equal(labels == -1, ref.labels_ == -1)       # the same outliers
        # the same partition of the core points
        for lab in set(labels[core]):
            ids = set(ref.labels_[core & (labels == lab)])
            assert len(ids) == 1
            (rid,) = ids
            assert np.array_equal(core & (labels == lab), core & (ref.labels_ == rid))
        # every reachable point is within r of a core point of its cluster
        for i in np.flatnonzero(~core & (labels >= 0)):
            mem = np.flatnonzero(core & (labels == labels[i]))
            assert (np.hypot(p[mem, 0] - p[i, 0], p[mem, 1] - p[i, 1]) <= r).any()


def test_cluster_candidates_reduces_to_best_member():
    rec = np.zeros(6, dtype=[("dm_index", "<i4"), ("t", "<i4"), ("w_index", "<i4"), ("snr", "<f4")])
    rec["dm_index"] = [5, 5, 6, 6, 40, 5]
    rec["t"] = [100, 101, 100, 102, 500, 103]
    rec["w_index"] = [0, 1, 2, 3, 0, 1]
    rec["snr"] = [7.0, 9.5, 8.0, 9.5, 12.0, 7.2]
    table = C.delay_ms(np.arange(64) * 0.1, 1200.0, 1456.0)      # 0.092 ms per DM step
    order, labels, core, clusters = C.cluster_candidates(rec, table, 64e-6, r_ms=0.5, k=1)
    assert [c["members"] for c in clusters] == [5]
    c = clusters[0]
    # the best S/N 9.5 appears twice: the earlier point in (DM, t) order wins
    assert (c["dm_index"], c["t"], c["snr"]) == (5, 101, 9.5)
    assert (c["dm_lo"], c["dm_hi"], c["t_lo"], c["t_hi"]) == (5, 6, 100, 103)
    assert labels[order.tolist().index(4)] == -1               # the far point is an outlier


def test_delay_table_closed_form():
    # K * DM * (1/f1^2 - 1/f2^2): DM 1 across 1000-2000 MHz is 4.148808e3 * 0.75e-6 s = 3.111606 ms
    assert C.delay_ms([1.0], 1000.0, 2000.0)[0] == pytest.approx(3.111606, rel=1e-12)
