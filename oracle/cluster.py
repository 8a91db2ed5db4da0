"""Oracle for candidate clustering (Sec. 2.5): DBSCAN on the DM-time plane.

Test infrastructure: only tests, the smoke check and the benchmark's CPU legs
use this module; the library never does.

Sec. 2.5 turns the S/N cube into the DM-time plane (best width per point),
keeps the points at or above the threshold, converts DM to dispersion delay
(Eq. 1) so that both axes are in milliseconds, and runs DBSCAN: a core point
has more than k neighbours within radius r; a reachable point is not core but
lies within r of a core point; other points are outliers; clusters are the
density-reachable sets of core points with their reachable points. Written
here as plain loops over an all-pairs distance test.

Readings (the paper leaves them open):
* delay of DM d = K DM_d (f_min^-2 - f_max^-2), the delay across the band, in
  ms; time = t * t_samp in ms;
* "within the radius": distance <= r; "exceeds k": more than k neighbours,
  the point itself not counted;
* the order of points is canonical, by (DM index, time); a cluster's id is
  the smallest canonical index among its core points; a reachable point next
  to several clusters joins the one with the smallest id (every label is then
  unique);
* a cluster is reported by its member of highest S/N (ties: smallest
  canonical index), with its member count and DM and time extents.
"""
from __future__ import annotations

import numpy as np

K_DM = 4.148808e3   # s MHz^2 pc^-1 cm^3 (Eq. 1)


def delay_ms(dms, f_min_mhz, f_max_mhz) -> np.ndarray:
    """Eq. 1 across the band, in milliseconds, float64."""
    dms = np.asarray(dms, dtype=np.float64)
    return K_DM * dms * (1.0 / (f_min_mhz * f_min_mhz) - 1.0 / (f_max_mhz * f_max_mhz)) * 1e3


def canonical_order(dm_index, t) -> np.ndarray:
    """Permutation that sorts points by (DM index, time)."""
    return np.lexsort((np.asarray(t), np.asarray(dm_index)))


def dbscan(x, y, r, k):
    """DBSCAN of points (x[i], y[i]) in canonical order.

    Returns (labels, core): labels[i] = cluster id (the smallest index of the
    cluster's core points) or -1 for an outlier; core[i] = more than k other
    points at distance <= r.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.size
    r2 = float(r) * float(r)
    nbr = []
    for i in range(n):
        dx = x - x[i]
        dy = y - y[i]
        d2 = dx * dx + dy * dy
        m = d2 <= r2
        m[i] = False
        nbr.append(np.flatnonzero(m))
    core = np.array([len(nb) > k for nb in nbr], dtype=bool)
    labels = np.full(n, -1, dtype=np.int64)
    # clusters: density-reachable sets grown from core points in canonical order
    for i in range(n):
        if not core[i] or labels[i] != -1:
            continue
        labels[i] = i                      # the first core point reached is the smallest index
        stack = [i]
        while stack:
            p = stack.pop()
            for q in nbr[p]:
                if core[q] and labels[q] == -1:
                    labels[q] = i
                    stack.append(q)
    # reachable points: the smallest id among their core neighbours
    for i in range(n):
        if core[i]:
            continue
        ids = [labels[q] for q in nbr[i] if core[q]]
        labels[i] = min(ids) if ids else -1
    return labels, core


def cluster_candidates(cands, delay_table_ms, tsamp_s, r_ms, k):
    """Clusters candidate records (fields dm_index, t, w_index, snr).

    Returns (order, labels, core, clusters): `order` is the canonical
    permutation of the records; labels/core are in canonical order; clusters
    is a list of dicts (id, dm_index, t, w_index, snr, members, dm_lo, dm_hi,
    t_lo, t_hi) sorted by id.
    """
    d = np.asarray(cands["dm_index"], dtype=np.int64)
    t = np.asarray(cands["t"], dtype=np.int64)
    order = canonical_order(d, t)
    d, t = d[order], t[order]
    w = np.asarray(cands["w_index"], dtype=np.int64)[order]
    snr = np.asarray(cands["snr"], dtype=np.float32)[order]
    x = np.asarray(delay_table_ms, dtype=np.float64)[d]
    y = t.astype(np.float64) * (tsamp_s * 1e3)
    labels, core = dbscan(x, y, r_ms, k)
    clusters = []
    for cid in sorted(set(labels.tolist()) - {-1}):
        mem = np.flatnonzero(labels == cid)
        best = mem[0]
        for i in mem[1:]:
            if snr[i] > snr[best]:
                best = i
        clusters.append(dict(id=int(cid), dm_index=int(d[best]), t=int(t[best]), w_index=int(w[best]),
                             snr=float(snr[best]), members=int(mem.size), dm_lo=int(d[mem].min()),
                             dm_hi=int(d[mem].max()), t_lo=int(t[mem].min()), t_hi=int(t[mem].max())))
    return order, labels, core, clusters
