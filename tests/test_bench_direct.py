"""The bench's brute-force timing leg on the CPU (no GPU needed).

cpu_direct times the oracle's direct de-dispersion of one block: every DM
trial when its budget allows, else a spread subset with the whole block's
time extrapolated from the time per trial.
"""
import importlib.util
import os
import sys

import numpy as np

import synth
from oracle import dedisp as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _block(wl):
    op = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, 0, wl.widths)
    X = np.random.default_rng(1).integers(0, 256, size=(wl.nchan, op.overlap + wl.nsamp), dtype=np.uint8)
    return op, X


def test_direct_leg_whole_block():
    b = _bench()
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=12, nsamp=800, dm_max=80.0, widths=(1, 2, 4, 8, 16, 32))
    op, X = _block(wl)
    assert O.direct_delays(wl.freqs_mhz, wl.tsamp_s, wl.dms).max() <= op.overlap   # the window holds every track
    r = b.cpu_direct(wl, X, 30.0)
    assert r["whole_block_extrapolated"] is False and r["sample"].startswith("all of 12 DM trials x 800 of 800")
    assert r["value"] > 0 and r["unit"] == b.UNIT and r["cores"] == 1
    assert abs(r["whole_block_s"] - 12 * wl.nsamp / r["value"]) <= 1e-9 * r["whole_block_s"]


def test_direct_leg_short_window_and_subset():
    b = _bench()
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=40, nsamp=800, dm_max=80.0, widths=(1, 2))
    op, X = _block(wl)
    dmax = int(O.direct_delays(wl.freqs_mhz, wl.tsamp_s, wl.dms).max())
    nout = min(wl.nsamp, X.shape[1] - dmax)   # the direct tracks may pass the sub-band overlap
    r = b.cpu_direct(wl, X, 0.0)               # the budget ends after the first trial
    assert r["sample"].startswith(f"1 of 40 DM trials x {nout} of 800") and r["whole_block_extrapolated"] is True
    # the whole block's time: per trial and per output, scaled to every trial and T outputs
    assert abs(r["whole_block_s"] - 40 * wl.nsamp / r["value"]) <= 1e-9 * r["whole_block_s"]
