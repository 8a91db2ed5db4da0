"""Autotuner for a plan's free choices on the current GPU.

Sec. 2.3 leaves the sub-band count N_s and the coarse DM grid to the
implementation; the kernels add tile shapes. For one beam shape the tuner
times candidate plans through the library (one block each, CUDA events,
median of a few executes after a warm-up) and keeps the fastest:

  1. N_s over the divisors of nchan giving 32..128 channels per sub-band, with
     the automatic group size G and automatic tiles;
  2. G in {automatic, automatic / 2} for the best N_s: never coarser than the
     automatic rule (whose coarse grid keeps the intra-sub-band smear below the
     fine grid's), sometimes finer, which trades stage-2 work for stage 1;
  3. the stage-1 tile length (tile_q1) among those that fit shared memory;
  4. the stage-2 warps per fine DM (tile_split2) among the valid ones.

N_s and G change which sums are formed (all of them valid sub-band
de-dispersion); tile shapes never change results. Choices are cached in a
JSON file keyed by the GPU name and the beam shape.

    python -m paper_2401_13834_gb300.autotune --workload batched [--out FILE]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuned", "gb300.json")


def shape_key(wl, layout, output, interm) -> str:
    """Identifies a beam shape: sizes, band, sampling, DM grid, widths and modes."""
    h = hashlib.sha1()
    for a in (np.asarray(wl.freqs_mhz, np.float64), np.asarray(wl.dms, np.float64), np.asarray(wl.widths, np.int32)):
        h.update(a.tobytes())
    h.update(repr((float(wl.tsamp_s), int(wl.nsamp), layout, output, interm)).encode())
    return f"{wl.nchan}ch-{wl.ndm}dm-T{wl.nsamp}-{layout}-{output}-{interm}-{h.hexdigest()[:12]}"


def load_cache(path=DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(wl, layout="tf", output="cands", interm="u16", path=DEFAULT_CACHE, gpu=None):
    """The cached choice for this shape on this GPU (a dict of Plan keywords), or None."""
    import torch
    gpu = gpu or torch.cuda.get_device_name()
    ent = load_cache(path).get(gpu, {}).get(shape_key(wl, layout, output, interm))
    return None if ent is None else {k: ent[k] for k in ("nsub", "group", "tile_q1", "tile_split2")}


class _Timer:
    """Times executes of candidate plans on one random block of the beam shape."""

    def __init__(self, tx, wl, layout, output, interm, snr_threshold, max_cands, reps):
        import torch
        self.tx, self.wl, self.torch = tx, wl, torch
        self.layout, self.output, self.interm = layout, output, interm
        self.snr_threshold, self.max_cands, self.reps = snr_threshold, max_cands, reps
        g = torch.Generator(device="cuda")
        g.manual_seed(12345)
        n = wl.nchan * wl.nsamp
        x = torch.randn(n, generator=g, device="cuda", dtype=torch.float32)
        self.block = x.mul_(float(wl.noise_std)).add_(float(wl.noise_mean)).round_().clamp_(0, 255).to(torch.uint8)
        del x
        self.ws = None

    def plan(self, nsub, group=0, tile_q1=0, tile_split2=0):
        wl = self.wl
        return self.tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, nsub, wl.widths, wl.nsamp, group=group,
                            layout=self.layout, interm=self.interm, output=self.output,
                            snr_threshold=self.snr_threshold, max_cands=self.max_cands,
                            tile_q1=tile_q1, tile_split2=tile_split2)

    def time(self, plan) -> float:
        torch, tx = self.torch, self.tx
        if self.ws is None or self.ws.numel() < plan.workspace_bytes:
            self.ws = None
            torch.cuda.empty_cache()
            self.ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
        beam = tx.Beam(plan)
        out, nc = plan.alloc_out()
        tx.execute(plan, beam, self.block, out=out, ncand=nc, workspace=self.ws)
        ms = []
        for _ in range(self.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tx.execute(plan, beam, self.block, out=out, ncand=nc, workspace=self.ws)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        del beam, out, nc
        return statistics.median(ms)


def tune(wl, layout="tf", output="cands", interm="u16", snr_threshold=7.0, max_cands=1 << 22, reps=3,
         verbose=False) -> dict:
    """Times the staged candidate set for one beam shape; returns the fastest choice and the trials."""
    import paper_2401_13834_gb300 as tx
    tm = _Timer(tx, wl, layout, output, interm, snr_threshold, max_cands, reps)
    trials = []

    def run(**kw):
        try:
            p = tm.plan(**kw)
        except tx.TxError:
            return None
        ms = tm.time(p)
        rec = dict(nsub=p.nsub, group=p.group, tile_q1=p.tile_q1, tile_split2=p.tile_split2, ms=ms)
        trials.append(rec)
        if verbose:
            print(f"  {wl.name}: {rec}", flush=True)
        return rec

    def best(recs):
        recs = [r for r in recs if r is not None]
        return min(recs, key=lambda r: r["ms"]) if recs else None

    nsubs = [wl.nchan // m for m in (32, 64, 128) if wl.nchan % m == 0 and wl.nchan // m >= 1]
    b = best(run(nsub=s) for s in nsubs)
    auto_g = b["group"]
    b = best([b] + ([run(nsub=b["nsub"], group=auto_g // 2)] if auto_g >= 2 else []))
    b = best([b] + [run(nsub=b["nsub"], group=b["group"], tile_q1=q) for q in (32, 64, 128, 256)
                    if q != b["tile_q1"]])
    splits = [s for s in (1, 2, 4, 8) if min(b["group"], 32) * s <= 32 and s != b["tile_split2"]]
    b = best([b] + [run(nsub=b["nsub"], group=b["group"], tile_q1=b["tile_q1"], tile_split2=s) for s in splits])
    tm.ws = None
    return dict(b, trials=trials)


def tune_all(workloads, layout="tf", output="cands", interm="u16", path=DEFAULT_CACHE, verbose=False, **kw):
    """Tunes every distinct shape among ``workloads`` not yet cached for this GPU; saves the cache."""
    import torch
    gpu = torch.cuda.get_device_name()
    cache = load_cache(path)
    mine = cache.setdefault(gpu, {})
    for wl in workloads:
        key = shape_key(wl, layout, output, interm)
        if key in mine:
            continue
        res = tune(wl, layout, output, interm, verbose=verbose, **kw)
        mine[key] = res
        save_cache(cache, path)
        if verbose:
            print(f"{key}: nsub {res['nsub']} group {res['group']} q1 {res['tile_q1']} split {res['tile_split2']} "
                  f"{res['ms']:.3f} ms", flush=True)
    return cache


def main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["batched", "meerkat_l", "small"], default="batched")
    ap.add_argument("--layout", default="tf")
    ap.add_argument("--output", default="cands")
    ap.add_argument("--out", default=DEFAULT_CACHE)
    args = ap.parse_args()
    from paper_2401_13834_gb300 import build
    build.build()
    wls = synth.batched_workloads() if args.workload == "batched" else [synth.WORKLOADS[args.workload]()]
    tune_all(wls, args.layout, args.output, path=args.out, verbose=True)


if __name__ == "__main__":
    main()
