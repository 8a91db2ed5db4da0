"""De-dispersion plans with downsampling (Sec. 2.3, last paragraph).

At high DM the smearing inside one channel exceeds the sampling time, so a
plan de-disperses each DM range on data downsampled to about that smearing.
The library makes the plan (tx_dsplan_create): every DM trial gets its factor
(the largest power of two not above the Eq. 1 delay across the lowest
channel, in samples, and dividing the block), runs of equal factors become
segments, and segment j is an ordinary plan with sampling time f_j t_samp,
blocks of T / f_j samples and widths W / f_j (at least 1, duplicates
dropped); its input is the block averaged over f_j samples per channel
(tx_downsample, rounded half up, still uint8). All segments of a block run
as one batched step. This module only marshals those calls.

Times: the library gives each segment its native offset, L - f_j L_j (L the
native overlap, L_j the segment's); segment j's output t' then refers to
native window time f_j t' + offset_j (native_time()).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import _native as N


@dataclasses.dataclass
class Segment:
    dm_lo: int          # first DM trial (index into the full DM list)
    dm_hi: int          # one past the last
    factor: int
    widths: np.ndarray  # in downsampled samples
    plan: "N.Plan"
    native_offset: int  # native window time of output 0


class DownsampledPlan:
    """Segments of a DM grid de-dispersed at their own time resolution."""

    def __init__(self, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, f_max: int = 64, group: int = 0, **plan_kw):
        self._ds = N.DsPlan(freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, f_max=f_max, group=group, **plan_kw)
        self.nsamp = int(nsamp)
        self.segments = [Segment(s["dm_lo"], s["dm_hi"], s["factor"], s["widths"], s["plan"], s["native_offset"])
                         for s in self._ds.segments]
        self.overlap = self._ds.overlap
        self.layout = self.segments[0].plan.layout
        self.nchan = self.segments[0].plan.nchan
        self.ndm = int(np.asarray(dms).size)

    # ---- work, for the record ------------------------------------------------------
    def relative_stage1_work(self) -> float:
        """Stage-1 sample-adds against the same DM grid at full resolution (~ sum nk_j / f_j)."""
        return sum(s.plan.ncoarse / s.factor for s in self.segments) / sum(s.plan.ncoarse for s in self.segments)

    # ---- beams ------------------------------------------------------------------------
    def beams(self, compact: bool = False):
        return [N.Beam(s.plan, compact=compact) for s in self.segments]

    def _window(self, x, n_native, keep):
        """The last `keep` native samples of x (n_native samples, plan layout), contiguous."""
        if self.layout == "tf":
            return x.view(n_native, self.nchan)[n_native - keep:].contiguous()
        return x.view(self.nchan, n_native)[:, n_native - keep:].contiguous()

    def prime(self, beams, tail):
        """tail: the `overlap` native samples before the first block (device, plan layout)."""
        for s, b in zip(self.segments, beams):
            keep = s.factor * s.plan.overlap
            if keep == 0:
                continue
            w = self._window(tail, self.overlap, keep)
            b.prime(N.downsample(w, self.layout, self.nchan, keep, s.factor) if s.factor > 1 else w)

    def batch(self, beams, workspace_budget: int = 0, graph: bool = False) -> "N.Batch":
        return N.Batch([s.plan for s in self.segments], beams, workspace_budget=workspace_budget, graph=graph)

    def alloc_staging(self, device=None):
        """Per segment: a buffer for the downsampled block (None at factor 1)."""
        import torch
        return [None if s.factor == 1 else
                torch.empty(self.nchan * (self.nsamp // s.factor), dtype=torch.uint8, device=device or "cuda")
                for s in self.segments]

    def execute(self, batch, block, outs, workspace, staging, stream=None):
        """One native block (device, plan layout) through every segment as one batched step."""
        blocks = []
        for s, st in zip(self.segments, staging):
            if s.factor == 1:
                blocks.append(block)
            else:
                blocks.append(N.downsample(block, self.layout, self.nchan, self.nsamp, s.factor, out=st, stream=stream))
        batch.execute(blocks, outs, workspace, stream=stream)

    # ---- outputs -------------------------------------------------------------------
    def native_time(self, j: int, t):
        """Native window time of segment j's output times t (the library's offset; see the module doc)."""
        s = self.segments[j]
        return s.factor * np.asarray(t, dtype=np.int64) + s.native_offset

    def merge_cands(self, outs):
        """All segments' candidates as one structured array with global DM index and
        native window time (widths stay per segment: w_index indexes its widths)."""
        recs = []
        for j, (s, (o, nc)) in enumerate(zip(self.segments, outs)):
            r, _ = N.cands_view(s.plan, o, nc)
            r = r.copy()
            seg = np.full(r.size, j, dtype=np.int32)
            r["dm_index"] += s.dm_lo
            t = self.native_time(j, r["t"])
            recs.append((r, t, seg))
        dt = np.dtype([("dm_index", "<i4"), ("t_native", "<i8"), ("segment", "<i4"), ("w_index", "<i4"),
                       ("snr", "<f4")])
        out = np.zeros(sum(r.size for r, _, _ in recs), dtype=dt)
        i = 0
        for r, t, seg in recs:
            n = r.size
            out["dm_index"][i:i + n] = r["dm_index"]
            out["t_native"][i:i + n] = t
            out["segment"][i:i + n] = seg
            out["w_index"][i:i + n] = r["w_index"]
            out["snr"][i:i + n] = r["snr"]
            i += n
        return out
