"""Continuous-batching request loop: blocks of many beams on one GPU.

The paper processes each beam as a stream of blocks with a carried overlap
(Sec. 2.3 data flow) and sizes blocks at about a second of data (Sec. 3). A
server takes such blocks from many beams as they arrive, at any time:

* every beam is a compact beam: its overlap tail and running statistics stay
  resident on the device between blocks;
* a block is admitted, in arrival order, when its beam has no block on the
  device (a beam's blocks depend on each other through the tail) and the
  block's workspace and output fit the HBM budget next to everything already
  admitted;
* all blocks admitted since the last launch go to the GPU together as one
  batched step (tx_execute_batch), on one of two streams, so a new step is
  launched while the previous one is still running and their work overlaps
  on the device; memory of a step returns to the budget when it completes;
* a block's latency runs from its arrival to its results being on the host;
* a step whose kernels gave up a bounded wait (tx_beam_failed) completes its
  jobs with ``error`` set and no result, and takes the beams concerned out
  of service: their carried state is no longer valid.

The GPU side is behind a small engine interface (launch / done / finish), so
the scheduling logic also runs, and is tested, with a simulated engine.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable, Optional

import numpy as np


@dataclasses.dataclass
class Job:
    """One block of one beam."""
    beam: int
    block: Any                 # device tensor (the plan's layout), or whatever the engine takes
    arrival: float
    seq: int                   # position in the beam's stream of blocks
    reserve: int               # bytes held against the budget while admitted
    admitted: Optional[float] = None
    launched: Optional[float] = None
    done: Optional[float] = None
    result: Any = None
    error: Optional[str] = None   # set when the block's results are not valid

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class Server:
    """Admission, batching and completion of beam blocks (see the module doc)."""

    def __init__(self, engine, budget_bytes: int, max_batch: int = 64, nstreams: int = 2,
                 clock: Callable[[], float] = time.perf_counter):
        if nstreams < 1 or max_batch < 1:
            raise ValueError("need nstreams >= 1 and max_batch >= 1")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.nstreams = int(nstreams)
        self.clock = clock
        self.beams = []                    # per beam: (plan, reserve bytes)
        self.busy = []                     # per beam: a block of it is admitted or on the device
        self.next_seq = []
        self.pending = collections.deque()  # submitted, not admitted (arrival order)
        self.ready = []                    # admitted, not launched
        self.inflight = []                 # (handle, stream index, jobs)
        self.reserved = 0
        self.peak_reserved = 0
        self.completed = []
        self.steps = 0
        self.batch_sizes = []
        self.t0 = None
        self.removed = set()

    # ---- set-up ---------------------------------------------------------------
    def add_beam(self, plan, reserve_bytes: Optional[int] = None) -> int:
        """Registers a beam of `plan` (the engine makes its resident state); returns its id."""
        reserve = int(self.engine.reserve_bytes(plan) if reserve_bytes is None else reserve_bytes)
        if reserve > self.budget:
            raise ValueError(f"a block of this plan needs {reserve} bytes, more than the budget {self.budget}")
        bid = len(self.beams)
        self.engine.add_beam(bid, plan)
        self.beams.append((plan, reserve))
        self.busy.append(False)
        self.next_seq.append(0)
        return bid

    def remove_beam(self, beam: int) -> list:
        """Takes a beam out of service: its blocks not yet admitted are dropped
        (returned); a block already on the device completes normally."""
        dropped = [j for j in self.pending if j.beam == beam]
        self.pending = collections.deque(j for j in self.pending if j.beam != beam)
        self.removed.add(beam)
        return dropped

    # ---- requests -----------------------------------------------------------------
    def submit(self, beam: int, block, arrival: Optional[float] = None) -> Job:
        if beam in self.removed or not 0 <= beam < len(self.beams):
            raise ValueError(f"beam {beam} is not in service")
        check = getattr(self.engine, "check_block", None)
        if check is not None:
            check(self.beams[beam][0], block)      # a malformed block is refused here, not on the GPU
        now = self.clock()
        if self.t0 is None:
            self.t0 = now
        job = Job(beam=beam, block=block, arrival=now if arrival is None else arrival, seq=self.next_seq[beam],
                  reserve=self.beams[beam][1])
        self.next_seq[beam] += 1
        self.pending.append(job)
        return job

    # ---- the loop ----------------------------------------------------------------
    def _complete(self):
        out = []
        still = []
        for h, s, jobs in self.inflight:
            if self.engine.done(h):
                self.engine.finish(h, jobs)
                t = self.clock()
                for j in jobs:
                    j.done = t
                    self.busy[j.beam] = False
                    self.reserved -= j.reserve
                    if j.error is not None:
                        self.remove_beam(j.beam)
                out += jobs
            else:
                still.append((h, s, jobs))
        self.inflight = still
        self.completed += out
        return out

    def _admit(self):
        # arrival order; a beam's later blocks wait behind its earlier ones
        blocked = set()
        keep = collections.deque()
        now = self.clock()
        while self.pending:
            j = self.pending.popleft()
            if j.beam in blocked or self.busy[j.beam] or self.reserved + j.reserve > self.budget:
                blocked.add(j.beam)
                keep.append(j)
                continue
            self.busy[j.beam] = True
            self.reserved += j.reserve
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            j.admitted = now
            self.ready.append(j)
        self.pending = keep

    def _launch(self):
        while self.ready and len(self.inflight) < self.nstreams:
            used = {s for _, s, _ in self.inflight}
            s = min(set(range(self.nstreams)) - used)
            jobs, self.ready = self.ready[:self.max_batch], self.ready[self.max_batch:]
            t = self.clock()
            for j in jobs:
                j.launched = t
            h = self.engine.launch(jobs, s)
            self.inflight.append((h, s, jobs))
            self.steps += 1
            self.batch_sizes.append(len(jobs))

    def pump(self):
        """One pass: completions, admissions, launches. Returns the newly completed jobs."""
        done = self._complete()
        self._admit()
        self._launch()
        return done

    def idle(self) -> bool:
        return not (self.pending or self.ready or self.inflight)

    def drain(self, poll_s: float = 0.0, timeout_s: Optional[float] = None):
        """Pumps until idle; raises TimeoutError if `timeout_s` (on the server's clock) runs out."""
        t0 = self.clock()
        while not self.idle():
            self.pump()
            if timeout_s is not None and self.clock() - t0 > timeout_s:
                raise TimeoutError(f"{len(self.inflight)} steps still running and {len(self.pending)} blocks "
                                   f"waiting after {timeout_s} s")
            if poll_s:
                time.sleep(poll_s)

    def reset_stats(self):
        """Forgets completed blocks and step counts (after a warm-up)."""
        self.completed = []
        self.batch_sizes = []
        self.steps = 0
        self.peak_reserved = self.reserved
        self.t0 = None

    # ---- metrics ----------------------------------------------------------------------
    def stats(self, data_seconds: Optional[Callable[[Job], float]] = None) -> dict:
        lat = np.array([j.latency for j in self.completed if j.latency is not None])
        if not len(lat):
            return {"blocks": 0}
        span = max(j.done for j in self.completed) - min(j.arrival for j in self.completed)
        out = {
            "blocks": int(len(lat)), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "max_latency_s": float(lat.max()),
            "span_s": float(span), "beam_blocks_per_s": float(len(lat) / span) if span > 0 else None,
            "steps": self.steps, "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
            "peak_reserved_bytes": int(self.peak_reserved), "budget_bytes": int(self.budget),
        }
        if data_seconds is not None and span > 0:
            out["real_time_factor"] = float(sum(data_seconds(j) for j in self.completed) / span)
        return out


class TxEngine:
    """The GPU engine: compact beams, one tx_execute_batch per launch, results to the host.

    `results` selects what finish() brings back per job: "cands" (records and
    the count), "raw" (the whole output buffer) or None (nothing).
    """

    def __init__(self, tx, device=None, nstreams: int = 2, results: str = "cands"):
        import torch
        self.tx, self.torch = tx, torch
        self.device = torch.device(device or "cuda")
        self.streams = [torch.cuda.Stream(self.device) for _ in range(nstreams)]
        self.beams = {}
        self.results = results

    @staticmethod
    def reserve_bytes(plan) -> int:
        return int(plan.workspace_bytes_compact + plan.out_bytes + 8)

    def check_block(self, plan, block):
        torch = self.torch
        if not (isinstance(block, torch.Tensor) and block.is_cuda and block.dtype == torch.uint8
                and block.is_contiguous() and block.numel() == plan.nchan * plan.nsamp):
            raise ValueError(f"a block of this beam is a contiguous uint8 CUDA tensor of {plan.nchan * plan.nsamp} "
                             "samples")

    def add_beam(self, bid, plan):
        self.beams[bid] = (plan, self.tx.Beam(plan, compact=True))

    def beam(self, bid):
        return self.beams[bid][1]

    def launch(self, jobs, s):
        torch, tx = self.torch, self.tx
        st = self.streams[s]
        plans = [self.beams[j.beam][0] for j in jobs]
        beams = [self.beams[j.beam][1] for j in jobs]
        with torch.cuda.stream(st):
            batch = tx.Batch(plans, beams, graph=False)
            ws = batch.alloc_workspace(self.device)
            outs = batch.alloc_outs(self.device)
            # the blocks were produced on other streams: order them before this step
            st.wait_stream(torch.cuda.default_stream(self.device))
            batch.execute([j.block for j in jobs], outs, ws, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"batch": batch, "ws": ws, "outs": outs, "ev": ev, "stream": st}

    def done(self, h) -> bool:
        return h["ev"].query()

    def finish(self, h, jobs):
        torch, tx = self.torch, self.tx
        try:
            h["batch"].wait()          # also checks that no member's kernels gave up a wait
        except tx.TxError as e:
            if e.code != tx.TX_ERR_ABORTED:
                raise
            for j in jobs:
                if self.beams[j.beam][1].failed():
                    j.error = "aborted: a kernel gave up a bounded wait"
        with torch.cuda.stream(h["stream"]):
            for j, p, (o, nc) in zip(jobs, [self.beams[j.beam][0] for j in jobs], h["outs"]):
                if j.error is not None:
                    j.result = None
                elif self.results is None:
                    j.result = None
                elif self.results == "cands" and p.output == "cands":
                    n = int(nc.item())
                    j.result = (n, o[:min(n, p.max_cands)].cpu().numpy())
                else:
                    j.result = o.cpu().numpy()
        h.clear()   # frees the batch, its workspace and outputs (tensors return to the allocator)


class SimEngine:
    """A stand-in engine for testing the scheduling: each launch takes a given
    time per job on a simulated clock; results are the jobs' sequence numbers.
    `stall` makes every launch from then on never finish (a hung step, made
    on the host)."""

    def __init__(self, cost: Callable[[Any], float], clock):
        self.cost, self.clock = cost, clock
        self.plans = {}
        self.launches = []
        self.stall = False

    def check_block(self, plan, block):
        if block is not None and block != plan.get("block", block):
            raise ValueError("malformed block")

    def reserve_bytes(self, plan) -> int:
        return int(plan["reserve"])

    def add_beam(self, bid, plan):
        self.plans[bid] = plan

    def launch(self, jobs, s):
        t = self.clock()
        end = float("inf") if self.stall else t + sum(self.cost(self.plans[j.beam]) for j in jobs)
        h = {"end": end, "jobs": list(jobs), "stream": s}
        self.launches.append(h)
        return h

    def done(self, h) -> bool:
        return self.clock() >= h["end"]

    def finish(self, h, jobs):
        for j in jobs:
            j.result = (j.beam, j.seq)
