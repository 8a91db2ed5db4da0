"""ctypes marshalling for libtransientx_gb300.so (argument conversion only)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libtransientx_gb300.so")

LAYOUTS = {"ft": 0, "tf": 1}
INTERMS = {"u16": 0, "i32": 1, "f16": 2, "f32": 3}
NORMS = {"none": 0, "unit": 1, "invvar": 2}
OUTPUTS = {"cands": 0, "plane": 1, "cube": 2, "series": 3}
STATS = {"block": 0, "running": 1}

TX_ERR_INVALID_ARG = -1
TX_ERR_TIMEOUT = -5
TX_ERR_CAND_OVERFLOW = -6
TX_ERR_ABORTED = -9

CAND_DTYPE = np.dtype([("dm_index", np.int32), ("t", np.int32), ("w_index", np.int32), ("snr", np.float32)])
CLUSTER_DTYPE = np.dtype([("id", np.int32), ("dm_index", np.int32), ("t", np.int32), ("w_index", np.int32),
                          ("snr", np.float32), ("members", np.int32), ("dm_lo", np.int32), ("dm_hi", np.int32),
                          ("t_lo", np.int32), ("t_hi", np.int32)])


class TxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"transientx error {code}: {msg}")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [
        ("nchan", C.c_int32), ("freq_mhz", C.POINTER(C.c_double)), ("tsamp_s", C.c_double),
        ("ndm", C.c_int32), ("dm", C.POINTER(C.c_double)), ("nsub", C.c_int32), ("group", C.c_int32),
        ("nwidth", C.c_int32), ("widths", C.POINTER(C.c_int32)), ("nsamp", C.c_int64),
        ("layout", C.c_int32), ("interm", C.c_int32), ("output", C.c_int32),
        ("snr_threshold", C.c_float), ("max_cands", C.c_int64), ("stats", C.c_int32),
        ("stats_lambda", C.c_double), ("tile_q1", C.c_int32), ("tile_split2", C.c_int32), ("norm", C.c_int32),
        ("tile_box", C.c_int32),
    ]


class _Info(C.Structure):
    _fields_ = [
        ("nchan", C.c_int32), ("nsub", C.c_int32), ("ndm", C.c_int32), ("ncoarse", C.c_int32),
        ("group", C.c_int32), ("nwidth", C.c_int32), ("wmax", C.c_int32), ("tile_box", C.c_int32),
        ("nsamp", C.c_int64), ("overlap", C.c_int64), ("max_delay", C.c_int64), ("series_len", C.c_int64),
        ("workspace_bytes", C.c_int64), ("beam_state_bytes", C.c_int64), ("out_bytes", C.c_int64),
        ("export_bytes", C.c_int64), ("block_bytes", C.c_int64), ("ring_len", C.c_int64),
        ("ring_head0", C.c_int64), ("tile_q1", C.c_int32), ("tile_split2", C.c_int32),
        ("workspace_bytes_compact", C.c_int64), ("compact_beam_state_bytes", C.c_int64),
    ]


class _Segment(C.Structure):
    _fields_ = [
        ("dm_lo", C.c_int32), ("dm_hi", C.c_int32), ("factor", C.c_int32), ("nwidth", C.c_int32),
        ("widths", C.c_int32 * 32), ("nsamp", C.c_int64), ("overlap", C.c_int64), ("native_offset", C.c_int64),
    ]


class _BatchInfo(C.Structure):
    _fields_ = [
        ("nbeams", C.c_int32), ("nwaves", C.c_int32), ("nlaunches", C.c_int32), ("flags", C.c_int32),
        ("workspace_bytes", C.c_int64), ("dm_trial_samples", C.c_int64),
    ]


TX_BATCH_GRAPH = 1
TX_BATCH_PROFILE = 2


def library_path() -> str:
    return _LIB_PATH


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"{_LIB_PATH} is missing: build it with `python -m paper_2401_13834_gb300.build` "
            "(there is no CPU fallback)")
    L = C.CDLL(_LIB_PATH)
    P, I32, I64, VP = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "tx_version": (I32, []),
        "tx_last_error": (I32, [C.c_char_p, C.c_size_t]),
        "tx_plan_create": (I32, [C.POINTER(_Desc), C.POINTER(P)]),
        "tx_plan_get_info": (I32, [P, C.POINTER(_Info)]),
        "tx_plan_tables": (I32, [P, VP, VP, VP, VP]),
        "tx_geometric_widths": (I32, [C.c_double, I32, VP, I32]),
        "tx_plan_stage1_layout": (I32, [P, C.POINTER(I64), C.POINTER(I64), VP]),
        "tx_plan_destroy": (None, [P]),
        "tx_beam_create": (I32, [P, C.POINTER(P)]),
        "tx_beam_create_compact": (I32, [P, C.POINTER(P)]),
        "tx_beam_reset": (I32, [P, P, VP]),
        "tx_beam_prime": (I32, [P, P, VP, VP]),
        "tx_beam_export": (I32, [P, P, VP, I64]),
        "tx_beam_import": (I32, [P, P, VP, I64]),
        "tx_beam_blocks": (I32, [P, C.POINTER(I64)]),
        "tx_beam_destroy": (None, [P]),
        "tx_execute": (I32, [P, P, VP, VP, VP, VP, VP]),
        "tx_execute_host": (I32, [P, P, VP, VP, VP, VP, VP, VP, VP, VP]),
        "tx_timer_create": (I32, [I32, C.POINTER(P)]),
        "tx_timer_clear": (I32, [P]),
        "tx_execute_timed": (I32, [P, P, VP, VP, VP, VP, VP, P]),
        "tx_timer_read": (I32, [P, VP, C.POINTER(I32), VP]),
        "tx_timer_destroy": (None, [P]),
        "tx_dedisperse_noalloc": (I32, [P, VP, I64, VP, VP]),
        "tx_batch_create": (I32, [I32, VP, VP, I64, I32, C.POINTER(P)]),
        "tx_batch_get_info": (I32, [P, C.POINTER(_BatchInfo)]),
        "tx_execute_batch": (I32, [P, VP, VP, VP, VP, VP]),
        "tx_batch_read_profile": (I32, [P, VP, C.POINTER(I32)]),
        "tx_batch_wait": (I32, [P, I64]),
        "tx_plan_delay_table": (I32, [P, VP]),
        "tx_plan_segments": (I32, [I32, VP, C.c_double, I32, VP, I32, VP]),
        "tx_downsample": (I32, [VP, I32, I32, I64, I32, VP, VP]),
        "tx_clusterer_create": (I32, [P, C.c_double, I32, I64, C.POINTER(P)]),
        "tx_cluster_run": (I32, [P, VP, I64, VP, VP, VP, VP, VP]),
        "tx_clusterer_destroy": (None, [P]),
        "tx_batch_destroy": (None, [P]),
        "tx_pipeline_create": (I32, [P, P, I32, VP, C.POINTER(P)]),
        "tx_pipeline_push": (I32, [P, VP]),
        "tx_pipeline_pop": (I32, [P, VP, VP, I64]),
        "tx_pipeline_destroy": (None, [P]),
        "tx_wait_timeouts": (I32, [C.POINTER(I64)]),
        "tx_set_wait_polls": (I32, [I64, C.POINTER(I64)]),
        "tx_measure_smem_bandwidth": (I32, [I32, C.POINTER(C.c_double), VP]),
        "tx_dsplan_create": (I32, [C.POINTER(_Desc), I32, C.POINTER(P)]),
        "tx_dsplan_get_info": (I32, [P, C.POINTER(I32), C.POINTER(I64)]),
        "tx_dsplan_segment": (I32, [P, I32, C.POINTER(_Segment), C.POINTER(P)]),
        "tx_dsplan_destroy": (None, [P]),
        "tx_beam_failed": (I32, [P, P, C.POINTER(I64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def version() -> int:
    return int(lib.tx_version())


def _check(rc):
    if rc != 0:
        buf = C.create_string_buffer(1024)
        lib.tx_last_error(buf, 1024)
        raise TxError(rc, buf.value.decode(errors="replace"))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def geometric_widths(ratio: float, wmax: int) -> np.ndarray:
    """Geometric boxcar ladder from the library (Sec. 2.4)."""
    n = lib.tx_geometric_widths(float(ratio), int(wmax), None, 0)
    if n < 0:
        _check(n)
    out = np.zeros(n, dtype=np.int32)
    lib.tx_geometric_widths(float(ratio), int(wmax), out.ctypes.data_as(C.c_void_p), n)
    return out


def _make_desc(keep, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, group, layout, interm, output, snr_threshold,
               max_cands, stats, stats_lambda, tile_q1, tile_split2, norm="none", tile_box=0):
    """A tx_plan_desc over arrays kept alive in `keep` (a dict)."""
    keep["freqs"] = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    keep["dms"] = np.ascontiguousarray(dms, dtype=np.float64)
    keep["widths"] = np.ascontiguousarray(widths, dtype=np.int32)
    d = _Desc()
    d.nchan = keep["freqs"].size
    d.freq_mhz = keep["freqs"].ctypes.data_as(C.POINTER(C.c_double))
    d.tsamp_s = float(tsamp_s)
    d.ndm = keep["dms"].size
    d.dm = keep["dms"].ctypes.data_as(C.POINTER(C.c_double))
    d.nsub = int(nsub)
    d.group = int(group)
    d.nwidth = keep["widths"].size
    d.widths = keep["widths"].ctypes.data_as(C.POINTER(C.c_int32))
    d.nsamp = int(nsamp)
    d.layout = LAYOUTS[layout]
    d.interm = INTERMS[interm]
    d.output = OUTPUTS[output]
    d.snr_threshold = float(snr_threshold)
    d.max_cands = int(max_cands)
    d.stats = STATS[stats]
    d.stats_lambda = float(stats_lambda)
    d.tile_q1 = int(tile_q1)
    d.tile_split2 = int(tile_split2)
    d.norm = NORMS[norm]
    d.tile_box = int(tile_box)
    return d


class Plan:
    """A de-dispersion + matched-filter plan (tables on the host until first use)."""

    @classmethod
    def _wrap(cls, handle, owner, freqs_mhz, dms, widths, layout, interm, output, stats, snr_threshold, max_cands):
        """A Plan over a handle that `owner` holds (and frees): a segment of a downsampled plan."""
        self = cls.__new__(cls)
        self._owner = owner
        self.norm = "none"
        self.freqs = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.widths = np.ascontiguousarray(widths, dtype=np.int32)
        self.layout, self.interm, self.output, self.stats = layout, interm, output, stats
        self.snr_threshold, self.max_cands = float(snr_threshold), int(max_cands)
        self._h = None
        self._borrowed = handle
        self._read_info(handle)
        return self

    def _read_info(self, h):
        inf = _Info()
        _check(lib.tx_plan_get_info(h, C.byref(inf)))
        self.info = {k: int(getattr(inf, k)) for k, _ in _Info._fields_}
        for k, v in self.info.items():
            setattr(self, k, v)

    def __init__(self, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, group=0, layout="ft", interm="u16",
                 output="cands", snr_threshold=6.0, max_cands=1 << 20, stats="block", stats_lambda=0.25,
                 tile_q1=0, tile_split2=0, norm="none", tile_box=0):
        if norm != "none" and interm == "u16":
            interm = "f32"                     # a normalisation runs the float path
        keep = {}
        d = _make_desc(keep, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, group, layout, interm, output,
                       snr_threshold, max_cands, stats, stats_lambda, tile_q1, tile_split2, norm, tile_box)
        self.norm = norm
        self.freqs, self.dms, self.widths = keep["freqs"], keep["dms"], keep["widths"]
        self.layout, self.interm, self.output, self.stats = layout, interm, output, stats
        self.snr_threshold = float(snr_threshold)
        self.max_cands = int(max_cands)
        h = C.c_void_p()
        _check(lib.tx_plan_create(C.byref(d), C.byref(h)))
        self._h = h
        self._read_info(h)

    @property
    def handle(self):
        return self._h if self._h is not None else getattr(self, "_borrowed", None)

    def tables(self):
        nk, nc, nd, ns = self.ncoarse, self.nchan, self.ndm, self.nsub
        d1 = np.zeros((nk, nc), dtype=np.int32)
        d2 = np.zeros((nd, ns), dtype=np.int32)
        kof = np.zeros(nd, dtype=np.int32)
        cdm = np.zeros(nk, dtype=np.float64)
        _check(lib.tx_plan_tables(self.handle, d1.ctypes.data_as(C.c_void_p), d2.ctypes.data_as(C.c_void_p),
                                  kof.ctypes.data_as(C.c_void_p), cdm.ctypes.data_as(C.c_void_p)))
        return {"d1": d1, "d2": d2, "coarse_of_fine": kof, "coarse_dm": cdm}

    def delay_table(self):
        """Delay of each DM trial across the band, ms (the clustering axis)."""
        out = np.zeros(self.ndm, dtype=np.float64)
        _check(lib.tx_plan_delay_table(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def stage1_layout(self):
        off, pitch = C.c_int64(), C.c_int64()
        base = np.zeros((self.ncoarse, self.nsub), dtype=np.int32)
        _check(lib.tx_plan_stage1_layout(self.handle, C.byref(off), C.byref(pitch), base.ctypes.data_as(C.c_void_p)))
        return int(off.value), int(pitch.value), base

    def alloc_workspace(self, device=None, compact=False):
        """Workspace of one execute (on a compact beam: with room for its borrowed ring)."""
        import torch
        n = self.workspace_bytes_compact if compact else self.workspace_bytes
        return torch.empty(n, dtype=torch.uint8, device=device or "cuda")

    def alloc_out(self, device=None):
        import torch
        dev = device or "cuda"
        if self.output == "cands":
            return (torch.empty((self.max_cands, 4), dtype=torch.int32, device=dev),
                    torch.zeros(1, dtype=torch.int64, device=dev))
        return torch.empty(self.out_bytes, dtype=torch.uint8, device=dev), None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_plan_destroy(h)
            self._h = None


class Beam:
    """Per-beam device state: the carried tail and running statistics.

    A full beam keeps a circular buffer of L + T samples per channel resident;
    a compact beam (``compact=True``) only the L-sample tail, and borrows the
    buffer from each execute's workspace (``plan.alloc_workspace(compact=True)``).
    """

    def __init__(self, plan: Plan, compact: bool = False):
        self.plan = plan
        self.compact = bool(compact)
        h = C.c_void_p()
        _check((lib.tx_beam_create_compact if compact else lib.tx_beam_create)(plan.handle, C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def reset(self, stream=None):
        _check(lib.tx_beam_reset(self.plan.handle, self._h, _stream_ptr(stream)))

    def prime(self, tail, stream=None):
        """Set the carried tail from L samples (uint8 CUDA tensor in the plan's layout)."""
        assert tail.is_cuda and tail.dtype.is_floating_point is False and tail.numel() == self.plan.nchan * self.plan.overlap
        _check(lib.tx_beam_prime(self.plan.handle, self._h, _ptr(tail.contiguous()), _stream_ptr(stream)))

    def export(self) -> bytes:
        buf = (C.c_uint8 * self.plan.export_bytes)()
        _check(lib.tx_beam_export(self.plan.handle, self._h, buf, self.plan.export_bytes))
        return bytes(buf)

    def import_(self, state: bytes):
        buf = (C.c_uint8 * len(state)).from_buffer_copy(state)
        _check(lib.tx_beam_import(self.plan.handle, self._h, buf, len(state)))

    @property
    def nblocks(self) -> int:
        n = C.c_int64()
        _check(lib.tx_beam_blocks(self._h, C.byref(n)))
        return int(n.value)

    def failed(self) -> int:
        """Waits this beam's kernels gave up since create/reset/import (tx_beam_failed;
        synchronises the device). Nonzero: its results and state are not valid."""
        n = C.c_int64()
        _check(lib.tx_beam_failed(self.plan.handle, self._h, C.byref(n)))
        return int(n.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_beam_destroy(h)
            self._h = None


def execute(plan: Plan, beam: Beam, block, out=None, ncand=None, workspace=None, stream=None):
    """Run one block (uint8 CUDA tensor, nchan*T bytes in the plan's layout).

    Returns the raw output tensor(s) without synchronising: (out, ncand) for
    candidates, else out (uint8 bytes of the plan's output mode).
    """
    if out is None:
        out, ncand = plan.alloc_out(block.device)
    if workspace is None:
        workspace = plan.alloc_workspace(block.device, compact=beam.compact)
    assert block.is_cuda and block.numel() == plan.nchan * plan.nsamp and block.is_contiguous()
    _check(lib.tx_execute(plan.handle, beam.handle, _ptr(block), _ptr(out), _ptr(ncand), _ptr(workspace),
                          _stream_ptr(stream)))
    return (out, ncand) if plan.output == "cands" else out


PHASES = ("ingest", "stage1", "stage2", "stats", "boxcar")


class Timer:
    """CUDA events recorded between the phases of timed executes (on their stream)."""

    def clear(self):
        _check(lib.tx_timer_clear(self._h))

    def __init__(self, max_steps: int):
        h = C.c_void_p()
        _check(lib.tx_timer_create(int(max_steps), C.byref(h)))
        self._h = h
        self.max_steps = int(max_steps)

    def read(self):
        """(summed ms per phase, step count, per-step total ms) over the recorded steps."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        steps = np.zeros(self.max_steps, dtype=np.float64)
        n = C.c_int32()
        _check(lib.tx_timer_read(self._h, ms.ctypes.data_as(C.c_void_p), C.byref(n), steps.ctypes.data_as(C.c_void_p)))
        return dict(zip(PHASES, ms.tolist())), int(n.value), steps[:n.value]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_timer_destroy(h)
            self._h = None


def execute_timed(plan: Plan, beam: Beam, block, out, ncand, workspace, timer: Timer, stream=None):
    """``execute`` that also records the phase boundaries into ``timer``."""
    _check(lib.tx_execute_timed(plan.handle, beam.handle, _ptr(block), _ptr(out), _ptr(ncand), _ptr(workspace),
                                _stream_ptr(stream), timer._h))


def execute_host(plan: Plan, beam: Beam, h_block: np.ndarray, h_out: np.ndarray, staging, out, ncand,
                 workspace, stream=None):
    """Host-to-host execute through the C ABI (copies inside; synchronises).

    Returns the number of candidates (cands mode) or None.
    """
    h_block = np.ascontiguousarray(h_block)
    hn = np.zeros(1, dtype=np.int64)
    rc = lib.tx_execute_host(plan.handle, beam.handle, h_block.ctypes.data_as(C.c_void_p),
                             h_out.ctypes.data_as(C.c_void_p), hn.ctypes.data_as(C.c_void_p), _ptr(staging),
                             _ptr(out), _ptr(ncand), _ptr(workspace), _stream_ptr(stream))
    if rc not in (0, TX_ERR_CAND_OVERFLOW):
        _check(rc)
    return int(hn[0]) if plan.output == "cands" else None


def wait_timeouts() -> int:
    """Waits the kernels gave up on the current device (tx_wait_timeouts); 0 in normal operation."""
    n = C.c_int64()
    _check(lib.tx_wait_timeouts(C.byref(n)))
    return int(n.value)


def measure_smem_bandwidth(iters: int = 4096, stream=None) -> float:
    """Shared-memory read bandwidth of the current device, bytes/s (tx_measure_smem_bandwidth)."""
    v = C.c_double()
    _check(lib.tx_measure_smem_bandwidth(int(iters), C.byref(v), _stream_ptr(stream)))
    return float(v.value)


def set_wait_polls(polls: int) -> int:
    """Polling limit of the kernels' first wait for each bulk copy (tx_set_wait_polls);
    returns the previous one. 0 makes every such wait give up at once (tests only)."""
    old = C.c_int64()
    _check(lib.tx_set_wait_polls(int(polls), C.byref(old)))
    return int(old.value)


class Pipeline:
    """A stream of one beam's host blocks with up to ``depth`` in flight
    (tx_pipeline_*): ``push`` enqueues a block's copy and kernels, ``pop``
    returns the oldest block's results. Input blocks should be pinned uint8
    tensors (or numpy arrays) of nchan * T bytes in the plan's layout, kept
    unchanged until their pop returns. The plan and beam must outlive it.
    """

    def __init__(self, plan: Plan, beam: Beam, depth: int = 2, stream=None):
        import torch
        self.plan, self.beam, self.depth = plan, beam, int(depth)
        h = C.c_void_p()
        _check(lib.tx_pipeline_create(plan.handle, beam.handle, self.depth, _stream_ptr(stream), C.byref(h)))
        self._h = h
        self._inflight = []
        nbytes = plan.max_cands * CAND_DTYPE.itemsize if plan.output == "cands" else plan.out_bytes
        self.h_out = torch.empty(max(nbytes, 1), dtype=torch.uint8, pin_memory=True)
        self._hn = np.zeros(1, dtype=np.int64)

    def push(self, h_block):
        n = self.plan.nchan * self.plan.nsamp
        if isinstance(h_block, np.ndarray):
            assert h_block.flags.c_contiguous and h_block.nbytes == n
            ptr = h_block.ctypes.data
        else:
            assert not h_block.is_cuda and h_block.is_contiguous() and h_block.numel() * h_block.element_size() == n
            ptr = h_block.data_ptr()
        _check(lib.tx_pipeline_push(self._h, C.c_void_p(ptr)))
        self._inflight.append(h_block)    # keeps the block alive until its pop

    def pop(self, timeout_s=None):
        """The oldest block's results, or None if ``timeout_s`` ran out first (pop
        again). Candidate mode: (records, n) with n the count found (records hold
        min(n, max_cands)); other modes: the raw output bytes (pinned; copy them
        before the next pop)."""
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc = lib.tx_pipeline_pop(self._h, C.c_void_p(self.h_out.data_ptr()), self._hn.ctypes.data_as(C.c_void_p), us)
        if rc == TX_ERR_TIMEOUT:
            return None
        if rc == TX_ERR_ABORTED:
            self._inflight.pop(0)          # popped; its results are not valid
        if rc not in (0, TX_ERR_CAND_OVERFLOW):
            _check(rc)
        self._inflight.pop(0)
        if self.plan.output == "cands":
            n = int(self._hn[0])
            k = min(n, self.plan.max_cands)
            return self.h_out.numpy()[: k * CAND_DTYPE.itemsize].view(CAND_DTYPE).copy(), n
        return self.h_out

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib.tx_pipeline_destroy(self._h)
            self._h = None
            self._inflight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- decoding helpers (views of the raw output, no arithmetic) -------------
def cands_view(plan: Plan, out, ncand):
    import torch
    n = min(int(ncand.item()), plan.max_cands)
    raw = out[:n].contiguous().cpu().numpy()
    return raw.view(CAND_DTYPE).reshape(-1), int(ncand.item())


def plane_view(plan: Plan, out):
    import torch
    nd, T = plan.ndm, plan.nsamp
    snr = out[: nd * T * 4].view(torch.float32).view(nd, T)
    w = out[nd * T * 4: nd * T * 5].view(nd, T)
    return snr, w


def cube_view(plan: Plan, out):
    import torch
    return out.view(torch.float32).view(plan.ndm, plan.nwidth, plan.nsamp)


def series_view(plan: Plan, out):
    import torch
    dt = torch.float32 if plan.interm == "f32" else torch.int32   # float series on the float path
    return out.view(dt).view(plan.ndm, plan.series_len)


def dedisperse_noalloc(plan: Plan, x, ld: int, series, stream=None):
    """De-dispersed series of one window through the allocation-free entry point.

    x: contiguous uint8 CUDA tensor holding [nchan][ld] (tail then block);
    series: contiguous int32 CUDA tensor of ndm * (T + W_max - 1) elements.
    Nothing is allocated. The tensors are checked here (device, dtype,
    contiguity, size) because the library sees only their addresses.
    """
    import torch
    ld = int(ld)
    args = (("x", x, torch.uint8, plan.nchan * ld), ("series", series, torch.int32, plan.ndm * plan.series_len))
    for name, t, dt, n in args:
        if not isinstance(t, torch.Tensor):
            raise TxError(TX_ERR_INVALID_ARG, f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise TxError(TX_ERR_INVALID_ARG, f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise TxError(TX_ERR_INVALID_ARG, f"{name} must be contiguous")
        if t.numel() < n:
            raise TxError(TX_ERR_INVALID_ARG, f"{name} holds {t.numel()} elements, needs {n}")
    for name, t, _, _ in args:
        if not t.is_cuda:
            raise TxError(TX_ERR_INVALID_ARG, f"{name} must be a CUDA tensor")
    _check(lib.tx_dedisperse_noalloc(plan.handle, _ptr(x), ld, _ptr(series), _stream_ptr(stream)))


class Batch:
    """Many (plan, beam) pairs run one block each per step (tx_execute_batch).

    ``workspace_budget`` > 0 splits the beams into waves that share a workspace
    of at most that many bytes; ``graph`` replays the step's launches as CUDA
    graphs; ``profile`` (direct launches) times every launch for
    ``read_profile``. The plans and beams must outlive the batch.
    """

    def __init__(self, plans, beams, workspace_budget=0, graph=True, profile=False):
        assert len(plans) == len(beams) and len(plans) > 0
        self.plans, self.beams = list(plans), list(beams)
        n = len(plans)
        ph = (C.c_void_p * n)(*[p.handle.value for p in plans])
        bh = (C.c_void_p * n)(*[b.handle.value for b in beams])
        h = C.c_void_p()
        flags = (TX_BATCH_GRAPH if graph else 0) | (TX_BATCH_PROFILE if profile else 0)
        _check(lib.tx_batch_create(n, ph, bh, int(workspace_budget), flags, C.byref(h)))
        self._h = h
        inf = _BatchInfo()
        _check(lib.tx_batch_get_info(h, C.byref(inf)))
        self.info = {k: int(getattr(inf, k)) for k, _ in _BatchInfo._fields_}
        for k, v in self.info.items():
            setattr(self, k, v)

    def alloc_workspace(self, device=None):
        import torch
        return torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=device or "cuda")

    def alloc_outs(self, device=None):
        """[(out, ncand or None)] per beam."""
        return [p.alloc_out(device) for p in self.plans]

    def execute(self, blocks, outs, workspace, stream=None):
        """One block per beam (uint8 CUDA tensors); outs as from alloc_outs."""
        n = len(self.plans)
        assert len(blocks) == n and len(outs) == n
        for p, blk in zip(self.plans, blocks):
            assert blk.is_cuda and blk.is_contiguous() and blk.numel() == p.nchan * p.nsamp
        bp = (C.c_void_p * n)(*[b.data_ptr() for b in blocks])
        op = (C.c_void_p * n)(*[o.data_ptr() for o, _ in outs])
        cp = (C.c_void_p * n)(*[0 if c is None else c.data_ptr() for _, c in outs])
        _check(lib.tx_execute_batch(self._h, bp, op, cp, _ptr(workspace), _stream_ptr(stream)))

    def wait(self, timeout_s=None) -> bool:
        """Waits for the last step; False if `timeout_s` ran out first (nothing is cancelled)."""
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc = lib.tx_batch_wait(self._h, us)
        if rc == TX_ERR_TIMEOUT:
            return False
        _check(rc)
        return True

    def read_profile(self):
        """(summed ms per phase over the profiled steps, step count)."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        n = C.c_int32()
        _check(lib.tx_batch_read_profile(self._h, ms.ctypes.data_as(C.c_void_p), C.byref(n)))
        return dict(zip(PHASES, ms.tolist())), int(n.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_batch_destroy(h)
            self._h = None


class Clusterer:
    """DBSCAN of a block's candidates on the GPU (tx_cluster_run)."""

    def __init__(self, plan: Plan, radius_ms: float, k: int, max_points: int):
        self.plan = plan
        self.max_points = int(max_points)
        h = C.c_void_p()
        _check(lib.tx_clusterer_create(plan.handle, float(radius_ms), int(k), self.max_points, C.byref(h)))
        self._h = h

    def run(self, cands, n: int, out=None, nclusters=None, labels=None, order=None, stream=None):
        """cands: the device candidate buffer (records); n: how many. Returns (out, nclusters)
        device tensors (out holds int32 [n, 10] cluster records)."""
        import torch
        dev = cands.device
        if out is None:
            out = torch.empty((max(int(n), 1), 10), dtype=torch.int32, device=dev)
        if nclusters is None:
            nclusters = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(lib.tx_cluster_run(self._h, _ptr(cands), int(n), _ptr(out), _ptr(nclusters), _ptr(labels),
                                  _ptr(order), _stream_ptr(stream)))
        return out, nclusters

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_clusterer_destroy(h)
            self._h = None


def clusters_view(out, nclusters):
    """Host structured array of the cluster records."""
    n = int(nclusters.item())
    return out[:n].contiguous().cpu().numpy().view(CLUSTER_DTYPE).reshape(-1)


class DsPlan:
    """tx_dsplan: a DM grid split into downsampled segments, each with its own plan."""

    def __init__(self, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, f_max=64, group=0, layout="ft", interm="u16",
                 output="cands", snr_threshold=6.0, max_cands=1 << 20, stats="block", stats_lambda=0.25,
                 tile_q1=0, tile_split2=0):
        keep = {}
        d = _make_desc(keep, freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, group, layout, interm, output,
                       snr_threshold, max_cands, stats, stats_lambda, tile_q1, tile_split2)
        h = C.c_void_p()
        _check(lib.tx_dsplan_create(C.byref(d), int(f_max), C.byref(h)))
        self._h = h
        n, L = C.c_int32(), C.c_int64()
        _check(lib.tx_dsplan_get_info(h, C.byref(n), C.byref(L)))
        self.overlap = int(L.value)
        self.segments = []
        for j in range(n.value):
            sg, ph = _Segment(), C.c_void_p()
            _check(lib.tx_dsplan_segment(h, j, C.byref(sg), C.byref(ph)))
            w = np.array(sg.widths[:sg.nwidth], dtype=np.int32)
            plan = Plan._wrap(ph, self, keep["freqs"], keep["dms"][sg.dm_lo:sg.dm_hi], w, layout, interm, output,
                              stats, snr_threshold, max_cands)
            self.segments.append(dict(dm_lo=sg.dm_lo, dm_hi=sg.dm_hi, factor=sg.factor, widths=w,
                                      nsamp=sg.nsamp, overlap=sg.overlap, native_offset=sg.native_offset,
                                      plan=plan))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            lib.tx_dsplan_destroy(h)
            self._h = None


def segment_factors(freqs_mhz, tsamp_s, dms, f_max: int = 64) -> np.ndarray:
    """Downsampling factor of every DM trial (tx_plan_segments)."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.zeros(d.size, dtype=np.int32)
    _check(lib.tx_plan_segments(f.size, f.ctypes.data_as(C.c_void_p), float(tsamp_s), d.size,
                                d.ctypes.data_as(C.c_void_p), int(f_max), out.ctypes.data_as(C.c_void_p)))
    return out


def downsample(x, layout: str, nchan: int, nsamp: int, factor: int, out=None, stream=None):
    """tx_downsample of a uint8 CUDA tensor; returns the downsampled tensor."""
    import torch
    if out is None:
        out = torch.empty(nchan * (nsamp // factor), dtype=torch.uint8, device=x.device)
    _check(lib.tx_downsample(_ptr(x), LAYOUTS[layout], int(nchan), int(nsamp), int(factor), _ptr(out),
                             _stream_ptr(stream)))
    return out
