"""GB300-native sub-band de-dispersion + boxcar matched filter (TransientX hot path).

A thin ctypes binding over the C ABI declared in include/transientx.h; every
step of the computation runs in the library's CUDA kernels. PyTorch provides
device memory and streams only. There is no CPU fallback: the first use of any
name below loads libtransientx_gb300.so and raises ImportError if it is
missing (build it with ``python -m paper_2401_13834_gb300.build``).

    plan = Plan(freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, output="cands")
    beam = Beam(plan)
    beam.prime(tail_u8_cuda)            # optional: the first L samples
    res = execute(plan, beam, block_u8_cuda)
"""
from __future__ import annotations

_EXPORTS = (
    "LAYOUTS", "INTERMS", "OUTPUTS", "STATS", "CAND_DTYPE", "PHASES", "TxError", "Plan", "Beam", "Timer",
    "execute", "execute_timed", "execute_host", "geometric_widths", "lib", "library_path", "version",
    "cands_view", "plane_view", "cube_view", "series_view", "dedisperse_noalloc", "Batch", "Clusterer",
    "clusters_view", "CLUSTER_DTYPE", "segment_factors", "downsample", "Pipeline", "wait_timeouts",
    "set_wait_polls", "measure_smem_bandwidth", "TX_ERR_ABORTED", "TX_ERR_TIMEOUT", "TX_ERR_INVALID_ARG",
)
__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import _native
        return getattr(_native, name)
    raise AttributeError(name)
