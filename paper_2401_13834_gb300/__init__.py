"""GB300-native sub-band de-dispersion + boxcar matched filter (TransientX hot path).

A thin ctypes binding over the C ABI declared in include/transientx.h; every
step of the computation runs in the library's CUDA kernels. PyTorch provides
device memory and streams only. There is no CPU fallback: if the shared
library is missing the import of the native layer raises.

    plan = Plan(freqs_mhz, tsamp_s, dms, nsub, widths, nsamp, output="cands")
    beam = Beam(plan)
    beam.prime(tail_u8_cuda)            # optional: the first L samples
    res = execute(plan, beam, block_u8_cuda)
"""
from __future__ import annotations

from ._native import (  # noqa: F401
    LAYOUTS, INTERMS, OUTPUTS, STATS, CAND_DTYPE, TxError, Plan, Beam, execute, execute_host,
    geometric_widths, lib, library_path, version, cands_view, plane_view, cube_view, series_view,
    PHASES, Timer, execute_timed,
)
