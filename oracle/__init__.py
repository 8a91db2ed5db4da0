"""Plain CPU oracle for TransientX's de-dispersion + matched-filter path.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import, call or run anything in this package.
The product path (the C-ABI library and its Python binding) never imports it
and shares no code, table or constant generator with it.

Everything here is deliberately slow and literal: integer sums in int64/Python
ints, floating point in float64, one library primitive (a vector add, a sum) per
step, and no blocking, fusion or reordering beyond what the paper's definition
or algorithm states.

Modules:
  dedisp  -- Eq. 1 delays, brute-force (direct) and sub-band de-dispersion
             (Sec. 2.3), block statistics, boxcar S/N (Eq. 5), the DM-time
             plane and candidates (Sec. 2.5), running statistics.
  losses  -- the closed-form and semi-analytic S/N-loss expressions: Eqs. 3-4,
             6-8, 12-15 and Appendix A.
  normalise -- per-channel normalisation of each block (Sec. 2.1): unit
             variance or inverse-variance weights, as float32 values.
  plans   -- de-dispersion plans with downsampling (Sec. 2.3).
  cluster -- DBSCAN of the candidates (Sec. 2.5).
"""
from . import dedisp, losses, normalise  # noqa: F401
