"""The allocation-free entry point against the regular one.

tx_dedisperse_noalloc exists for callers that cannot call cudaMalloc (real-time
loops that must not take the allocator's locks or its implicit
synchronisation, hosts with a device-memory budget owned elsewhere). It keeps
its scratch in a static device array; here two calls in a row, on different
windows, must each give exactly the series that tx_execute gives for the same
window. This file is collected last on purpose: it also runs correctly in a
fresh process on its own.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def _series_via_execute(tx, wl, X):
    """The regular path: a beam primed with the window's tail, then one execute."""
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, output="series")
    L = plan.overlap
    beam = tx.Beam(plan)
    beam.prime(torch.from_numpy(np.ascontiguousarray(X[:, :L])).cuda())
    out = tx.execute(plan, beam, torch.from_numpy(np.ascontiguousarray(X[:, L:])).cuda())
    torch.cuda.synchronize()
    return tx.series_view(plan, out).cpu().numpy()


@pytest.mark.parametrize("mk", [synth.small_workload,
                                lambda: synth.tiny_workload(nchan=64, nsub=8, ndm=37, nsamp=1500, group=5)])
def test_noalloc_matches_execute_on_two_calls(tx, mk):
    wl = mk()
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, output="series")
    L, T = plan.overlap, plan.nsamp
    ld = (L + T + 63) // 64 * 64
    stream = synth.make_spectrum(wl, L + 2 * T, [], seed=21)
    series = torch.empty(plan.ndm * plan.series_len, dtype=torch.int32, device="cuda")
    for b in range(2):  # two calls in a row on different windows
        X = stream[:, b * T:b * T + L + T]
        ref = _series_via_execute(tx, wl, X)
        xd = torch.zeros((plan.nchan, ld), dtype=torch.uint8, device="cuda")
        xd[:, :L + T] = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        series.fill_(-1)
        tx.dedisperse_noalloc(plan, xd, ld, series)
        torch.cuda.synchronize()
        got = series.view(plan.ndm, plan.series_len).cpu().numpy()
        assert np.array_equal(got, ref), f"call {b}"


def test_noalloc_rejects_plans_beyond_its_scratch(tx):
    """A plan whose scratch exceeds the static array is refused (TX_ERR_BUDGET)
    before the library touches the buffers, so small ones do here; the C entry
    point is called directly, past the binding's size checks."""
    import ctypes as C
    wl = synth.meerkat_l_workload()
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, output="series")
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    s = torch.zeros(64, dtype=torch.int32, device="cuda")
    ld = (plan.overlap + plan.nsamp + 63) // 64 * 64
    rc = tx.lib.tx_dedisperse_noalloc(plan.handle, C.c_void_p(x.data_ptr()), ld, C.c_void_p(s.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -7
    buf = C.create_string_buffer(1024)
    tx.lib.tx_last_error(buf, 1024)
    assert "static scratch" in buf.value.decode()
