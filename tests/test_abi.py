"""The C-ABI library on the CPU: it loads, exports what include/*.h declares,
and its host-side plan (Eq. 1 tables, grouping, overlap) equals the oracle's.

No compute call is made here; these tests need no GPU.
"""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import synth
from oracle import dedisp as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tx():
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tx_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(tx):
    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", tx.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared - exported
    assert not missing, missing
    for n in declared:
        assert hasattr(tx.lib, n)


def _plan(tx, wl, **kw):
    return tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp, group=wl.group, **kw)


@pytest.mark.parametrize("mk", [
    lambda: synth.small_workload(),
    lambda: synth.meerkat_l_workload(),
    lambda: synth.tiny_workload(descending=True),
    lambda: synth.tiny_workload(nchan=48, nsub=48, ndm=9, group=4),
    lambda: synth.tiny_workload(nchan=40, nsub=1, ndm=7, group=1),
    lambda: synth.tiny_workload(nchan=64, nsub=8, ndm=13, group=5),
])
def test_plan_tables_equal_oracle(tx, mk):
    wl = mk()
    p = _plan(tx, wl)
    o = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group, wl.widths)
    t = p.tables()
    assert p.group == o.group and p.ncoarse == o.nk
    assert np.array_equal(t["coarse_of_fine"], o.coarse_of_fine)
    assert np.array_equal(t["coarse_dm"], o.coarse_dm)
    assert np.array_equal(t["d1"], o.d1)
    assert np.array_equal(t["d2"], o.d2)
    assert p.overlap == o.overlap and p.max_delay == o.max_delay
    assert p.series_len == wl.nsamp + o.wmax - 1


def test_meerkat_plan_sizes(tx):
    wl = synth.meerkat_l_workload()
    p = _plan(tx, wl, output="plane")
    assert p.group == 16 and p.ncoarse == 256
    assert p.overlap == p.max_delay + 255 and 55000 < p.max_delay < 55500
    assert p.out_bytes == 4096 * 65536 * 5
    assert p.block_bytes == 4096 * 65536
    off, pitch, base = p.stage1_layout()
    assert off == 0 and pitch >= 65536 + 255 and np.all(base % 16 == 0)


def test_geometric_widths_match_ladder(tx):
    for r, w in [(2.0, 256), (1.5, 100), (1.1, 40), (3.0, 1)]:
        assert np.array_equal(tx.geometric_widths(r, w), synth.geometric_widths(w, r))


@pytest.mark.parametrize("kw,code", [
    (dict(nsub=7), -2),
    (dict(widths=[4, 2]), -1),
    (dict(dms=[5.0, 1.0]), -1),
    (dict(tsamp=0.0), -1),
    (dict(nsamp=0), -1),
    (dict(output="cands", max_cands=0), -1),
    (dict(tile_q1=48), -1),
    (dict(tile_split2=3), -1),
    (dict(group=8, tile_split2=8), -1),        # 8 DMs x 8 warps > 32 warps
])
def test_invalid_plans_rejected(tx, kw, code):
    wl = synth.tiny_workload(nchan=32, nsub=4)
    args = dict(freqs=wl.freqs_mhz, tsamp=wl.tsamp_s, dms=wl.dms, nsub=4, widths=wl.widths, nsamp=wl.nsamp)
    extra = {}
    for k, v in kw.items():
        if k in args:
            args[k] = v
        else:
            extra[k] = v
    with pytest.raises(tx.TxError) as e:
        tx.Plan(args["freqs"], args["tsamp"], args["dms"], args["nsub"], args["widths"], args["nsamp"], **extra)
    assert e.value.code == code


def test_too_many_channels_per_subband_unsupported(tx):
    wl = synth.tiny_workload(nchan=520, nsub=2)
    with pytest.raises(tx.TxError) as e:
        _plan(tx, wl)
    assert e.value.code == -8


def test_tile_knobs_reported(tx):
    wl = synth.tiny_workload(nchan=64, nsub=4, ndm=40)
    auto = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 4, wl.widths, wl.nsamp, group=4)
    # groups of up to 16 DMs run the pipelined stage 2: 4, 2 or 1 consumer warps per DM, at most 28 in all
    assert auto.tile_q1 == 256 and auto.tile_split2 == 4
    p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 4, wl.widths, wl.nsamp, group=4, tile_q1=64, tile_split2=1)
    assert p.tile_q1 == 64 and p.tile_split2 == 4
    for g, sp in ((7, 4), (8, 2), (14, 2), (16, 1)):
        assert tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 4, wl.widths, wl.nsamp, group=g).tile_split2 == sp
    # larger groups: the other kernel, whose warps per DM the description sets
    big = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 4, wl.widths, wl.nsamp, group=32, tile_split2=1)
    assert big.tile_split2 == 1
    # the tile shapes change neither the tables nor the overlap
    assert p.overlap == auto.overlap
    for k in ("d1", "d2", "coarse_of_fine", "coarse_dm"):
        assert np.array_equal(p.tables()[k], auto.tables()[k])


def test_boxcar_unit_choice(tx):
    """The boxcar unit grows to 4 or 2 sub-tiles of 2048 outputs only while at
    least 4864 (DM, unit) pairs remain; an explicit length is taken as given."""
    f = synth.channel_centres(1200.0, 1456.0, 32)
    def plan(ndm, T, **kw):
        return tx.Plan(f, 256e-6, np.linspace(0.0, 50.0, ndm), 4, (1, 2, 4), T, **kw)
    assert plan(24, 3000).tile_box == 2048
    assert plan(2432, 16384).tile_box == 8192        # 2432 DMs x 2 units
    assert plan(1216, 16384).tile_box == 4096        # 1216 x 4
    assert plan(1215, 16384).tile_box == 2048        # 1215 x 4 < 4864
    assert plan(24, 3000, tile_box=8192).tile_box == 8192
    for bad in (1000, 2047, 16384, -2048):
        with pytest.raises(tx.TxError) as e:
            plan(24, 3000, tile_box=bad)
        assert e.value.code == -1


def test_tile_q1_that_does_not_fit_is_unsupported(tx):
    wl = synth.tiny_workload(nchan=257, nsub=1, ndm=8)
    with pytest.raises(tx.TxError) as e:
        tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 1, wl.widths, wl.nsamp, tile_q1=256)
    assert e.value.code == -8


@pytest.mark.parametrize("mk", [synth.small_workload, synth.meerkat_l_workload])
def test_delay_table_equals_oracle(tx, mk):
    """The clustering axis: Eq. 1 across the band, identical to the last bit."""
    from oracle import cluster as CL
    wl = mk()
    plan = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, wl.nsamp)
    ref = CL.delay_ms(wl.dms, float(wl.freqs_mhz.min()), float(wl.freqs_mhz.max()))
    assert np.array_equal(plan.delay_table(), ref)


@pytest.mark.parametrize("m", [1, 16, 64, 128, 257])
def test_stage1_tile_fits_shared_memory_for_every_subband_width(tx, m):
    """The automatic stage-1 tile is the largest whose staged words, raw
    windows, offset tables, row bases, item descriptors and delay rows fit the
    227 KB of shared memory (MeerKAT-L's 64 channels per sub-band keep the
    largest tile; 257 channels, the most the 16-bit sums allow, still fit)."""
    wl = synth.tiny_workload(nchan=m * 2, nsub=2, ndm=16)
    p = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 2, wl.widths, wl.nsamp)
    assert p.tile_q1 in (32, 64, 128, 256)
    if m <= 64:
        assert p.tile_q1 == 256
    if p.tile_q1 < 256:   # the next larger tile would not have fitted
        with pytest.raises(tx.TxError) as e:
            tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 2, wl.widths, wl.nsamp, tile_q1=2 * p.tile_q1)
        assert e.value.code == -8


def test_noalloc_refuses_misaligned_buffers_before_any_launch(tx):
    """tx_dedisperse_noalloc checks its pointers before it touches the GPU: a
    series buffer that is 4- but not 8-byte aligned (the kernel stores two
    outputs at a time) and an unaligned window are refused with
    TX_ERR_INVALID_ARG. The addresses are never dereferenced."""
    import ctypes as C
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=6, nsamp=300)
    p = _plan(tx, wl, output="series")
    ld = (p.overlap + p.nsamp + 63) // 64 * 64
    st = C.c_void_p(0)
    rc = tx.lib.tx_dedisperse_noalloc(p.handle, C.c_void_p(0x10000), ld, C.c_void_p(0x20004), st)
    assert rc == -1
    rc = tx.lib.tx_dedisperse_noalloc(p.handle, C.c_void_p(0x10008), ld, C.c_void_p(0x20000), st)
    assert rc == -1
    rc = tx.lib.tx_dedisperse_noalloc(p.handle, C.c_void_p(0x10000), ld + 1, C.c_void_p(0x20000), st)
    assert rc == -1


def test_noalloc_wrapper_checks_tensors(tx):
    """The binding checks what the C side cannot see (dtype, contiguity, size,
    device) and raises before calling into the library."""
    torch = pytest.importorskip("torch")
    wl = synth.tiny_workload(nchan=32, nsub=4, ndm=6, nsamp=300)
    p = _plan(tx, wl, output="series")
    ld = (p.overlap + p.nsamp + 63) // 64 * 64
    x = torch.zeros(p.nchan * ld, dtype=torch.uint8)
    ser = torch.zeros(p.ndm * p.series_len, dtype=torch.int32)
    cases = [
        (x.to(torch.int16), ser, "must be torch.uint8"),
        (x, ser.to(torch.int64), "must be torch.int32"),
        (x.view(p.nchan, ld).t(), ser, "contiguous"),
        (x[: p.nchan * ld - 1], ser, "needs"),
        (x, ser[:-1], "needs"),
        (x, ser, "CUDA tensor"),
    ]
    for xx, ss, msg in cases:
        with pytest.raises(tx.TxError) as e:
            tx.dedisperse_noalloc(p, xx, ld, ss)
        assert e.value.code == -1 and msg in str(e.value), (msg, str(e.value))


def test_wait_polls_setting_is_range_checked(tx):
    """tx_set_wait_polls takes 0 .. 2^22 and returns the previous limit."""
    import ctypes as C
    old = C.c_int64()
    assert tx.lib.tx_set_wait_polls(-1, C.byref(old)) == -1
    assert tx.lib.tx_set_wait_polls((1 << 22) + 1, C.byref(old)) == -1
    prev = tx.set_wait_polls(1000)
    assert prev == 1 << 22
    assert tx.set_wait_polls(prev) == 1000
