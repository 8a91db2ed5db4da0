"""The batched path at its largest beam shapes against the CPU oracle.

The batched workload draws beams of 1024, 2048 or 4096 channels, 32768 to
131072-sample blocks and up to 8192 DM trials over 0-3000 pc cm^-3 in the
MeerKAT-L band. Ring length, the stage-1 row pitch and the stage-2 offsets
all grow with the block length and the DM range, so the largest shapes are
run here: three uneven beams in one batched step (tx_execute_batch, replayed
as a CUDA graph), with the sub-band counts and groups the autotuner chose for
them when its cache has them. On sampled DM trials (the first and last
groups, the DM grid's segment edges, the injected pulses) the series equal
the oracle's two-stage sums bit for bit over two consecutive blocks (uint16
intermediates) and the oracle's emulation of the FP16 form (FP16
intermediates); the DM-time plane equals the oracle's Eq. 5 S/N within
1e-5 relative. Inputs are drawn on the device (seeded) and copied to the host
for the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import dedisp as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5
# (channels, DM trials, block length): the largest of each kind in the batched workload
SHAPES = [(1024, 8192, 131072), (2048, 4096, 65536), (4096, 8192, 32768)]


@pytest.fixture(scope="module")
def tx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    return tx


def _choice(wl):
    """The autotuner's sub-band count and group for this shape (candidate mode, time-major), if cached."""
    from paper_2401_13834_gb300 import autotune
    ch = autotune.lookup(wl, "tf", "cands", "u16")
    return {"nsub": wl.nsub, "group": 0} if ch is None else {"nsub": ch["nsub"], "group": ch["group"]}


def _sample(wl, plan, pulses):
    nd, G = wl.ndm, plan.group
    s = {0, 1, G - 1, G, nd - G - 1, nd - G, nd - 2, nd - 1}
    q = nd // 4
    for j in range(1, 4):
        s |= {j * q - 1, j * q}
    s |= {int(np.argmin(np.abs(wl.dms - p.dm))) for p in pulses}
    return sorted(d for d in s if 0 <= d < nd)


@pytest.fixture(scope="module")
def beams(tx):
    """Workloads, plan choices, pulses and host copies of two blocks plus the carried tail."""
    out = []
    for i, (nc, nd, T) in enumerate(SHAPES):
        wl = synth.batched_beam(nc, nd, T, name=f"c3max{i}")
        ch = _choice(wl)
        wl.nsub = ch["nsub"]
        wl.group = ch["group"]
        probe = tx.Plan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.widths, T, group=wl.group, output="series")
        L = probe.overlap
        # arrival times (at the top of the band) inside the first block's outputs
        pulses = synth.batched_pulses(wl, n=3, seed=40 + i)
        x = synth.device_spectrum(wl, L + 2 * T, pulses, seed=70 + i)
        X = x.cpu().numpy()
        del x
        out.append(dict(wl=wl, L=L, X=X, pulses=pulses, sample=_sample(wl, probe, pulses),
                        op=O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group, wl.widths)))
    torch.cuda.empty_cache()
    return out


def _lay(a, layout):
    return torch.from_numpy(np.ascontiguousarray(a.T if layout == "tf" else a)).cuda()


def _run(tx, beams, nblocks, layout, **kw):
    """All beams as one batched step per block (graph replay); yields per block the outputs."""
    plans = [tx.Plan(b["wl"].freqs_mhz, b["wl"].tsamp_s, b["wl"].dms, b["wl"].nsub, b["wl"].widths,
                     b["wl"].nsamp, group=b["wl"].group, layout=layout, **kw) for b in beams]
    bms = []
    for p, b in zip(plans, beams):
        assert p.overlap == b["L"] == b["op"].overlap
        bm = tx.Beam(p)
        bm.prime(_lay(b["X"][:, :b["L"]], layout))
        bms.append(bm)
    batch = tx.Batch(plans, bms, graph=True)
    ws = batch.alloc_workspace()
    outs = batch.alloc_outs()
    for k in range(nblocks):
        blocks = [_lay(b["X"][:, b["L"] + k * p.nsamp:b["L"] + (k + 1) * p.nsamp], layout)
                  for p, b in zip(plans, beams)]
        batch.execute(blocks, outs, ws)
        batch.wait()
        del blocks
        yield plans, outs
    del ws, outs, batch, bms
    torch.cuda.empty_cache()


def test_batched_series_equal_oracle_u16_two_blocks(tx, beams):
    for k, (plans, outs) in enumerate(_run(tx, beams, 2, "tf", output="series")):
        for p, (o, _), b in zip(plans, outs, beams):
            sample = b["sample"]
            got = tx.series_view(p, o)[sample].cpu().numpy()
            T = p.nsamp
            ref = O.subband_dedisperse(b["X"][:, k * T:k * T + b["L"] + T], b["op"], p.series_len, sample)
            assert np.array_equal(got, ref), (b["wl"].name, k)


def test_batched_series_equal_oracle_f16(tx, beams):
    (plans, outs), = list(_run(tx, beams, 1, "ft", output="series", interm="f16"))
    for p, (o, _), b in zip(plans, outs, beams):
        sample = b["sample"]
        got = tx.series_view(p, o)[sample].cpu().numpy().astype(np.float64)
        L, T = b["L"], p.nsamp
        ref = O.subband_dedisperse_f16(b["X"][:, :L + T], b["op"], p.series_len, slice(L, L + T), sample)
        assert np.array_equal(got, ref), b["wl"].name


def test_batched_plane_equals_oracle_snr(tx, beams):
    (plans, outs), = list(_run(tx, beams, 1, "ft", output="plane"))
    for p, (o, _), b in zip(plans, outs, beams):
        sample = b["sample"]
        snr_d, w_d = tx.plane_view(p, o)
        got_s = snr_d[sample].cpu().numpy().astype(np.float64)
        got_w = w_d[sample].cpu().numpy()
        T = p.nsamp
        D = O.subband_dedisperse(b["X"][:, :b["L"] + T], b["op"], p.series_len, sample)
        _, _, mu, sg = O.block_stats(D, T)
        snr = O.boxcar_snr(D, b["op"].widths, T, mu, sg)             # [dm][w][t]
        best, bw = O.dm_time_plane(snr)
        err = np.abs(got_s - best) / np.maximum(1.0, np.abs(best))
        assert err.max() <= RTOL, (b["wl"].name, err.max())
        # the best width is the oracle's wherever the top two widths are not within the tolerance
        srt = np.sort(snr, axis=1)
        clear = (srt[:, -1, :] - srt[:, -2, :]) > 2 * RTOL * np.maximum(1.0, np.abs(srt[:, -1, :]))
        assert np.array_equal(got_w[clear], bw[clear]), b["wl"].name
        # the injected pulses stand out at their DM trials
        for pl in b["pulses"]:
            d = int(np.argmin(np.abs(b["wl"].dms - pl.dm)))
            assert best[sample.index(d)].max() > 6.0, (b["wl"].name, pl.dm)
