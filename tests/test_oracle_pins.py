"""Pins for the CPU oracle: closed forms, brute force, invariants, paper values.

None of these tests needs a GPU. Each one checks the oracle against something
other than itself: exact rational arithmetic, pure-Python brute force on tiny
inputs, textbook/library routines, physical injections, or numbers the paper
prints (tests/golden/paper_values.json).
"""
import json
import math
import os
from decimal import ROUND_HALF_UP, Decimal
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, optimize
from scipy.special import erf

import synth
from oracle import dedisp as O
from oracle import losses as LS

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
KF = Fraction(4.148808e3)


# ---------------------------------------------------------------------------
# exact reference delays (rational arithmetic on the exact binary inputs)
# ---------------------------------------------------------------------------
def _round_half_away(q: Fraction) -> int:
    n = math.floor(abs(q) + Fraction(1, 2))
    return n if q >= 0 else -n


def exact_delay(dm, f, fr, tsamp):
    q = KF * Fraction(dm) * (1 / Fraction(f) ** 2 - 1 / Fraction(fr) ** 2) / Fraction(tsamp)
    return q


def near_tie(q: Fraction, eps=1e-9) -> bool:
    fr = abs(q) - math.floor(abs(q))
    return abs(float(fr) - 0.5) < eps


# ---------------------------------------------------------------------------
# Eq. 1 and rounding
# ---------------------------------------------------------------------------
def test_rnd_matches_decimal_half_up():
    rng = np.random.default_rng(3)
    xs = list(rng.uniform(-1e6, 1e6, 2000)) + [0.5, 1.5, 2.5, -0.5, -2.5, 0.49999999999999994,
                                                  -0.49999999999999994, 1e15 + 0.5, 0.0, -0.0, 7.0]
    for x in xs:
        ref = int(Decimal(x).quantize(Decimal(1), rounding=ROUND_HALF_UP))
        assert O.rnd(x) == ref, x
    arr = np.array(xs)
    assert list(O.rnd_array(arr)) == [O.rnd(x) for x in xs]


def test_delay_two_channel_toy():
    g = GOLD["delay_toy"]
    tau = O.delay_seconds(g["dm"], g["f_lo_mhz"], g["f_hi_mhz"])
    assert tau == pytest.approx(g["delay_s"], rel=1e-7)
    assert int(O.delay_samples(g["dm"], g["f_lo_mhz"], g["f_hi_mhz"], g["tsamp_s"])) == g["delay_samples"]
    # the reference channel itself has no delay, and delays grow with DM and 1/f^2
    assert int(O.delay_samples(5.0, 2000.0, 2000.0, 1e-3)) == 0
    assert O.delay_seconds(2.0, 1000.0, 2000.0) == pytest.approx(2 * g["delay_s"], rel=1e-12)


def test_delay_tables_match_exact_rationals():
    rng = np.random.default_rng(11)
    freqs = np.sort(rng.uniform(300.0, 2000.0, 40))
    fr = float(freqs.max())
    for dm in rng.uniform(0.0, 3000.0, 25):
        got = O.delay_samples(float(dm), freqs, fr, 64e-6)
        for f, g in zip(freqs, got):
            q = exact_delay(float(dm), float(f), fr, 64e-6)
            if near_tie(q):
                continue
            assert int(g) == _round_half_away(q)


# ---------------------------------------------------------------------------
# Direct (brute-force) de-dispersion
# ---------------------------------------------------------------------------
def _tiny_inputs(wl, seed=0):
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group, wl.widths)
    rng = np.random.default_rng(seed)
    # room for both schemes: sub-band rounding can reach a sample past direct, or fall short
    l_dir = int(O.direct_delays(wl.freqs_mhz, wl.tsamp_s, wl.dms).max()) + plan.wmax - 1
    X = rng.integers(0, 256, size=(wl.nchan, wl.nsamp + max(plan.overlap, l_dir)), dtype=np.uint8)
    return plan, X


def _brute_direct(X, freqs, tsamp, dms, nout):
    fr = max(freqs)
    out = []
    for dm in dms:
        dl = []
        for f in freqs:
            q = exact_delay(float(dm), float(f), float(fr), tsamp)
            assert not near_tie(q)
            dl.append(_round_half_away(q))
        row = []
        for t in range(nout):
            acc = 0
            for c in range(len(freqs)):
                acc += int(X[c][t + dl[c]])
            row.append(acc)
        out.append(row)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("descending", [False, True])
def test_direct_matches_brute_force(descending):
    wl = synth.tiny_workload(nchan=16, nsub=4, ndm=6, nsamp=64, descending=descending)
    plan, X = _tiny_inputs(wl, seed=1)
    nout = wl.nsamp + plan.wmax - 1
    D = O.direct_dedisperse(X, wl.freqs_mhz, wl.tsamp_s, wl.dms, nout)
    ref = _brute_direct(X, list(wl.freqs_mhz), wl.tsamp_s, list(wl.dms), nout)
    assert np.array_equal(D, ref)


def test_direct_impulse_track_sums_to_nchan():
    wl = synth.tiny_workload(nchan=32, ndm=8, nsamp=128)
    fr = float(wl.freqs_mhz.max())
    L = 400
    for d, dm in enumerate(wl.dms):
        X = np.zeros((wl.nchan, wl.nsamp + L), dtype=np.uint8)
        t0 = 37
        for c, f in enumerate(wl.freqs_mhz):
            X[c, t0 + _round_half_away(exact_delay(float(dm), float(f), fr, wl.tsamp_s))] = 1
        D = O.direct_dedisperse(X, wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsamp)
        assert D[d, t0] == wl.nchan
        assert D[d].sum() == wl.nchan  # every impulse lands exactly once in range


def test_direct_constant_and_linearity():
    wl = synth.tiny_workload()
    plan, X = _tiny_inputs(wl, seed=2)
    _, Y = _tiny_inputs(wl, seed=3)
    nout = wl.nsamp + plan.wmax - 1
    f = lambda A: O.direct_dedisperse(A, wl.freqs_mhz, wl.tsamp_s, wl.dms, nout)
    C = np.full_like(X, 7)
    assert np.all(f(C) == 7 * wl.nchan)
    Z = X.astype(np.int64) + Y.astype(np.int64)
    assert np.array_equal(f(Z), f(X) + f(Y))


# ---------------------------------------------------------------------------
# Sub-band plan and algorithm
# ---------------------------------------------------------------------------
def test_coarse_grouping_and_midpoints():
    wl = synth.tiny_workload(ndm=12)
    p = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 4, 5, wl.widths)
    assert p.nk == 3
    assert list(p.coarse_of_fine) == [0] * 5 + [1] * 5 + [2] * 2
    assert p.coarse_dm[2] == (wl.dms[10] + wl.dms[11]) / 2
    assert p.coarse_dm[0] == (wl.dms[0] + wl.dms[4]) / 2


@pytest.mark.parametrize("mk", [synth.small_workload, synth.meerkat_l_workload])
def test_auto_group_rule(mk):
    wl = mk()
    G = O.auto_group(wl.freqs_mhz, wl.tsamp_s, wl.nsub, wl.ndm)
    assert G == {"small-256ch-128dm": 8, "meerkat-l-4096ch-4096dm": 16}[wl.name]
    # the rule's inequality, from independent arithmetic on sorted sub-bands
    f = np.sort(wl.freqs_mhz)
    m = wl.nchan // wl.nsub
    smear = lambda lo, hi: 4.148808e3 * (lo ** -2 - hi ** -2) / wl.tsamp_s
    s_full = smear(f[0], f[-1])
    s_sub = max(smear(f[i * m], f[(i + 1) * m - 1]) for i in range(wl.nsub))
    assert (G - 1) * s_sub <= s_full * (1 + 1e-12)
    assert (2 * G - 1) * s_sub > s_full


def _brute_subband(X, wl, G, nout):
    """Two-stage sub-band sums with exact-rational delays and Python loops."""
    freqs = [float(f) for f in wl.freqs_mhz]
    nchan, nsub = len(freqs), wl.nsub
    m = nchan // nsub
    fr = max(freqs)
    frs = [max(freqs[s * m:(s + 1) * m]) for s in range(nsub)]
    out = []
    for d, dm in enumerate(wl.dms):
        k = d // G
        a, b = float(wl.dms[k * G]), float(wl.dms[min((k + 1) * G, len(wl.dms)) - 1])
        dmk = (Fraction(a) + Fraction(b)) / 2
        row = [0] * nout
        for s in range(nsub):
            q2 = KF * Fraction(float(dm)) * (1 / Fraction(frs[s]) ** 2 - 1 / Fraction(fr) ** 2) / Fraction(wl.tsamp_s)
            assert not near_tie(q2)
            d2 = _round_half_away(q2)
            for c in range(s * m, (s + 1) * m):
                q1 = KF * dmk * (1 / Fraction(freqs[c]) ** 2 - 1 / Fraction(frs[s]) ** 2) / Fraction(wl.tsamp_s)
                assert not near_tie(q1)
                d1 = _round_half_away(q1)
                for t in range(nout):
                    row[t] += int(X[c][t + d1 + d2])
        out.append(row)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("group,descending", [(3, False), (0, False), (4, True)])
def test_subband_matches_brute_force(group, descending):
    wl = synth.tiny_workload(nchan=16, nsub=4, ndm=7, nsamp=48, group=group, descending=descending)
    plan, X = _tiny_inputs(wl, seed=4)
    nout = wl.nsamp + plan.wmax - 1
    D = O.subband_dedisperse(X, plan, nout)
    ref = _brute_subband(X, wl, plan.group, nout)
    assert np.array_equal(D, ref)


def test_subband_equals_direct_one_channel_per_subband():
    wl = synth.tiny_workload(nchan=32, nsub=32, ndm=10, nsamp=200, group=4)
    plan, X = _tiny_inputs(wl, seed=5)
    assert np.all(plan.d1 == 0)
    nout = wl.nsamp + plan.wmax - 1
    assert np.array_equal(O.subband_dedisperse(X, plan, nout),
                          O.direct_dedisperse(X, wl.freqs_mhz, wl.tsamp_s, wl.dms, nout))


def test_subband_equals_direct_single_subband_unit_group():
    wl = synth.tiny_workload(nchan=24, nsub=1, ndm=9, nsamp=150, group=1)
    plan, X = _tiny_inputs(wl, seed=6)
    assert np.all(plan.d2 == 0)
    nout = wl.nsamp + plan.wmax - 1
    assert np.array_equal(O.subband_dedisperse(X, plan, nout),
                          O.direct_dedisperse(X, wl.freqs_mhz, wl.tsamp_s, wl.dms, nout))


def test_subband_impulse_track_and_overlap_bound():
    wl = synth.tiny_workload(nchan=32, nsub=8, ndm=16, nsamp=100, group=4)
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, wl.group, wl.widths)
    nout = wl.nsamp + plan.wmax - 1
    for d in (0, 5, 15):
        k = plan.coarse_of_fine[d]
        X = np.zeros((wl.nchan, wl.nsamp + plan.overlap), dtype=np.uint8)
        t0 = nout - 1  # the last output sample reaches furthest into the buffer
        for c in range(wl.nchan):
            X[c, t0 + plan.d1[k, c] + plan.d2[d, c // plan.m]] = 1
        D = O.subband_dedisperse(X, plan, nout, [d])
        assert D[0, t0] == wl.nchan
    # the overlap is exactly what the furthest access needs
    far = max(int(plan.d1[plan.coarse_of_fine[d], c] + plan.d2[d, c // plan.m])
              for d in range(plan.ndm) for c in range(plan.nchan))
    assert plan.overlap == far + plan.wmax - 1


def test_subband_loss_small_versus_direct_on_pulse():
    """The sub-band approximation keeps >= 95% of the direct S/N on a real pulse."""
    wl = synth.small_workload()
    wl.nsamp = 4096
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, 0, wl.widths)
    p = synth.Pulse(dm=100.0, t_arr=1500.0, fwhm=1e-3 / wl.tsamp_s)
    p.amp = synth.amplitude_for_snr(20.0, wl, p)
    X = synth.make_spectrum(wl, wl.nsamp + plan.overlap, [p], seed=0)
    d = int(np.argmin(np.abs(wl.dms - 100.0)))
    nout = wl.nsamp + plan.wmax - 1
    sb = O.subband_dedisperse(X, plan, nout, [d])
    dr = O.direct_dedisperse(X, wl.freqs_mhz, wl.tsamp_s, wl.dms[d:d + 1], nout)
    best = []
    for D in (sb, dr):
        _, _, mu, sg = O.block_stats(D, wl.nsamp)
        best.append(O.boxcar_snr(D, wl.widths, wl.nsamp, mu, sg).max())
    assert best[0] >= 0.95 * best[1]
    assert best[1] > 15.0


def test_injected_pulse_recovered_at_dm_and_time():
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=40, nsamp=2048, dm_max=100.0, tsamp=128e-6,
                             widths=(1, 2, 4, 8, 16, 32))
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, 0, wl.widths)
    p = synth.Pulse(dm=57.3, t_arr=900.0, fwhm=8.0)
    p.amp = synth.amplitude_for_snr(30.0, wl, p)
    X = synth.make_spectrum(wl, wl.nsamp + plan.overlap, [p], seed=7)
    D = O.subband_dedisperse(X, plan, wl.nsamp + plan.wmax - 1)
    _, _, mu, sg = O.block_stats(D, wl.nsamp)
    snr = O.boxcar_snr(D, wl.widths, wl.nsamp, mu, sg)
    d, w, t = np.unravel_index(np.argmax(snr), snr.shape)
    step = wl.dms[1] - wl.dms[0]
    assert abs(wl.dms[d] - p.dm) <= 1.5 * step
    # with a DM error the band-averaged arrival moves by the mean residual delay
    resid = synth.sky_delay_samples(p.dm - wl.dms[d], wl.freqs_mhz, wl.freqs_mhz.max(), wl.tsamp_s)
    expect = p.t_arr + float(resid.mean())
    centre = t + (wl.widths[w] - 1) / 2.0
    assert abs(centre - expect) <= 2.0 + wl.widths[w] / 4.0
    assert snr[d, w, t] > 20.0


def test_stream_split_invariance():
    wl = synth.tiny_workload(nchan=16, nsub=4, ndm=8, nsamp=64)
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, 0, wl.widths)
    rng = np.random.default_rng(8)
    T, nb = wl.nsamp, 3
    stream = rng.integers(0, 256, size=(wl.nchan, plan.overlap + nb * T), dtype=np.uint8)
    blocks = O.stream_series(stream, plan, T, nb)
    whole = O.subband_dedisperse(stream, plan, nb * T + plan.wmax - 1)
    for b in range(nb):
        assert np.array_equal(blocks[b], whole[:, b * T:b * T + T + plan.wmax - 1])


# ---------------------------------------------------------------------------
# Boxcar matched filter (Eq. 5), statistics, plane and candidates
# ---------------------------------------------------------------------------
def test_window_sums_match_convolution():
    rng = np.random.default_rng(9)
    row = rng.integers(-1000, 1000, 700)
    T = 500
    for W in (1, 2, 3, 7, 64, 200):
        ref = np.convolve(row, np.ones(W, dtype=np.int64), mode="valid")[:T]
        assert np.array_equal(O.window_sums(row, W, T), ref)


def test_block_stats_match_numpy():
    rng = np.random.default_rng(10)
    D = rng.integers(30000, 40000, size=(5, 1000))
    S1, S2, mu, sg = O.block_stats(D, 900)
    for i in range(5):
        assert S1[i] == int(D[i, :900].sum())
        assert S2[i] == int((D[i, :900].astype(object) ** 2).sum())
        assert mu[i] == pytest.approx(float(np.mean(D[i, :900])), rel=1e-15)
        assert sg[i] == pytest.approx(float(np.std(D[i, :900])), rel=1e-12)
    _, _, mu, sg = O.block_stats(np.full((1, 10), 5), 10)
    assert sg[0] == 0.0
    snr = O.boxcar_snr(np.full((1, 20), 5), [1, 4], 10, mu, sg)
    assert np.all(snr == 0.0)


def test_width_mismatch_exact_for_top_hat():
    """Eq. 8 holds exactly for a noise-free top-hat aligned with the boxcar start."""
    T = 400
    for Wt in (4, 16, 25):
        row = np.zeros(T + 100, dtype=np.int64)
        row[100:100 + Wt] = 10
        widths = [1, 2, 3, 4, 8, 16, 25, 32, 50]
        snr = O.boxcar_snr(row[None, :], widths, T, [0.0], [1.0])[0]
        opt = snr[widths.index(Wt)].max()
        for i, W in enumerate(widths):
            got = snr[i, 100] / opt
            assert got == pytest.approx(LS.width_mismatch_ratio(Wt, W - Wt), rel=1e-12)


def test_false_alarm_rate_on_gaussian_noise():
    """Eq. 6: on white Gaussian noise the count of S/N >= gamma is binomial(N, P_FA)."""
    rng = np.random.default_rng(12)
    N = 2_000_000
    D = rng.standard_normal((1, N + 1))
    _, _, mu, sg = O.block_stats(D, N)
    snr = O.boxcar_snr(D, [1], N, mu, sg)[0, 0]
    for gamma in (2.5, 3.0, 3.5):
        p = float(LS.p_false_alarm(gamma))
        n = int((snr >= gamma).sum())
        assert abs(n - N * p) <= 5.0 * math.sqrt(N * p * (1 - p))


def test_plane_ties_and_candidates():
    snr = np.zeros((2, 3, 4))
    snr[0, :, 1] = [5.0, 7.0, 7.0]       # tie -> smaller width index 1
    snr[1, 2, 3] = 9.0
    snr[1, 0, 0] = 6.0
    best, bw = O.dm_time_plane(snr)
    assert bw[0, 1] == 1 and best[0, 1] == 7.0
    c = O.candidates(best, bw, 6.0)
    assert sorted((int(r["d"]), int(r["t"]), int(r["w"])) for r in c) == [(0, 1, 1), (1, 0, 0), (1, 3, 2)]


def test_running_stats_update():
    st = O.running_stats(None, 10.0, 4.0, 0.25)
    assert st == (10.0, 4.0)
    st = O.running_stats(st, 14.0, 8.0, 0.25)
    assert st == (11.0, 5.0)


# ---------------------------------------------------------------------------
# S/N-loss expressions
# ---------------------------------------------------------------------------
def test_zeta_coefficient_matches_paper():
    g = GOLD["zeta_coefficient"]
    assert LS.zeta_coefficient() == pytest.approx(g["value"], rel=g["rel_tol"])


def test_amplitude_ratio_from_linearised_integral():
    """Eq. 3 equals the peak of the band-averaged Gaussian (Appendix A's model), by quadrature."""
    assert float(LS.amplitude_ratio(0.0)) == GOLD["amplitude_ratio_small_zeta"]["value"]
    for z in (0.3, 1.0, 2.5, 6.0):
        # average over a uniformly spread delay tau in [-z, z] (units of w) of exp(-tau^2), t = 0
        num, _ = integrate.quad(lambda u: math.exp(-u * u), -z, z)
        assert float(LS.amplitude_ratio(z)) == pytest.approx(num / (2 * z), rel=1e-10)
        assert float(LS.dedispersed_profile(np.array([0.0]), z)[0]) == pytest.approx(num / (2 * z), rel=1e-10)


def test_appendix_profile_by_quadrature():
    for z in (0.5, 2.0):
        for t in (-1.7, 0.0, 0.4, 3.0):
            num, _ = integrate.quad(lambda u: math.exp(-(t - u) ** 2), -z, z)
            assert float(LS.dedispersed_profile(np.array([t]), z)[0]) == pytest.approx(num / (2 * z), rel=1e-9)
            # and the boxcar integral of Appendix A
        for wm in (0.5, 2.0, 7.0):
            num, _ = integrate.quad(lambda t: float(LS.dedispersed_profile(np.array([t]), z)[0]), -wm / 2, wm / 2)
            assert LS.boxcar_response(wm, z) == pytest.approx(num / math.sqrt(wm), rel=1e-9)


def test_dm_mismatch_snr_curve_properties():
    assert LS.dm_mismatch_snr_ratio(0.0) == pytest.approx(1.0, abs=1e-12)
    prev = 1.0
    for z in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0):
        r = LS.dm_mismatch_snr_ratio(z)
        assert r < prev
        prev = r
        # Sec. 2.3: the S/N falls more slowly than the amplitude
        assert r > float(LS.amplitude_ratio(z))
    g = GOLD["dm_mismatch_wm_over_2zeta"]
    for z in (g["zeta_min"], 20.0, 40.0):
        wm, _ = LS.optimal_width(z)
        assert wm / (2 * z) == pytest.approx(g["value"], abs=g["abs_tol"])
    # zeta = 0: the textbook Gaussian/boxcar optimum, erf(u)/sqrt(u) maximal near u = 1
    res = optimize.minimize_scalar(lambda u: -erf(u) / math.sqrt(u), bounds=(0.1, 3), method="bounded")
    wm0, _ = LS.optimal_width(0.0)
    assert wm0 / 2 == pytest.approx(res.x, rel=1e-4)


def test_dm_mismatch_end_to_end_against_appendix_a():
    """A noise-free dispersed Gaussian de-dispersed at DM + dDM loses S/N as Appendix A predicts."""
    nchan, f_lo, f_hi, tsamp = 64, 1400.0, 1416.0, 10e-6
    freqs = synth.channel_centres(f_lo, f_hi, nchan)
    fwhm = 100.0  # samples = 1 ms
    dm0 = 100.0
    p = synth.Pulse(dm=dm0, t_arr=2500.0, fwhm=fwhm, amp=1.0)
    nsamp = 9000
    x = np.zeros((nchan, nsamp), dtype=np.float64)
    synth.add_pulse(x, p, freqs, tsamp)
    bw = nchan * (f_hi - f_lo) / nchan
    nu = 0.5 * (f_lo + f_hi) / 1e3
    ref = None
    for z in (0.0, 0.5, 1.0, 2.0, 4.0):
        ddm = z / LS.zeta(1.0, bw, fwhm * tsamp * 1e3, nu)
        D = O.direct_dedisperse(x, freqs, tsamp, [dm0 + ddm], 6000)[0]
        C = np.concatenate([[0.0], np.cumsum(D)])
        best = max(float((C[W:] - C[:-W]).max()) / math.sqrt(W) for W in range(1, 1500))
        if ref is None:
            ref = best
            continue
        assert best / ref == pytest.approx(LS.dm_mismatch_snr_ratio(z), rel=0.03), z


def test_pulse_shape_loss_matches_paper():
    r0 = LS.pulse_shape_ratio(0.0)
    # textbook Gaussian vs best boxcar: (pi/2)^(1/4) max_u erf(u)/sqrt(u)
    res = optimize.minimize_scalar(lambda u: -erf(u) / math.sqrt(u), bounds=(0.1, 3), method="bounded")
    assert r0 == pytest.approx((math.pi / 2) ** 0.25 * (-res.fun), rel=2e-3)
    g = GOLD["pulse_shape_loss_tau10"]
    assert 1.0 - LS.pulse_shape_ratio(g["tau_over_w"]) == pytest.approx(g["loss"], abs=g["abs_tol"])


def test_spectral_index_loss():
    assert LS.spectral_index_ratio(0.0, 2.0) == pytest.approx(1.0, abs=1e-12)
    f = np.linspace(1.0, 2.0, 200001)
    for a in (-3.0, -1.0, 0.5, 1.0, 2.0, 3.0):
        assert LS.spectral_index_ratio(a, 2.0) == pytest.approx(
            LS.spectral_index_ratio_discrete(a, f), rel=1e-4)
    g = GOLD["spectral_loss_index2_eta2"]
    assert 1.0 - LS.spectral_index_ratio(-g["alpha_text"], g["eta"]) == pytest.approx(g["loss"], abs=g["abs_tol"])
    # wider bands lose more (Sec. 4.1)
    assert LS.spectral_index_ratio(2.0, 5.0) < LS.spectral_index_ratio(2.0, 2.0)


def test_detection_probability_symmetry():
    assert float(LS.p_detect(5.0, 5.0)) == pytest.approx(0.5)
    assert float(LS.p_false_alarm(0.0)) == pytest.approx(0.5)
    assert float(LS.p_detect(5.0, 8.0)) > float(LS.p_detect(5.0, 5.0))


def test_detection_probabilities_by_value():
    """Eqs. 6-7 are the Gaussian tail and the Gaussian CDF of the excess S/N
    over gamma: pinned to the textbook 95% quantile of the standard normal
    (1.6448536269514722), to P(Z > 6) and P(Z > 3), and to the normal CDF
    computed by integrating the density with quadrature (not through erfc)."""
    z95 = 1.6448536269514722
    for gamma in (0.0, 5.0, 7.0):
        assert float(LS.p_detect(gamma, gamma + z95)) == pytest.approx(0.95, abs=1e-12)
        assert float(LS.p_detect(gamma, gamma - z95)) == pytest.approx(0.05, abs=1e-12)
    assert float(LS.p_false_alarm(z95)) == pytest.approx(0.05, abs=1e-12)
    assert float(LS.p_false_alarm(6.0)) == pytest.approx(9.865876450376946e-10, rel=1e-9)
    assert float(LS.p_false_alarm(3.0)) == pytest.approx(1.3498980316300946e-3, rel=1e-12)

    def phi(x):  # standard normal CDF by quadrature of the density
        v, _ = integrate.quad(lambda u: math.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi), -40.0, x,
                              epsabs=1e-14, epsrel=1e-12, limit=200)
        return v

    for gamma, snr in ((7.0, 5.0), (7.0, 8.3), (5.0, 10.0), (6.0, 6.5)):
        assert float(LS.p_detect(gamma, snr)) == pytest.approx(phi(snr - gamma), rel=1e-9, abs=1e-13)


def test_scattered_pulse_against_numerical_convolution():
    """Eq. 15 for tau > 0: the closed form (both of its branches) equals the
    convolution of exp(-u^2/w^2) with the causal (1/tau) exp(-t/tau) done by
    quadrature, point by point; its area is that of the Gaussian, w sqrt(pi)
    (the kernel has unit area), whatever tau; and tau -> 0 gives the Gaussian."""
    w = 1.3
    for tau in (0.05, 0.4, 1.0, 3.0, 13.0):
        t = np.array([-3.0, -1.0, -0.2, 0.0, 0.3, 1.0, 2.5, 6.0, 15.0, 40.0]) * w
        got = LS.scattered_pulse(t, w, tau)
        for ti, gi in zip(t, got):
            ref, _ = integrate.quad(lambda u: math.exp(-(u / w) ** 2) * math.exp(-(ti - u) / tau) / tau,
                                    -12.0 * w, ti, epsabs=1e-15, epsrel=1e-11, limit=400)
            assert gi == pytest.approx(ref, rel=1e-8, abs=1e-14), (tau, ti, gi, ref)
        # area over a grid wide enough for the tail
        tt = np.linspace(-8.0 * w, 8.0 * w + 60.0 * tau, 400001)
        area = integrate.trapezoid(LS.scattered_pulse(tt, w, tau), tt)
        assert area == pytest.approx(w * math.sqrt(math.pi), rel=2e-6), tau
    t = np.linspace(-3.0, 3.0, 61)
    assert np.allclose(LS.scattered_pulse(t, 1.0, 1e-6), np.exp(-t * t), atol=2e-6)


# ---------------------------------------------------------------------------
# Half-precision storage of the stage-1 sums (the FP16 form)
# ---------------------------------------------------------------------------
def _one_subband_plan(nchan, T):
    """One sub-band, DM 0 only, width 1: every delay is 0, so D[t] = P[t] = sum_c X[c][t]."""
    f = synth.channel_centres(1400.0, 1401.0, nchan)
    return O.SubbandPlan(f, 1e-3, np.array([0.0]), 1, 1, (1,))


def test_f16_form_exact_while_offsets_keep_sums_small():
    """With 8 channels per sub-band every |P - o_s| <= 8 * 255 = 2040 < 2048,
    and every integer up to 2048 is an FP16 value: the FP16 form is exact."""
    wl = synth.tiny_workload(nchan=64, nsub=8, ndm=20, nsamp=900, dm_max=80.0)
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, wl.nsub, 0, wl.widths)
    X = np.random.default_rng(3).integers(0, 256, size=(64, plan.overlap + 900)).astype(np.uint8)
    nout = 900 + plan.wmax - 1
    exact = O.subband_dedisperse(X, plan, nout)
    f16 = O.subband_dedisperse_f16(X, plan, nout, slice(plan.overlap, plan.overlap + 900))
    assert np.array_equal(f16, exact.astype(np.float64))


def test_f16_form_rounds_to_nearest_even():
    """Sums placed at 2047, 2049, 3001, 4098 and 4102 on a zero background.
    FP16 holds the integers up to 2048, every second one in [2048, 4096) and
    every fourth in [4096, 8192); ties go to the even significand:
    2049 -> 2048, 3001 -> 3000 (3000 = 1.4648... x 2^11 with significand 476,
    even), 4098 -> 4096, 4102 -> 4104 (significand 2). The block's channel
    means round to 0 (at most 1275 counts over 4096 samples), so o_s = 0."""
    T, m = 4096, 20
    plan = _one_subband_plan(m, T)
    X = np.zeros((m, T), dtype=np.uint8)
    targets = {100: 2047, 700: 2049, 1300: 3001, 2500: 4098, 3900: 4102}
    for t, v in targets.items():
        left = v
        for c in range(m):
            x = min(255, left)
            X[c, t] = x
            left -= x
        assert left == 0
    assert np.array_equal(O.half_offsets(X, plan, slice(0, T)), [0])
    D = O.subband_dedisperse_f16(X, plan, T, slice(0, T))[0]
    expect = np.zeros(T)
    expect[[100, 700, 1300, 2500, 3900]] = [2047, 2048, 3000, 4096, 4104]
    assert np.array_equal(D, expect)


def test_f16_form_saturates():
    """257 channels of 255 sum to 65535, above the largest FP16 value 65504."""
    T, m = 4096, 257
    plan = _one_subband_plan(m, T)
    X = np.zeros((m, T), dtype=np.uint8)
    X[:, 10] = 255
    D = O.subband_dedisperse_f16(X, plan, T, slice(0, T))[0]
    assert D[10] == 65504.0 and D[11] == 0.0


def test_half_offsets_definition():
    """o_s = sum over the sub-band's channels of their block means rounded half up."""
    wl = synth.tiny_workload(nchan=8, nsub=2, ndm=4, nsamp=10)
    plan = O.SubbandPlan(wl.freqs_mhz, wl.tsamp_s, wl.dms, 2, 0, wl.widths)
    X = np.zeros((8, 30), dtype=np.uint8)
    X[0, 20:30] = 5           # mean 5
    X[1, 20:25] = 1           # mean 0.5 -> 1 (half up)
    X[2, 20:24] = 1           # mean 0.4 -> 0
    X[5, 0:20] = 200          # outside the block: ignored
    X[6, 20:30] = 255         # mean 255
    assert list(O.half_offsets(X, plan, slice(20, 30))) == [6, 255]
