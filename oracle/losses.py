"""Oracle: S/N-loss expressions of Secs. 2.3, 2.4, 4.1, 4.2 and Appendix A.

TEST INFRASTRUCTURE ONLY (see the package docstring).

All in float64. Where the paper gives a closed form it is written out; where it
computes numerically (Appendix A's optimal width, the pulse-shape loss of
Sec. 4.2) the integrals are done in closed form where one exists and the
maximisation by golden-section search.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc

# Eq. 1 constant, s MHz^2 pc^-1 cm^3.
K_DM = 4.148808e3


# ----------------------------------------------------------------------------
# Eqs. 3-4: DM mismatch, amplitude
# ----------------------------------------------------------------------------
def zeta_coefficient() -> float:
    """The constant of Eq. 4 from Eq. 1 and Appendix A, unrounded.

    Appendix A linearises the delay across the band: tau(f) ~ -2 K dDM (f - f_c)/f_c^3,
    so the smear across the bandwidth is dtau = 2 K dDM dnu / f_c^3, and the
    de-dispersed profile it gives is that of Appendix A with zeta = dtau / (2 w),
    w the 1/e half-width of exp(-t^2/w^2). With the FWHM W = 2 sqrt(ln 2) w, and
    dnu in MHz, nu in GHz, W in ms: zeta = K * 1e3 * 2 sqrt(ln 2) / 1e9 * ...
    """
    return K_DM * 1e3 * 2.0 * math.sqrt(math.log(2.0)) / 1e9


def zeta(ddm, bw_mhz, w_ms, nu_ghz) -> float:
    """Eq. 4: zeta = 6.91e-3 dDM dnu_MHz / (W_ms nu_GHz^3), unrounded constant."""
    return zeta_coefficient() * ddm * bw_mhz / (w_ms * nu_ghz ** 3)


def amplitude_ratio(z):
    """Eq. 3: S(dDM)/S = (sqrt(pi)/2) zeta^-1 erf(zeta), -> 1 as zeta -> 0."""
    z = np.asarray(z, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = 0.5 * math.sqrt(math.pi) * erf(z) / z
    return np.where(z == 0.0, 1.0, r)


# ----------------------------------------------------------------------------
# Appendix A: S/N vs DM mismatch
# ----------------------------------------------------------------------------
def _G(x):
    """Antiderivative of erf: x erf(x) + exp(-x^2)/sqrt(pi)."""
    return x * erf(x) + np.exp(-x * x) / math.sqrt(math.pi)


def dedispersed_profile(t, z):
    """Appendix A: s(t) = (sqrt(pi)/4) zeta^-1 [erf(zeta - t) + erf(zeta + t)], t in units of w."""
    t = np.asarray(t, dtype=np.float64)
    if z == 0.0:
        return np.exp(-t * t)
    return 0.25 * math.sqrt(math.pi) / z * (erf(z - t) + erf(z + t))


def boxcar_response(wm, z):
    """Appendix A: F(zeta, w_m) = w_m^-1/2 int_{-w_m/2}^{w_m/2} s(t) dt (w = 1).

    The integral in closed form: int_{-a}^{a} [erf(z - t) + erf(z + t)] dt
    = 2 [G(z + a) - G(z - a)], with G the antiderivative of erf.
    """
    a = 0.5 * wm
    if z == 0.0:
        integral = math.sqrt(math.pi) * erf(a)
    else:
        integral = 0.25 * math.sqrt(math.pi) / z * 2.0 * (_G(z + a) - _G(z - a))
    return float(integral) / math.sqrt(wm)


def _golden_max(f, lo, hi, tol=1e-10, it=300):
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c = b - g * (b - a)
    d = a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(it):
        if abs(b - a) < tol * (1.0 + abs(a) + abs(b)):
            break
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    x = 0.5 * (a + b)
    return x, f(x)


def optimal_width(z):
    """Appendix A: the boxcar width w_m (units of w) that maximises F(zeta, w_m)."""
    hi = 4.0 * z + 8.0
    return _golden_max(lambda wm: boxcar_response(wm, z), 1e-6, hi)


def dm_mismatch_snr_ratio(z) -> float:
    """Appendix A: measured over optimal S/N, max_wm F(zeta, wm) / max_wm F(0, wm)."""
    _, fz = optimal_width(z)
    _, f0 = optimal_width(0.0)
    return fz / f0


# ----------------------------------------------------------------------------
# Eqs. 6-8: detection statistics and width mismatch
# ----------------------------------------------------------------------------
def p_false_alarm(gamma):
    """Eq. 6: P_FA = erfc(gamma / sqrt 2) / 2."""
    return 0.5 * erfc(np.asarray(gamma, dtype=np.float64) / math.sqrt(2.0))


def p_detect(gamma, snr):
    """Eq. 7: P_D = erfc((gamma - S/N) / sqrt 2) / 2."""
    return 0.5 * erfc((np.asarray(gamma, dtype=np.float64) - snr) / math.sqrt(2.0))


def width_mismatch_ratio(W, dW):
    """Eq. 8: sqrt((W + dW)/W) for dW <= 0, sqrt(W/(W + dW)) for dW > 0."""
    if dW <= 0:
        return math.sqrt((W + dW) / W)
    return math.sqrt(W / (W + dW))


# ----------------------------------------------------------------------------
# Sec. 4.1, Eqs. 9-13: spectral-index mismatch
# ----------------------------------------------------------------------------
def spectral_index_ratio(alpha, eta):
    """Eq. 12: S/N(flat weights) / S/N(optimal weights) for a power law of index alpha.

    ((eta^(1-alpha) - 1)/(1-alpha)) / sqrt((eta - 1)(eta^(1-2 alpha) - 1)/(1 - 2 alpha)),
    with the limits log(eta) where an exponent vanishes.
    """
    def integ(p):  # int_1^eta x^(p-1) dx
        return math.log(eta) if abs(p) < 1e-12 else (eta ** p - 1.0) / p
    return integ(1.0 - alpha) / math.sqrt((eta - 1.0) * integ(1.0 - 2.0 * alpha))


def spectral_index_ratio_discrete(alpha, freqs):
    """Eqs. 9-11 directly on channels: equal weights vs weights a_j = f_j^-alpha.

    S/N with weights v_j is sum v_j a_j / sqrt(sum v_j^2) (white noise, equal
    sigma); optimal v = a. Ratio of the equal-weight to the optimal value.
    """
    f = np.asarray(freqs, dtype=np.float64)
    a = (f / f.min()) ** (-alpha)
    flat = a.sum() / math.sqrt(f.size)
    opt = math.sqrt((a * a).sum())
    return flat / opt


# ----------------------------------------------------------------------------
# Sec. 4.2, Eqs. 14-15: pulse-shape mismatch
# ----------------------------------------------------------------------------
def scattered_pulse(t, w, tau_s):
    """Eq. 15: exp(-t^2/w^2) convolved with (1/tau_s) exp(-t/tau_s) (t >= 0), closed form."""
    t = np.asarray(t, dtype=np.float64)
    if tau_s == 0.0:
        return np.exp(-(t / w) ** 2)
    from scipy.special import erfcx
    b = w / (2.0 * tau_s) - t / w
    pref = w * math.sqrt(math.pi) / (2.0 * tau_s)
    out = np.empty_like(t)
    pos = b >= 0
    out[pos] = pref * np.exp(-(t[pos] / w) ** 2) * erfcx(b[pos])
    neg = ~pos
    out[neg] = pref * np.exp(b[neg] ** 2 - (t[neg] / w) ** 2) * erfc(b[neg])
    return out


def pulse_shape_ratio(tau_over_w, dt=None):
    """Sec. 4.2: best boxcar S/N (Eq. 5) over the matched S/N_G (Eq. 14) for Eq. 15's pulse.

    On a fine grid: S/N_G = sqrt(sum s^2) (noise-free, unit sigma); the boxcar
    value is max over start and width of sum_window s / sqrt(N_box).
    """
    w = 1.0
    tau = float(tau_over_w) * w
    if dt is None:
        dt = min(0.02, 0.02 * max(tau, 1.0))
    t = np.arange(-6.0 * w, 6.0 * w + 20.0 * tau, dt)
    s = scattered_pulse(t, w, tau)
    matched = math.sqrt(float((s * s).sum()))
    C = np.concatenate([[0.0], np.cumsum(s)])
    best = 0.0
    n = s.size
    # widths on a geometric grid fine enough that the maximum is flat
    nb = 1
    widths = set()
    while nb < n:
        widths.add(nb)
        nb = max(nb + 1, int(nb * 1.01))
    for nbox in sorted(widths):
        sums = C[nbox:] - C[:-nbox]
        best = max(best, float(sums.max()) / math.sqrt(nbox))
    return best / matched
