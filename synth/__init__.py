"""Seeded synthetic filterbank inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the smoke check. It holds
none of the de-dispersion or matched-filter arithmetic: it only describes the
workloads (channel frequencies, DM grids, width ladders, block sizes) and draws
uint8 dynamic spectra with injected pulses.

The pulse injector places each pulse with the physical cold-plasma arrival
time (a continuous value, never rounded to samples) so that a recovered pulse
checks the method rather than re-using its integer delay tables.

Workloads (the paper's benchmark simulates MMGPS-L-like data at 153 us, Sec. 3):

* ``small``      -- 256 channels over 1200-1456 MHz, 64 us, 16384-sample
  blocks, 128 DMs linear over 0-200, 16 sub-bands, widths 1..64, one pulse.
* ``meerkat_l``  -- 4096 channels over 856-1712 MHz, 153.12 us, 65536-sample
  blocks, 4096 DMs over 0-2000 in four segments whose step doubles, 64
  sub-bands, widths 1..256, twenty pulses.
* ``batched``    -- 64 beams of uneven shape on the same band and sampling:
  channels in {1024, 2048, 4096}, blocks in {32768, 65536, 131072} samples,
  {1024, 4096, 8192} DM trials over 0-3000 (four doubling-step segments),
  widths 1..256, a few pulses per beam; drawn with a fixed seed.
* ``serving``    -- 480 beams, every other one MeerKAT-L-like and the rest
  drawn like the batched beams.
* ``small_beams`` -- beams of the small workload's shape, for batches whose
  members are each too small to fill the GPU.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Cold-plasma dispersion constant in s MHz^2 pc^-1 cm^3 (used only to place
# injected pulses on the sky; the method's own tables live elsewhere).
_KDISP_SKY = 4.148808e3


@dataclasses.dataclass
class Workload:
    name: str
    freqs_mhz: np.ndarray          # channel centres, float64 [nchan]
    tsamp_s: float
    dms: np.ndarray                # float64 [ndm], ascending
    nsub: int
    widths: np.ndarray             # int32 [nw], ascending
    nsamp: int                     # new samples per block (T)
    noise_mean: float
    noise_std: float
    group: int = 0                 # 0 = automatic coarse-DM group size

    @property
    def nchan(self) -> int:
        return int(self.freqs_mhz.size)

    @property
    def ndm(self) -> int:
        return int(self.dms.size)


def channel_centres(f_lo: float, f_hi: float, nchan: int) -> np.ndarray:
    """Centres of ``nchan`` equal channels covering [f_lo, f_hi] MHz, ascending."""
    bw = (f_hi - f_lo) / nchan
    return f_lo + (np.arange(nchan, dtype=np.float64) + 0.5) * bw


def geometric_widths(wmax: int, ratio: float = 2.0) -> np.ndarray:
    """Boxcar widths 1, ratio, ratio^2, ... rounded to integers, deduplicated."""
    out = []
    w = 1.0
    while True:
        iw = int(math.floor(w + 0.5))
        if iw > wmax:
            break
        if not out or iw != out[-1]:
            out.append(iw)
        w *= ratio
    return np.asarray(out, dtype=np.int32)


def small_workload() -> Workload:
    return Workload(
        name="small-256ch-128dm",
        freqs_mhz=channel_centres(1200.0, 1456.0, 256),
        tsamp_s=64e-6,
        dms=200.0 * np.arange(128, dtype=np.float64) / 127.0,
        nsub=16,
        widths=geometric_widths(64),
        nsamp=16384,
        noise_mean=128.0,
        noise_std=10.0,
    )


def meerkat_dm_grid(ndm: int = 4096, dm_max: float = 2000.0, nseg: int = 4) -> np.ndarray:
    """DM trials in ``nseg`` equal-count segments whose step doubles each time."""
    per = ndm // nseg
    total = float(2 ** nseg - 1)
    out = []
    for j in range(nseg):
        start = dm_max * (2 ** j - 1) / total
        step = dm_max * (2 ** j) / total / per
        out.append(start + step * np.arange(per, dtype=np.float64))
    return np.concatenate(out)


def meerkat_l_workload() -> Workload:
    return Workload(
        name="meerkat-l-4096ch-4096dm",
        freqs_mhz=channel_centres(856.0, 1712.0, 4096),
        tsamp_s=153.12e-6,
        dms=meerkat_dm_grid(),
        nsub=64,
        widths=geometric_widths(256),
        nsamp=65536,
        noise_mean=128.0,
        noise_std=12.0,
    )


def tiny_workload(nchan=32, nsub=4, ndm=12, nsamp=300, dm_max=60.0, widths=(1, 2, 3, 5, 8),
                  f_lo=1200.0, f_hi=1456.0, tsamp=256e-6, group=0, descending=False) -> Workload:
    f = channel_centres(f_lo, f_hi, nchan)
    if descending:
        f = f[::-1].copy()
    return Workload(
        name=f"tiny-{nchan}ch-{ndm}dm",
        freqs_mhz=f,
        tsamp_s=tsamp,
        dms=np.linspace(0.0, dm_max, ndm),
        nsub=nsub,
        widths=np.asarray(widths, dtype=np.int32),
        nsamp=nsamp,
        noise_mean=128.0,
        noise_std=10.0,
        group=group,
    )


def batched_beam(nchan: int, ndm: int, nsamp: int, dm_max: float = 3000.0, name: str = "beam") -> Workload:
    """One beam of the batched workload: the MeerKAT-L band and sampling time
    with its own channel count, DM-trial count (the MeerKAT-L grid's doubling
    steps up to dm_max) and block length; 64 channels per sub-band."""
    return Workload(
        name=f"{name}-{nchan}ch-{ndm}dm-T{nsamp}",
        freqs_mhz=channel_centres(856.0, 1712.0, nchan),
        tsamp_s=153.12e-6,
        dms=meerkat_dm_grid(ndm, dm_max),
        nsub=nchan // 64,
        widths=geometric_widths(256),
        nsamp=nsamp,
        noise_mean=128.0,
        noise_std=12.0,
    )


def batched_workloads(nbeams: int = 64, seed: int = 3, dm_max: float = 3000.0) -> list:
    """Beams of uneven shape sharing the MeerKAT-L band and sampling time.

    Each beam draws its channel count, block length and DM-trial count
    independently and uniformly from the three values of each; the sub-band
    count defaults to 64 channels per sub-band (an autotuner may change it).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nbeams):
        nchan = int(rng.choice([1024, 2048, 4096]))
        nsamp = int(rng.choice([32768, 65536, 131072]))
        ndm = int(rng.choice([1024, 4096, 8192]))
        out.append(batched_beam(nchan, ndm, nsamp, dm_max, name=f"beam{i}"))
    return out


def small_beams(nbeams: int = 64) -> list:
    """Beams of the small workload's shape (256 channels, 128 DM trials, 16384
    samples): each too small to fill the GPU alone."""
    out = []
    for i in range(nbeams):
        wl = small_workload()
        wl.name = f"beam{i}-" + wl.name
        out.append(wl)
    return out


def serving_workloads(nbeams: int = 480, seed: int = 4) -> list:
    """Beams of a served stream: half MeerKAT-L-like, half drawn like the batched beams."""
    drawn = batched_workloads(nbeams - nbeams // 2, seed=seed)
    out = []
    for i in range(nbeams):
        wl = meerkat_l_workload() if i % 2 == 0 else drawn[i // 2]
        wl.name = f"beam{i}-" + wl.name.split("-", 1)[-1] if i % 2 else f"beam{i}-{wl.name}"
        out.append(wl)
    return out


WORKLOADS = {"small": small_workload, "meerkat_l": meerkat_l_workload}


# ----------------------------------------------------------------------------
# Pulses
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Pulse:
    dm: float          # pc cm^-3
    t_arr: float       # arrival time at the highest channel centre, in samples
    fwhm: float        # samples
    tau_s: float = 0.0  # exponential scattering time, samples (0 = none)
    alpha: float = 0.0  # spectral index, amplitude ~ (f/f_mid)^-alpha
    amp: float = 1.0   # peak amplitude per channel at f_mid (before scattering)


def _emg(x: np.ndarray, w: float, tau: float) -> np.ndarray:
    """exp(-x^2/w^2) convolved with the unit-area causal tail (1/tau) exp(-u/tau).

    Closed form of the exponentially modified Gaussian, written with erfcx
    where its argument is non-negative so that no term overflows.
    """
    from scipy.special import erfc, erfcx
    b = w / (2.0 * tau) - x / w
    pref = w * math.sqrt(math.pi) / (2.0 * tau)
    out = np.empty_like(x)
    pos = b >= 0
    out[pos] = pref * np.exp(-(x[pos] / w) ** 2) * erfcx(b[pos])
    neg = ~pos
    a = b[neg] ** 2 - (x[neg] / w) ** 2
    out[neg] = pref * np.exp(a) * erfc(b[neg])
    return out


def pulse_profile(t: np.ndarray, fwhm: float, tau_s: float, oversample: int = 8) -> np.ndarray:
    """Sample-averaged Gaussian (FWHM ``fwhm``) convolved with a causal exponential.

    ``t`` is the sample-centre offset from the Gaussian peak, in samples. The
    Gaussian is exp(-x^2/w^2) with w = fwhm / (2 sqrt(ln 2)) (Eq. 15 shape);
    with ``tau_s`` = 0 it is the bare Gaussian of peak 1.
    """
    w = fwhm / (2.0 * math.sqrt(math.log(2.0)))
    sub = (np.arange(oversample) + 0.5) / oversample - 0.5
    x = (np.asarray(t, dtype=np.float64)[:, None] + sub[None, :]).ravel()
    if tau_s <= 0:
        y = np.exp(-(x / w) ** 2)
    else:
        y = _emg(x, w, tau_s)
    return y.reshape(-1, oversample).mean(axis=1)


def sky_delay_samples(dm: float, f: np.ndarray, f_top: float, tsamp: float) -> np.ndarray:
    """Continuous cold-plasma arrival offset (samples) of frequency f relative to f_top."""
    return _KDISP_SKY * dm * (1.0 / (f * f) - 1.0 / (f_top * f_top)) / tsamp


def _pulse_half_span(p: Pulse) -> int:
    return int(math.ceil(2.0 * p.fwhm + 14.0 * p.tau_s + 4))


def add_pulse(x: np.ndarray, p: Pulse, freqs: np.ndarray, tsamp: float, f_top=None, f_mid=None) -> None:
    """Add one dispersed pulse, in place, to a float dynamic spectrum x[nchan, nsamp].

    f_top (arrival reference) and f_mid (spectral pivot) default to the band of
    ``freqs``; pass the full band's values when ``freqs`` is a slice of it.
    """
    nsamp = x.shape[1]
    f_top = float(freqs.max()) if f_top is None else f_top
    f_mid = 0.5 * (float(freqs.min()) + f_top) if f_mid is None else f_mid
    centres = p.t_arr + sky_delay_samples(p.dm, freqs, f_top, tsamp)
    spec = (freqs / f_mid) ** (-p.alpha)
    half = _pulse_half_span(p)
    # profile on a 1/16-sample lattice of offsets, interpolated per channel
    lat = np.arange(-half - 1, half + 1 + 1e-9, 1.0 / 16.0)
    prof = pulse_profile(lat, p.fwhm, p.tau_s)
    for c in range(freqs.size):
        t0 = max(int(math.floor(centres[c])) - half, 0)
        t1 = min(int(math.ceil(centres[c])) + half + 1, nsamp)
        if t1 <= t0:
            continue
        rel = np.arange(t0, t1, dtype=np.float64) - centres[c]
        x[c, t0:t1] += (p.amp * spec[c] * np.interp(rel, lat, prof, left=0.0, right=0.0)).astype(x.dtype)


def pulse_points(p: Pulse, freqs: np.ndarray, tsamp: float, nsamp: int, f_top=None, f_mid=None):
    """The (channel, sample, value) points ``add_pulse`` adds, as flat arrays.

    Same window per channel (max(floor(c) - half, 0) .. min(ceil(c) + half + 1,
    nsamp), c the continuous arrival) and the same interpolated values, for
    adders that work on other array types.
    """
    f_top = float(freqs.max()) if f_top is None else f_top
    f_mid = 0.5 * (float(freqs.min()) + f_top) if f_mid is None else f_mid
    centres = p.t_arr + sky_delay_samples(p.dm, freqs, f_top, tsamp)
    spec = (freqs / f_mid) ** (-p.alpha)
    half = _pulse_half_span(p)
    lat = np.arange(-half - 1, half + 1 + 1e-9, 1.0 / 16.0)
    prof = pulse_profile(lat, p.fwhm, p.tau_s)
    lo = np.floor(centres).astype(np.int64) - half
    hi = np.ceil(centres).astype(np.int64) + half + 1
    tt = lo[:, None] + np.arange(2 * half + 2, dtype=np.int64)[None, :]
    keep = (tt < hi[:, None]) & (tt >= 0) & (tt < nsamp)
    rel = tt - centres[:, None]
    vals = (p.amp * spec[:, None] * np.interp(rel, lat, prof, left=0.0, right=0.0)).astype(np.float32)
    chan = np.broadcast_to(np.arange(freqs.size, dtype=np.int64)[:, None], tt.shape)
    return chan[keep], tt[keep], vals[keep]


def device_spectrum(wl: Workload, nsamp_total: int, pulses=(), seed: int = 0, device="cuda", rfi: Rfi = None):
    """uint8 [nchan, nsamp_total] torch tensor drawn on a CUDA device.

    clip(round(N(mean, std) + pulses), 0, 255) like ``make_spectrum``, with the
    noise from torch's counter-based generator on the device (seeded; the same
    seed, shape and device type give the same values) so that volumes of many
    GB need no host work. Pulses are added as ``pulse_points`` gives them.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.randn((wl.nchan, nsamp_total), generator=g, device=device, dtype=torch.float32)
    x.mul_(float(wl.noise_std)).add_(float(wl.noise_mean))
    for p in pulses:
        c, t, v = pulse_points(p, wl.freqs_mhz, wl.tsamp_s, nsamp_total)
        if c.size:
            x.index_put_((torch.from_numpy(c).to(device), torch.from_numpy(t).to(device)),
                         torch.from_numpy(v).to(device), accumulate=True)
    if rfi is not None:
        add_rfi(x, rfi)
    return x.round_().clamp_(0.0, 255.0).to(torch.uint8)


def batched_pulses(wl: Workload, n: int = 4, seed: int = 0) -> list:
    """Pulses of one batched beam: DM U(0, DM_max), FWHM logU(0.3, 20) ms, S/N U(8, 50), flat spectrum, no scattering."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        fwhm = math.exp(rng.uniform(math.log(0.3e-3), math.log(20e-3))) / wl.tsamp_s
        p = Pulse(dm=float(rng.uniform(0.0, float(wl.dms.max()))), t_arr=float(rng.uniform(0.05, 0.95) * wl.nsamp),
                  fwhm=fwhm)
        p.amp = amplitude_for_snr(float(rng.uniform(8.0, 50.0)), wl, p)
        out.append(p)
    return out


@dataclasses.dataclass
class Rfi:
    """Interference for the precision workload: narrow-band sinusoids in some
    channels (amplitude in noise sigmas, period and phase per channel) and
    zero-DM broadband bursts (every channel at once, no dispersion delay)."""
    channels: np.ndarray       # int [n]
    amp: float                 # counts
    period: np.ndarray         # samples [n]
    phase: np.ndarray          # radians [n]
    bursts: list               # (start sample, width, amplitude in counts)


def make_rfi(wl: Workload, nsamp_total: int, seed: int = 0, frac: float = 0.05, amp_sigma: float = 50.0,
             nbursts: int = 4, burst_sigma: float = 3.0) -> Rfi:
    """5% of channels carrying 50-sigma sinusoids of random period (4..4096 samples) and phase,
    and a few zero-DM bursts of burst_sigma sigmas lasting 8..256 samples."""
    rng = np.random.default_rng(seed)
    n = max(1, int(round(frac * wl.nchan)))
    ch = np.sort(rng.choice(wl.nchan, size=n, replace=False))
    period = np.exp(rng.uniform(math.log(4.0), math.log(4096.0), size=n))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n)
    bursts = []
    for _ in range(nbursts):
        w = int(rng.integers(8, 257))
        bursts.append((int(rng.integers(0, max(1, nsamp_total - w))), w, burst_sigma * wl.noise_std))
    return Rfi(channels=ch, amp=amp_sigma * wl.noise_std, period=period, phase=phase, bursts=bursts)


def add_rfi(x, rfi: Rfi) -> None:
    """Adds the interference, in place, to a float dynamic spectrum [nchan, nsamp]
    (a numpy array or a torch tensor)."""
    nsamp = x.shape[1]
    if isinstance(x, np.ndarray):
        t = np.arange(nsamp, dtype=np.float64)
        for c, P, ph in zip(rfi.channels, rfi.period, rfi.phase):
            x[c] += (rfi.amp * np.sin(2.0 * math.pi * t / P + ph)).astype(x.dtype)
    else:
        import torch
        t = torch.arange(nsamp, device=x.device, dtype=torch.float64)
        for c, P, ph in zip(rfi.channels, rfi.period, rfi.phase):
            x[int(c)] += (rfi.amp * torch.sin(2.0 * math.pi * t / float(P) + float(ph))).to(x.dtype)
    for t0, w, a in rfi.bursts:
        x[:, t0:t0 + w] += a


def quantise(values: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(values), 0, 255).astype(np.uint8)


def make_spectrum(wl: Workload, nsamp_total: int, pulses=(), seed: int = 0,
                  dtype_noise=np.float32, rfi: Rfi = None) -> np.ndarray:
    """uint8 [nchan, nsamp_total] = clip(round(N(mean, std) + pulses + rfi), 0, 255)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((wl.nchan, nsamp_total), dtype=dtype_noise)
    x *= dtype_noise(wl.noise_std)
    x += dtype_noise(wl.noise_mean)
    for p in pulses:
        add_pulse(x, p, wl.freqs_mhz, wl.tsamp_s)
    if rfi is not None:
        add_rfi(x, rfi)
    return quantise(x)


def make_stream(wl: Workload, nsamp_total: int, pulses=(), seed: int = 0, chunk: int = 256) -> np.ndarray:
    """Like ``make_spectrum`` but drawn in channel chunks to bound host memory.

    Chunk i uses the generator seeded with (seed, i), so the result depends
    only on (seed, chunk), not on the machine.
    """
    out = np.empty((wl.nchan, nsamp_total), dtype=np.uint8)
    f32 = np.float32
    for c0 in range(0, wl.nchan, chunk):
        c1 = min(c0 + chunk, wl.nchan)
        rng = np.random.default_rng([seed, c0 // chunk])
        x = rng.standard_normal((c1 - c0, nsamp_total), dtype=f32)
        x *= f32(wl.noise_std)
        x += f32(wl.noise_mean)
        for p in pulses:
            add_pulse(x, p, wl.freqs_mhz[c0:c1], wl.tsamp_s, f_top=float(wl.freqs_mhz.max()),
                      f_mid=0.5 * (float(wl.freqs_mhz.min()) + float(wl.freqs_mhz.max())))
        out[c0:c1] = quantise(x)
    return out


def amplitude_for_snr(snr_g: float, wl: Workload, p: Pulse) -> float:
    """Per-channel amplitude giving a noise-free de-dispersed S/N_G (Eq. 14) of snr_g.

    Uses the ideal (continuous-delay) de-dispersed profile nchan * a * prof(t),
    with the spectral weights, against noise std sqrt(nchan) * noise_std.
    """
    f_top = float(wl.freqs_mhz.max())
    f_mid = 0.5 * (float(wl.freqs_mhz.min()) + f_top)
    spec_sum = float(((wl.freqs_mhz / f_mid) ** (-p.alpha)).sum())
    half = _pulse_half_span(p)
    t = np.arange(-half, half + 1, dtype=np.float64)
    prof = pulse_profile(t, p.fwhm, p.tau_s) * spec_sum
    sigma_d = math.sqrt(wl.nchan) * wl.noise_std
    return snr_g * sigma_d / math.sqrt(float((prof ** 2).sum()))


def small_pulses(wl: Workload) -> list:
    """The small workload's single pulse: DM 100, FWHM 1 ms, S/N 20, flat spectrum."""
    p = Pulse(dm=100.0, t_arr=0.37 * wl.nsamp, fwhm=1e-3 / wl.tsamp_s)
    p.amp = amplitude_for_snr(20.0, wl, p)
    return [p]


def meerkat_pulses(wl: Workload, n: int = 20, seed: int = 1) -> list:
    """Random pulses: DM U(0,2000), FWHM logU(0.3,20) ms, tau U(0,10)*FWHM, alpha U(-3,3), S/N U(8,50)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        fwhm = math.exp(rng.uniform(math.log(0.3e-3), math.log(20e-3))) / wl.tsamp_s
        p = Pulse(
            dm=float(rng.uniform(0.0, float(wl.dms.max()))),
            t_arr=float(rng.uniform(0.05, 0.95) * wl.nsamp),
            fwhm=fwhm,
            tau_s=float(rng.uniform(0.0, 10.0) * fwhm),
            alpha=float(rng.uniform(-3.0, 3.0)),
        )
        p.amp = amplitude_for_snr(float(rng.uniform(8.0, 50.0)), wl, p)
        out.append(p)
    return out
