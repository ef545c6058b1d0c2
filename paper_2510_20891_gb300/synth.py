"""Seeded synthetic inputs for the semi-coherent track statistic.

This module only draws inputs: strain time series (noise plus an injected
single harmonic), training frequency tracks for the basis, and candidate
track coefficients.  It holds none of the statistic's arithmetic (no SFT,
no normalisation, no track->bin mapping, no gather), so the FP64 oracle and
the CUDA path can both be fed from it without sharing any method code.

The workloads follow the paper's setting (Sec. II.E): a single harmonic in
stationary Gaussian noise with a known PSD, sampled every few seconds for up
to one year.  The paper's own EMRI trajectories (Eq. 3, computed with an
external package) are not available, so the frequency families below are
analytic stand-ins: quadratic chirps and the power law f0 (1 - t/tau)^-p.

Every generator takes a numpy ``Generator`` (PCG64, platform independent).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

YEAR_S = 365.0 * 86400.0          # 31,536,000 s: the one-year workloads
JULIAN_YEAR_S = 365.25 * 86400.0  # the paper's year (Sec. II.B segment counts)


# --------------------------------------------------------------------------
# Power spectral densities (one-sided, Hz^-1)
# --------------------------------------------------------------------------
def psd_white(f, sigma: float = 1.0, dt: float = 1.0):
    """One-sided PSD of white noise with per-sample std sigma: S_n = 2 sigma^2 dt."""
    f = np.asarray(f, dtype=np.float64)
    return np.full(f.shape, 2.0 * sigma * sigma * dt)


def psd_oneyear(f):
    """S_n(f) = 1e-40 [1 + (2e-3/f)^4] [1 + (f/2.5e-2)^2]; infinite at f = 0."""
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore"):
        s = 1e-40 * (1.0 + (2e-3 / f) ** 4) * (1.0 + (f / 2.5e-2) ** 2)
    return np.where(f > 0, s, np.inf)


def psd_oneyear_hp(f):
    """psd_oneyear held at its 1e-4 Hz value below 1e-4 Hz (data high-passed at 1e-4 Hz): the
    f^-4 wall would otherwise leak through the window's sidelobes into the lowest SFT bins."""
    f = np.asarray(f, dtype=np.float64)
    return np.where(f > 0, psd_oneyear(np.maximum(f, 1e-4)), np.inf)


def psd_bins(psd_fn, n_bin: int, T_sft: float):
    """PSD sampled at the SFT bin frequencies k / T_sft, k = 0..n_bin-1."""
    return psd_fn(np.arange(n_bin, dtype=np.float64) / T_sft)


# --------------------------------------------------------------------------
# Noise
# --------------------------------------------------------------------------
def white_noise(n: int, sigma: float, rng: np.random.Generator):
    return sigma * rng.standard_normal(n)


def coloured_noise(n: int, dt: float, psd_fn, rng: np.random.Generator):
    """Stationary Gaussian noise with one-sided PSD ``psd_fn`` (frequency-domain synthesis).

    The real FFT bins are complex Gaussians with E|X_k|^2 = S_n(f_k) n / (2 dt)
    (the Nyquist bin, for even n, is real with the same second moment); the DC
    bin is zero.  For white noise this reproduces per-sample variance sigma^2.
    """
    nf = n // 2 + 1
    f = np.arange(nf, dtype=np.float64) / (n * dt)
    s = psd_fn(f)
    s = np.where(np.isfinite(s), s, 0.0)
    var = s * n / (2.0 * dt)
    X = np.sqrt(var / 2.0) * (rng.standard_normal(nf) + 1j * rng.standard_normal(nf))
    X[0] = 0.0
    if n % 2 == 0:
        X[-1] = np.sqrt(var[-1]) * rng.standard_normal()
    return np.fft.irfft(X, n=n)


# --------------------------------------------------------------------------
# Injected single harmonic
# --------------------------------------------------------------------------
def chirp_signal(n: int, dt: float, f0: float, fdot: float, amp: float, phi0: float = 0.0):
    """h(t) = amp cos(2 pi (f0 t + fdot t^2 / 2) + phi0): instantaneous frequency f0 + fdot t."""
    t = np.arange(n, dtype=np.float64) * dt
    return amp * np.cos(2.0 * np.pi * (f0 * t + 0.5 * fdot * t * t) + phi0)


def powerlaw_freq(t, f0: float, tau: float, p: float):
    """f(t) = f0 (1 - t/tau)^(-p), the one-year family's frequency evolution."""
    t = np.asarray(t, dtype=np.float64)
    return f0 * (1.0 - t / tau) ** (-p)


def powerlaw_phase(t, f0: float, tau: float, p: float):
    """Phi(t) = 2 pi int_0^t f = 2 pi f0 tau / (1-p) [1 - (1 - t/tau)^(1-p)]."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 * np.pi * f0 * tau / (1.0 - p) * (1.0 - (1.0 - t / tau) ** (1.0 - p))


def powerlaw_signal(n: int, dt: float, f0: float, tau: float, p: float, a0: float, phi0: float = 0.0):
    """h(t) = a(t) cos(Phi(t) + phi0) with slowly varying a(t) = a0 (f(t)/f0)^(2/3)."""
    t = np.arange(n, dtype=np.float64) * dt
    f = powerlaw_freq(t, f0, tau, p)
    a = a0 * (f / f0) ** (2.0 / 3.0)
    return a * np.cos(powerlaw_phase(t, f0, tau, p) + phi0)


def snr_of_amplitude(a_t, f_t, dt: float, psd_fn):
    """SNR^2 = int a(t)^2 / S_n(f(t)) dt for a slowly varying harmonic (rectangle rule)."""
    return math.sqrt(float(np.sum(a_t * a_t / psd_fn(f_t)) * dt))


def powerlaw_amplitude_for_snr(n: int, dt: float, f0: float, tau: float, p: float, snr: float, psd_fn):
    t = np.arange(n, dtype=np.float64) * dt
    f = powerlaw_freq(t, f0, tau, p)
    shape = (f / f0) ** (2.0 / 3.0)
    return snr / snr_of_amplitude(shape, f, dt, psd_fn)


# --------------------------------------------------------------------------
# Frequency-track families for the basis and candidate coefficients
# --------------------------------------------------------------------------
def segment_midpoints(n_seg: int, T_sft: float):
    """t_alpha = (alpha + 1/2) T_sft, relative to the first sample."""
    return (np.arange(n_seg, dtype=np.float64) + 0.5) * T_sft


def quad_chirp_tracks(M: int, t_alpha, rng: np.random.Generator,
                      f0=(4e-3, 6e-3), fdot=(0.0, 2e-9), fddot=(0.0, 1e-16)):
    """f(t) = f0 + fdot t + fddot t^2 / 2 with uniform draws; rows are tracks [M, n_seg]."""
    a = rng.uniform(*f0, size=M)
    b = rng.uniform(*fdot, size=M)
    c = rng.uniform(*fddot, size=M)
    t = np.asarray(t_alpha, dtype=np.float64)[None, :]
    return a[:, None] + b[:, None] * t + 0.5 * c[:, None] * t * t


def powerlaw_params(M: int, rng: np.random.Generator,
                    f0=(2e-3, 8e-3), tau_yr=(1.5, 5.0), p=(0.25, 0.4)):
    return (rng.uniform(*f0, size=M), rng.uniform(*tau_yr, size=M) * YEAR_S, rng.uniform(*p, size=M))


def powerlaw_tracks(M: int, t_alpha, rng: np.random.Generator, **kw):
    f0, tau, p = powerlaw_params(M, rng, **kw)
    t = np.asarray(t_alpha, dtype=np.float64)[None, :]
    return f0[:, None] * (1.0 - t / tau[:, None]) ** (-p[:, None])


def uniform_coeffs(N: int, cmin, cmax, rng: np.random.Generator):
    """Candidate coefficients drawn uniformly inside the box [cmin, cmax] (one row per track)."""
    cmin = np.asarray(cmin, dtype=np.float64)
    cmax = np.asarray(cmax, dtype=np.float64)
    return cmin[None, :] + (cmax - cmin)[None, :] * rng.random((N, cmin.size))


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    dt: float
    n_samples: int
    T_sft: float
    K: int
    n_tracks: int
    m: int
    n_train: int
    family: str          # "quad" or "powerlaw"
    psd: str             # "white" or "oneyear"
    seed: int = 0
    tau_yr: tuple = (1.5, 5.0)  # power-law family: tau range (years); tau must exceed the duration

    @property
    def L(self):
        return int(round(self.T_sft / self.dt))

    @property
    def n_seg(self):
        return self.n_samples // self.L

    @property
    def n_bin(self):
        return self.L // 2 + 1

    def psd_fn(self):
        if self.psd == "white":
            return lambda f: psd_white(f, 1.0, self.dt)
        if self.psd == "oneyear_hp":
            return psd_oneyear_hp
        return psd_oneyear


WORKLOADS = {
    # 2^18 s of unit white noise, 64 x 4096-s segments, K = 3 quadratic-chirp basis, nearest bin.
    "tiny_white_2p18": Workload("tiny_white_2p18", 1.0, 1 << 18, 4096.0, 3, 10_000, 0, 1000, "quad", "white"),
    # one year at 5 s, 365 daily segments x 8641 bins, K = 6 power-law basis, +-1-bin neighbours.
    "oneyear_daily_fp32": Workload("oneyear_daily_fp32", 5.0, 6_307_200, 86400.0, 6, 10_000_000, 1, 5000,
                                   "powerlaw", "oneyear"),
    # finer resolution: 1577 x 20000-s segments x 20001 bins (sampled at 0.5 s so segments are full).
    # the plunge-time search of Sec. II.D: one Julian year at 5 s in 631 SFTs of 5e4 s, a K = 6 basis of
    # tracks that plunge just after the year, the chunks of 0.1 yr + 12 SFTs, +-1-bin neighbours.
    "oneyear_5e4_631": Workload("oneyear_5e4_631", 5.0, 631 * 10_000, 50_000.0, 6, 48 * 512, 1, 5000,
                                "powerlaw", "oneyear_hp", tau_yr=(1.0005, 1.05)),
    "oneyear_fine_1577x20001": Workload("oneyear_fine_1577x20001", 0.5, 1577 * 40000, 20000.0, 6,
                                        100_000_000, 1, 5000, "powerlaw", "oneyear"),
}


def make_strain(w: Workload, rng: np.random.Generator, snr: float | None = None, inject: bool = True):
    """Noise plus one injected harmonic for a named workload; returns (strain, injection dict)."""
    n, dt = w.n_samples, w.dt
    if w.psd == "white":
        x = white_noise(n, 1.0, rng)
        inj = dict(kind="chirp", f0=5e-3, fdot=1e-9, amp=0.05)
        if inject:
            x = x + chirp_signal(n, dt, inj["f0"], inj["fdot"], inj["amp"])
        return x, inj
    psd_fn = w.psd_fn()
    x = coloured_noise(n, dt, psd_fn, rng)
    f0, tau, p = powerlaw_params(1, rng, tau_yr=w.tau_yr)
    inj = dict(kind="powerlaw", f0=float(f0[0]), tau=float(tau[0]), p=float(p[0]), snr=30.0 if snr is None else snr)
    if inject:
        a0 = powerlaw_amplitude_for_snr(n, dt, inj["f0"], inj["tau"], inj["p"], inj["snr"], psd_fn)
        inj["a0"] = a0
        x = x + powerlaw_signal(n, dt, inj["f0"], inj["tau"], inj["p"], a0)
    return x, inj


def make_training_tracks(w: Workload, rng: np.random.Generator, M: int | None = None):
    t = segment_midpoints(w.n_seg, w.T_sft)
    M = w.n_train if M is None else M
    if w.family == "quad":
        return quad_chirp_tracks(M, t, rng)
    return powerlaw_tracks(M, t, rng, tau_yr=w.tau_yr)


# --------------------------------------------------------------------------
# Batched datasets and served datasets
# --------------------------------------------------------------------------
def batched_workloads(n: int = 64, seed0: int = 1):
    """Independent datasets of the one-year family for one batched launch: durations
    U[0.25, 2] yr at dt = 5 s, T_sft drawn from {1e4, 2e4, 5e4, 1e5} s, the one-year PSD,
    one power-law harmonic injected at SNR U[15, 40], K drawn from {4, 6, 8}, 10^U[4,6]
    candidate tracks, +-1-bin neighbours.  The family's tau is drawn from
    U[max(1.5, 1.25 D), max(5, that + 1)] yr for a dataset of D years, so that its
    frequency stays finite over the whole dataset.  Dataset i uses seed seed0 + i for every draw.
    Returns a list of (Workload, snr)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        dur = rng.uniform(0.25, 2.0) * YEAR_S
        T = float(rng.choice([1e4, 2e4, 5e4, 1e5]))
        K = int(rng.choice([4, 6, 8]))
        N = int(round(10.0 ** rng.uniform(4.0, 6.0)))
        snr = float(rng.uniform(15.0, 40.0))
        L = int(round(T / 5.0))
        n_seg = max(1, int(dur // T))
        # the family's frequency diverges at t = tau: keep tau beyond the dataset's span
        tau_lo = max(1.5, 1.25 * dur / YEAR_S)
        out.append((Workload(f"batch{seed0 + i}", 5.0, n_seg * L, T, K, N, 1, 2000, "powerlaw", "oneyear",
                             seed0 + i, (tau_lo, max(5.0, tau_lo + 1.0))), snr))
    return out


def make_batched_inputs(item):
    """Strain, PSD bins and training tracks of one batched dataset (picklable: for a
    process pool).  ``item`` is one entry of ``batched_workloads``."""
    w, snr = item
    rng = np.random.default_rng(w.seed)
    x, inj = make_strain(w, rng, snr=snr)
    psd = psd_bins(w.psd_fn(), w.n_bin, w.T_sft)
    F = make_training_tracks(w, rng)
    return x, psd, F


def noise_power_table(n_seg: int, n_bin: int, rng: np.random.Generator):
    """A normalised power table of stationary Gaussian noise without its window's bin
    correlations: every P[alpha][k] is chi^2_2 (exponential with mean 2), P[alpha][0] = 0.
    Stands in for tables built from strain where only their shape and value distribution
    matter (serving throughput)."""
    P = rng.exponential(2.0, (n_seg, n_bin))
    P[:, 0] = 0.0
    return P


def served_requests(n: int, rate_hz: float, n_datasets: int, seed: int = 0,
                    tracks=(1e3, 1e6), dtypes=("bf16", "f32")):
    """Poisson arrivals: (arrival time s, dataset index, track count, table dtype) per request,
    exponential inter-arrival times at ``rate_hz``, track counts log-uniform in ``tracks``."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    ds = rng.integers(0, n_datasets, n)
    N = np.round(10.0 ** rng.uniform(math.log10(tracks[0]), math.log10(tracks[1]), n)).astype(np.int64)
    dt = rng.integers(0, len(dtypes), n)
    return [(float(t[i]), int(ds[i]), int(N[i]), dtypes[int(dt[i])]) for i in range(n)]



def make_strain_device(w: Workload, seed: int, snr: float = 30.0):
    """The same draw as ``make_strain`` for a coloured-noise workload (noise of the workload's PSD
    plus one power-law harmonic at the given SNR), made on the current CUDA device with torch so
    that many long datasets can be drawn quickly: Philox normal draws stand in for PCG64's (not
    the same numbers; the same distributions and structure).  Returns (device strain, injection)."""
    import torch

    assert w.psd == "oneyear", "make_strain_device draws the one-year PSD's noise"
    dev = torch.device("cuda")
    n, dt = w.n_samples, w.dt
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    nf = n // 2 + 1
    f = torch.arange(nf, dtype=torch.float64, device=dev) / (n * dt)
    s = 1e-40 * (1.0 + (2e-3 / f.clamp_min(1e-300)) ** 4) * (1.0 + (f / 2.5e-2) ** 2)
    s[0] = 0.0
    var = s * (n / (2.0 * dt))
    sd = torch.sqrt(var / 2.0)
    X = torch.complex(sd * torch.randn(nf, generator=g, dtype=torch.float64, device=dev),
                      sd * torch.randn(nf, generator=g, dtype=torch.float64, device=dev))
    X[0] = 0.0
    if n % 2 == 0:
        X[-1] = torch.sqrt(var[-1]) * torch.randn(1, generator=g, dtype=torch.float64, device=dev)[0]
    del f, s, var, sd
    x = torch.fft.irfft(X, n=n)
    del X
    rng = np.random.default_rng(seed)
    f0, tau, p = powerlaw_params(1, rng, tau_yr=w.tau_yr)
    f0, tau, p = float(f0[0]), float(tau[0]), float(p[0])
    t = torch.arange(n, dtype=torch.float64, device=dev) * dt
    u = 1.0 - t / tau
    fr = f0 * u ** (-p)
    shape = (fr / f0) ** (2.0 / 3.0)
    # SNR^2 = int a^2 / S_n(f(t)) dt (rectangle rule), as powerlaw_amplitude_for_snr
    sn = 1e-40 * (1.0 + (2e-3 / fr) ** 4) * (1.0 + (fr / 2.5e-2) ** 2)
    a0 = snr / math.sqrt(float(torch.sum(shape * shape / sn)) * dt)
    x += a0 * shape * torch.cos(2.0 * math.pi * f0 * tau / (1.0 - p) * (1.0 - u ** (1.0 - p)))
    return x, dict(kind="powerlaw", f0=f0, tau=tau, p=p, snr=snr, a0=a0)
