"""Pins of the oracle's linear-chirp statistic (Sec. II.B, Eq. det_stat with the chirping
local template), each against something other than the oracle itself:

* the template of a bin-centred, non-chirping tone: the periodic Hann window's DFT
  (L/2 at the tone's bin, -L/4 at its neighbours, 0 elsewhere) times the phase of the
  segment midpoint;
* the template of a chirp against the continuous Fourier integral of the windowed
  linear chirp in closed form (Fresnel integrals from scipy), which the sampled SFT of a
  Hann-windowed chirp equals up to aliasing;
* Cauchy-Schwarz: data equal to a multiple of the template reach norm |A|^2 <h|h> and
  any other template gives less;
* a noise-free bin-centred real tone: S_alpha = A^2 L dt / S_n exactly, and a noise-free
  linear-chirp strain: the matched track reaches the Cauchy-Schwarz value while the
  opposite-sign fdot falls far below it;
* brute force: explicit loops over tracks, segments, bins and samples on a tiny case;
* the validity mask zeroes whole segments.
"""
import numpy as np
import pytest

import oracle.tfstat_oracle as O


def test_chirp_template_bin_centred_closed_form():
    L, dt = 256, 0.5
    T = L * dt
    for b in (3, 40, 101):
        bins = np.arange(b - 5, b + 6)[None, :]
        h = O.chirp_template_sft(np.array([b / T]), np.array([0.0]), T, dt, bins)[0]
        phase = np.exp(-1j * np.pi * b)
        want = np.zeros(11, dtype=complex)
        want[5] = dt * L / 2 * phase
        want[4] = want[6] = -dt * L / 4 * phase
        assert np.max(np.abs(h - want)) <= 1e-12 * dt * L


def _fresnel_rect(delta, beta):
    """R(delta, beta) = int_{-1/2}^{1/2} exp(i pi (2 delta x + beta x^2)) dx (beta > 0)."""
    from scipy.special import fresnel

    s = np.sqrt(2.0 * beta)
    S2, C2 = fresnel(s * (0.5 + delta / beta))
    S1, C1 = fresnel(s * (-0.5 + delta / beta))
    return np.exp(-1j * np.pi * delta ** 2 / beta) / s * ((C2 - C1) + 1j * (S2 - S1))


@pytest.mark.parametrize("beta", [0.3, 5.0, 40.0])
@pytest.mark.parametrize("delta0", [0.13, -0.41])
def test_chirp_template_matches_continuous_integral(beta, delta0):
    pytest.importorskip("scipy")
    L, dt = 4096, 2.0
    T = L * dt
    b = 700
    f = (b + delta0) / T
    fdot = beta / T ** 2
    k = np.arange(b - 100, b + 101)
    h = O.chirp_template_sft(np.array([f]), np.array([fdot]), T, dt, k[None, :])[0]
    dk = f * T - k
    # Hann = 1/2 + (e^{2 pi i x} + e^{-2 pi i x}) / 4 on x in [-1/2, 1/2]
    cont = T * np.exp(-1j * np.pi * k) * (0.5 * _fresnel_rect(dk, beta)
                                          + 0.25 * _fresnel_rect(dk + 1, beta) + 0.25 * _fresnel_rect(dk - 1, beta))
    assert np.max(np.abs(h - cont)) <= 1e-6 * np.max(np.abs(h))


def _single_segment_case(rng, n_bin=300, L=512, dt=1.0):
    T = L * dt
    psd = rng.uniform(0.5, 2.0, n_bin)
    return T, dt, psd


def test_chirp_cauchy_schwarz():
    rng = np.random.default_rng(0)
    L, dt = 512, 1.0
    T, _, psd = _single_segment_case(rng, L=L, dt=dt)
    f0, fd0 = 120.3 / T, 3.7 / T ** 2
    F = np.array([[f0]])
    b = int(np.floor(f0 * T + 0.5))
    k = np.arange(b - O.CHIRP_P, b + O.CHIRP_P + 1)
    A = 0.7 * np.exp(0.4j)
    d = np.zeros((1, 300), dtype=complex)
    inside = (k >= 1) & (k < 300)
    h = O.chirp_template_sft(np.array([f0]), np.array([fd0]), T, dt, k[None, :])[0]
    d[0, k[inside]] = A * h[inside]
    # one segment: fdot from finite differences is 0, so pass the chirp through a 3-segment track
    d3 = np.repeat(d, 3, axis=0)
    F3 = np.array([[f0 - fd0 * T, f0, f0 + fd0 * T]])
    w = O.window(L)
    norm = 4.0 / (dt * np.sum(w * w))
    S = O.chirp_statistic(d3, psd, dt, T, F3, valid=np.array([[False, True, False]]))
    want = norm * abs(A) ** 2 * np.sum(np.abs(h[inside]) ** 2 / psd[k[inside]])
    assert abs(S[0] - want) <= 1e-10 * want
    for df, dfd in [(0.2 / T, 0.0), (0.0, 0.5 / T ** 2), (-0.3 / T, -0.2 / T ** 2)]:
        Fo = np.array([[f0 + df - (fd0 + dfd) * T, f0 + df, f0 + df + (fd0 + dfd) * T]])
        So = O.chirp_statistic(d3, psd, dt, T, Fo, valid=np.array([[False, True, False]]))
        assert So[0] < want * (1 - 1e-3)


def test_chirp_bin_centred_real_tone():
    dt, L, n_seg = 1.0, 1024, 3
    T = L * dt
    A, k0, phi = 0.05, 123, 0.7
    t = np.arange(L * n_seg) * dt
    x = A * np.cos(2 * np.pi * k0 / T * t + phi)
    d = O.sft(x, dt, T)
    psd = np.full(L // 2 + 1, 2.0)
    F = np.full((4, n_seg), k0 / T)
    S = O.chirp_statistic(d, psd, dt, T, F)
    assert np.allclose(S, n_seg * A * A * L * dt / 2.0, rtol=1e-11, atol=0)
    # the nearest-bin power of the same tone is 2/3 of it (the Hann window spreads it over 3 bins)
    Pt = O.power_table(x, dt, T, psd)
    assert np.allclose(Pt[:, k0], (2.0 / 3.0) * A * A * L * dt / 2.0, rtol=1e-11)


def test_chirp_linear_chirp_strain():
    """A global linear chirp is, in every segment, the local chirp of its own track."""
    dt, L, n_seg = 1.0, 2048, 6
    T = L * dt
    A = 0.02
    f0, fdot = 300.2 / T, 6.0 / T ** 2
    t = np.arange(L * n_seg) * dt
    x = A * np.cos(2 * np.pi * (f0 * t + 0.5 * fdot * t * t) + 0.3)
    d = O.sft(x, dt, T)
    psd = np.full(L // 2 + 1, 1.0)
    ta = O.segment_times(n_seg, T)
    F = (f0 + fdot * ta)[None, :]
    S = O.chirp_statistic(d, psd, dt, T, F)
    # Cauchy-Schwarz value per segment: norm (A/2)^2 <h|h>, up to the negative-frequency image
    w = O.window(L)
    norm = 4.0 / (dt * np.sum(w * w))
    want = 0.0
    b = np.floor(F[0] * T + 0.5).astype(int)
    for a in range(n_seg):
        k = np.arange(b[a] - O.CHIRP_P, b[a] + O.CHIRP_P + 1)
        h = O.chirp_template_sft(np.array([F[0, a]]), np.array([fdot]), T, dt, k[None, :])[0]
        want += norm * (A / 2) ** 2 * np.sum(np.abs(h) ** 2)
    assert abs(S[0] - want) <= 1e-4 * want
    Fneg = (f0 + fdot * T * n_seg - fdot * ta)[None, :]   # same band, opposite-sign fdot
    Sneg = O.chirp_statistic(d, psd, dt, T, Fneg)
    assert Sneg[0] < 0.5 * want
    Fnear = F + 0.0                                         # the nearest-bin power misses the sweep
    Pt = O.power_table(x, dt, T, psd)
    bn, _ = O.bins_and_ties(Fnear * T)
    assert O.statistic(Pt, bn, 0)[0] < 0.5 * want


def test_chirp_statistic_brute_force():
    rng = np.random.default_rng(3)
    dt, L, n_seg, P = 0.25, 16, 4, 3
    T = L * dt
    x = rng.standard_normal(L * n_seg)
    nb = L // 2 + 1
    psd = rng.uniform(0.5, 2.0, nb)
    psd[5] = np.inf
    F = rng.uniform(0.5, nb - 1.5, (5, n_seg)) / T
    F[0] = np.linspace(-0.5, nb + 2, n_seg) / T       # tracks leaving the table at both ends
    got = O.chirp_statistic(O.sft(x, dt, T, method="direct"), psd, dt, T, F, P=P)
    w = np.sin(np.pi * np.arange(L) / L) ** 2
    sw2 = float(np.sum(w * w))
    want = np.zeros(5)
    for t in range(5):
        for a in range(n_seg):
            if a == 0:
                fd = (F[t, 1] - F[t, 0]) / T
            elif a == n_seg - 1:
                fd = (F[t, a] - F[t, a - 1]) / T
            else:
                fd = (F[t, a + 1] - F[t, a - 1]) / (2 * T)
            b = int(np.floor(F[t, a] * T + 0.5))
            if b < 0 or b >= nb:
                continue  # the track's own bin is outside the table
            num, den = 0j, 0.0
            for k in range(b - P, b + P + 1):
                if k < 1 or k >= nb or not np.isfinite(psd[k]):
                    continue
                dk = sum(dt * w[n] * x[a * L + n] * np.exp(-2j * np.pi * n * k / L) for n in range(L))
                hk = 0j
                for n in range(L):
                    u = n * dt - T / 2
                    hk += dt * w[n] * np.exp(1j * (2 * np.pi * F[t, a] * u + np.pi * fd * u * u)) \
                        * np.exp(-2j * np.pi * n * k / L)
                num += np.conj(dk) * hk / psd[k]
                den += abs(hk) ** 2 / psd[k]
            if den > 0:
                want[t] += 4.0 / (dt * sw2) * abs(num) ** 2 / den
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


def test_chirp_statistic_mask():
    rng = np.random.default_rng(4)
    dt, L, n_seg = 1.0, 64, 5
    T = L * dt
    x = rng.standard_normal(L * n_seg)
    d = O.sft(x, dt, T)
    psd = np.ones(L // 2 + 1)
    F = rng.uniform(5, 25, (6, n_seg)) / T
    valid = rng.uniform(0, 1, (6, n_seg)) < 0.5
    full = np.array([[O.chirp_statistic(d[a:a + 1], psd, dt, T, F[t:t + 1, a:a + 1])[0] for a in range(n_seg)]
                     for t in range(6)])
    # with one segment the finite difference is 0; compare against the masked sum of per-segment
    # values computed with the same fdot
    fd, _ = O.finite_differences(F, T)
    per = np.zeros((6, n_seg))
    for a in range(n_seg):
        Fa = np.stack([F[:, a] - fd[:, a] * T, F[:, a], F[:, a] + fd[:, a] * T], axis=1)
        per[:, a] = O.chirp_statistic(np.repeat(d[a:a + 1], 3, axis=0), psd, dt, T, Fa,
                                      valid=np.tile([False, True, False], (6, 1)))
    S = O.chirp_statistic(d, psd, dt, T, F, valid=valid)
    assert np.allclose(S, np.sum(np.where(valid, per, 0.0), axis=1), rtol=1e-12)
    assert not np.allclose(full, per)  # fdot matters

