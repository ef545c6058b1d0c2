"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against one of: a number the paper prints, a
closed form, a library routine reached by a different route, brute force on
tiny inputs (exact rational arithmetic), or chi^2 moments implied by the
normalisation.  A dropped term, wrong sign, wrong index or transposed
operand in the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle.tfstat_oracle as O
from paper_2510_20891_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# --------------------------------------------------------------------------
# Segment bookkeeping: the paper's segment counts (Sec. II.B)
# --------------------------------------------------------------------------
def test_segment_counts_match_paper():
    for dt, T, n_expected in _rows("paper_segment_counts.txt"):
        dt, T, n_expected = float(dt), float(T), int(n_expected)
        n_samples = int(round(synth.JULIAN_YEAR_S / dt))
        L, n_seg, n_bin = O.sft_layout(n_samples, dt, T)
        assert n_seg == n_expected
        assert L == int(T / dt) and n_bin == L // 2 + 1


def test_oneyear_daily_layout():
    w = synth.WORKLOADS["oneyear_daily_fp32"]
    assert O.sft_layout(w.n_samples, w.dt, w.T_sft) == (17280, 365, 8641)
    w = synth.WORKLOADS["oneyear_fine_1577x20001"]
    assert O.sft_layout(w.n_samples, w.dt, w.T_sft) == (40000, 1577, 20001)
    with pytest.raises(ValueError):
        O.sft_layout(1000, 3.0, 10.0)       # T/dt not an integer


def test_segment_times_are_midpoints():
    t = O.segment_times(4, 10.0)
    assert np.array_equal(t, [5.0, 15.0, 25.0, 35.0])


# --------------------------------------------------------------------------
# DFT: the definition against the library FFT, and closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [8, 12, 30, 250, 1000])
def test_direct_dft_matches_library_fft(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal((3, L))
    X1 = O.dft_direct(x)
    X2 = np.fft.rfft(x, axis=1)
    assert np.max(np.abs(X1 - X2)) <= 1e-12 * np.max(np.abs(X2)) * math.log2(L)


def test_dft_closed_forms():
    L = 30
    delta = np.zeros(L)
    delta[0] = 1.0
    assert np.allclose(O.dft_direct(delta), np.ones(L // 2 + 1), atol=1e-14)
    k0 = 7
    c = np.cos(2 * np.pi * k0 * np.arange(L) / L)
    X = O.dft_direct(c)
    expect = np.zeros(L // 2 + 1)
    expect[k0] = L / 2
    assert np.allclose(X, expect, atol=1e-12)


def test_sft_fft_and_direct_agree():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(4 * 64 + 5)
    d1 = O.sft(x, 0.5, 32.0, "hann", "fft")
    d2 = O.sft(x, 0.5, 32.0, "hann", "direct")
    assert d1.shape == (4, 33)
    assert np.max(np.abs(d1 - d2)) < 1e-12 * np.max(np.abs(d1))


# --------------------------------------------------------------------------
# Normalisation: closed form of a bin-centred sinusoid (golden fixture)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("row", _rows("hann_closed_form.txt"))
def test_power_closed_form(row):
    win, L, dt, Sn, A, k0, phi, Pk0, Ppm1 = row
    L, k0 = int(L), int(k0)
    dt, Sn, A, phi, Pk0, Ppm1 = map(float, (dt, Sn, A, phi, Pk0, Ppm1))
    n_seg = 5
    n = np.arange(n_seg * L)
    x = A * np.cos(2 * np.pi * k0 * n / L + phi)
    P = O.power_table(x, dt, L * dt, np.full(L // 2 + 1, Sn), win)
    assert P.shape == (n_seg, L // 2 + 1)
    assert np.allclose(P[:, k0], Pk0, rtol=1e-10)
    assert np.allclose(P[:, k0 - 1], Ppm1, rtol=1e-10, atol=1e-12 * Pk0)
    assert np.allclose(P[:, k0 + 1], Ppm1, rtol=1e-10, atol=1e-12 * Pk0)
    rest = np.delete(P, [k0 - 1, k0, k0 + 1], axis=1)
    assert np.max(rest) <= 1e-20 * Pk0 + 1e-24
    # the constant track at k0: S = n_seg P[k0] (m=0), n_seg (P[k0] + 2 P[k0+-1]) (m=1)
    V = np.ones((1, n_seg)) / math.sqrt(n_seg)
    c = np.array([[0.0]])
    f_ref = np.array([k0 / (L * dt)])
    S, idx, val, ties = O.eval_stat(P, V, c, f_ref, L * dt, 0, 1)
    assert math.isclose(S[0], n_seg * Pk0, rel_tol=1e-10)
    S1, *_ = O.eval_stat(P, V, c, f_ref, L * dt, 1, 1)
    assert math.isclose(S1[0], n_seg * (Pk0 + 2 * Ppm1), rel_tol=1e-10)
    assert ties == []


def test_dc_bin_and_bad_psd_give_zero():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(3 * 16) + 5.0
    psd = np.full(9, 2.0)
    psd[4] = np.inf
    psd[5] = 0.0
    psd[6] = np.nan
    P = O.power_table(x, 1.0, 16.0, psd)
    assert np.all(P[:, 0] == 0) and np.all(P[:, 4:7] == 0)
    assert np.all(P[:, 1:4] > 0)


# --------------------------------------------------------------------------
# Noise: chi^2_2 moments implied by the normalisation, and Hann bin correlations
# --------------------------------------------------------------------------
def test_noise_table_moments():
    rng = np.random.default_rng(11)
    L, n_seg = 4096, 64
    x = rng.standard_normal(L * n_seg)
    P = O.power_table(x, 1.0, float(L), np.full(L // 2 + 1, 2.0))
    inner = P[:, 1:-1]
    n = inner.size
    assert abs(inner.mean() - 2.0) < 5 * 2.0 / math.sqrt(n) * 2      # bins are correlated: x2 slack
    assert abs(inner.var() - 4.0) < 5 * math.sqrt(80.0 / n) * 2      # Var(P^2 est) ~ 80/n for chi2_2/2 * 2
    # lag-1 and lag-2 power correlations |rho|^2 of the periodic Hann window: 4/9 and 1/36
    a = inner - inner.mean()
    c1 = np.mean(a[:, 1:] * a[:, :-1]) / inner.var()
    c2 = np.mean(a[:, 2:] * a[:, :-2]) / inner.var()
    c3 = np.mean(a[:, 3:] * a[:, :-3]) / inner.var()
    assert abs(c1 - 4.0 / 9.0) < 0.03
    assert abs(c2 - 1.0 / 36.0) < 0.03
    assert abs(c3) < 0.03


def test_noise_statistic_moments_over_random_tracks():
    # Over random tracks on independent noise: E[S] = 2 N_a (2m+1); Var[S] = 4 N_a (m = 0)
    # and Var[S] = N_a (12 + 2 (2*4*4/9 + 4*1/36)) = 19.333 N_a (m = 1).
    rng = np.random.default_rng(5)
    L, n_seg, Nb = 256, 16, 129
    S0, S1 = [], []
    for _ in range(400):
        x = rng.standard_normal(L * n_seg)
        P = O.power_table(x, 1.0, float(L), np.full(Nb, 2.0))
        b = rng.integers(4, Nb - 4, size=(25, n_seg))
        S0.append(O.statistic(P, b, 0))
        S1.append(O.statistic(P, b, 1))
    S0, S1 = np.concatenate(S0), np.concatenate(S1)
    n = S0.size
    assert abs(S0.mean() - 2 * n_seg) < 5 * math.sqrt(4 * n_seg / n) * 2
    assert abs(S0.var() / (4 * n_seg) - 1) < 0.08
    assert abs(S1.mean() - 2 * n_seg * 3) < 5 * math.sqrt(19.34 * n_seg / n) * 2
    assert abs(S1.var() / (19.0 + 1.0 / 3.0) / n_seg - 1) < 0.08


# --------------------------------------------------------------------------
# Track -> bin: exact rational arithmetic on tiny inputs, ties, non-finite
# --------------------------------------------------------------------------
def _exact_x(V, c, f_ref, T):
    out = np.empty((c.shape[0], V.shape[1]), dtype=object)
    for t in range(c.shape[0]):
        for a in range(V.shape[1]):
            f = Fraction(float(f_ref[t]))
            for k in range(V.shape[0]):
                f += Fraction(float(c[t, k])) * Fraction(float(V[k, a]))
            out[t, a] = f * Fraction(float(T))
    return out


def test_track_bins_match_exact_rational_arithmetic():
    rng = np.random.default_rng(7)
    K, n_seg, N, T = 4, 9, 40, 4096.0
    V = rng.standard_normal((K, n_seg)) * 1e-3
    c = rng.standard_normal((N, K))
    f_ref = rng.uniform(0, 0.05, N)
    x = O.track_x(V, c, f_ref, T)
    b, tie = O.bins_and_ties(x)
    ex = _exact_x(V, c, f_ref, T)
    checked = 0
    for t in range(N):
        for a in range(n_seg):
            xe = ex[t, a]
            be = math.floor(xe + Fraction(1, 2))
            dist = abs(xe - math.floor(xe) - Fraction(1, 2))
            assert abs(float(xe) - x[t, a]) <= 1e-11 * max(1.0, abs(float(xe)))
            if dist > Fraction(1, 10 ** 9):
                assert b[t, a] == be and not tie[t, a]
                checked += 1
    assert checked > 0.99 * N * n_seg


def test_ties_are_flagged_and_round_half_up():
    T = 4096.0                                   # power of two: (k + 1/2)/T is exact in FP64
    V = np.zeros((1, 3))
    c = np.zeros((4, 1))
    f_ref = np.array([(10 + 0.5) / T, (11 + 0.5) / T, 12.25 / T, (13 + 0.5 + 5e-10) / T])
    b, tie = O.bins_and_ties(O.track_x(V, c, f_ref, T))
    assert b[:, 0].tolist() == [11, 12, 12, 14]
    assert tie[:, 0].tolist() == [True, True, False, True]


def test_nonfinite_and_far_tracks_contribute_zero():
    P = np.ones((2, 10))
    b, tie = O.bins_and_ties(np.array([[np.nan, np.inf], [-1e300, 3.0]]))
    assert not tie.any()
    S = O.statistic(P, b, 1)
    assert S.tolist() == [0.0, 3.0]


# --------------------------------------------------------------------------
# The statistic: vectorised gather against plain loops, out-of-range rule
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [0, 1, 2, 5])
def test_statistic_vectorised_equals_loops(m):
    rng = np.random.default_rng(m)
    n_seg, Nb = 6, 17
    P = rng.random((n_seg, Nb))
    b = rng.integers(-8, Nb + 8, size=(30, n_seg))
    assert np.allclose(O.statistic(P, b, m), O.statistic_loop(P.tolist(), b.tolist(), m), rtol=1e-14)


def test_edge_window_is_truncated_not_clamped():
    P = np.arange(1.0, 6.0)[None, :]             # one segment, bins 0..4 hold 1..5
    assert O.statistic(P, np.array([[0]]), 1)[0] == 1 + 2
    assert O.statistic(P, np.array([[4]]), 1)[0] == 4 + 5
    assert O.statistic(P, np.array([[-1]]), 1)[0] == 1
    assert O.statistic(P, np.array([[-2]]), 1)[0] == 0
    assert O.statistic(P, np.array([[5]]), 1)[0] == 5
    assert O.statistic(P, np.array([[6]]), 1)[0] == 0


# --------------------------------------------------------------------------
# Top-k: brute-force Python sort
# --------------------------------------------------------------------------
def test_topk_bruteforce():
    rng = np.random.default_rng(2)
    S = rng.integers(0, 6, 200).astype(np.float64)
    S[[3, 50, 77]] = np.nan
    S[[4, 5]] = [-0.0, 0.0]
    for k in (1, 5, 37, 200, 500):
        idx, val = O.topk(S, k)

        def key(i):
            v = S[i]
            return (1, 0.0, i) if math.isnan(v) else (0, -v, i)

        ref = sorted(range(S.size), key=key)[: min(k, S.size)]
        assert idx.tolist() == ref
        assert np.array_equal(val, S[ref], equal_nan=True)


# --------------------------------------------------------------------------
# Quantisers: library conversions reached by a different route, hand values
# --------------------------------------------------------------------------
def test_round_f16_matches_numpy():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 5, 20000),
                        [65504.0, 65519.0, 65520.0, 1e5, 6e-8, 2 ** -25, 2 ** -24 * 1.5]])
    assert np.array_equal(O.round_f16(x), x.astype(np.float16).astype(np.float64))


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x.astype(np.float64)), ref)
    # hand values: ties go to the even mantissa
    assert O.round_bf16(np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8])).tolist() == [1.0, 1 + 2 ** -6]


def test_round_f8e4m3_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    x = (rng.uniform(-440, 440, 20000) * 10.0 ** rng.integers(-4, 1, 20000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.round_f8e4m3(x.astype(np.float64)), ref)
    hv = O.round_f8e4m3(np.array([448.0, 500.0, 2 ** -9, 2 ** -10, 1.0625, 1.1875, 2 ** -6 * 1.0625]))
    assert hv.tolist() == [448.0, 448.0, 2 ** -9, 0.0, 1.0, 1.25, 2 ** -6]


def test_quantise_f8_per_segment_scale():
    # row 0: positive exponents floor(log2) = [0, 10]; lower median 0 -> M = min(1344, 256) = 256
    P = np.array([[0.0, 1.0, 448.0 * 3], [0.0, 0.0, 0.0]])
    deq, s = O.quantise_table(P, "f8e4m3")
    assert s.dtype == np.float32 and s.tolist() == [np.float32(256 / 448), 1.0]
    s0 = float(np.float32(256 / 448))
    q1 = O.round_f8e4m3(np.array([1.0 / s0]))[0]
    assert deq[0].tolist() == [0.0, float(np.float32(q1) * np.float32(s0)), float(np.float32(448.0) * np.float32(s0))]
    assert deq[1].tolist() == [0.0, 0.0, 0.0]
    # hand values of the row reference: exponents [1, 1, 5, 2] -> lower median 1 -> min(40, 512) = 40
    assert O.f8_row_reference([2.0, 3.0, 40.0, 5.0]) == 40.0
    # a leakage outlier: exponents [0, 1, 1, 26] -> lower median 1 -> M = 256 * 2 = 512
    assert O.f8_row_reference([1.0, 2.0, 3.0, 1e8]) == 512.0
    assert O.f8_row_reference([0.0, -1.0]) == 0.0


# --------------------------------------------------------------------------
# SVD basis: exact-rank family, Gram-matrix route to the singular values
# --------------------------------------------------------------------------
def test_svd_basis_quadratic_family_is_rank_three():
    w = synth.WORKLOADS["tiny_white_2p18"]
    rng = np.random.default_rng(0)
    F = synth.make_training_tracks(w, rng)
    V, s, cmin, cmax = O.svd_basis(F, 3)
    assert V.shape == (3, w.n_seg)
    assert np.allclose(V @ V.T, np.eye(3), atol=1e-13)
    held = synth.make_training_tracks(w, np.random.default_rng(99), 200)
    assert np.max(O.reconstruction_error(held, V)) <= 1e-12
    # singular values through the Gram matrix (a different LAPACK route)
    ev = np.sort(np.linalg.eigvalsh(F.T @ F))[::-1][:3]
    assert np.allclose(s, np.sqrt(ev), rtol=1e-9)
    C = F @ V.T
    assert np.allclose(cmin, C.min(0)) and np.allclose(cmax, C.max(0))
    # tolerance-driven K finds the exact rank
    V2, *_ = O.svd_basis(F, 0, 1e-12)
    assert V2.shape[0] == 3


def test_svd_basis_constant_family_closed_form():
    n_seg = 12
    f0 = np.linspace(1e-3, 2e-3, 7)
    F = f0[:, None] * np.ones((1, n_seg))
    V, s, cmin, cmax = O.svd_basis(F, 1)
    assert np.allclose(V[0], 1 / math.sqrt(n_seg), rtol=1e-13)
    assert math.isclose(s[0], math.sqrt(n_seg * np.sum(f0 ** 2)), rel_tol=1e-13)
    assert math.isclose(cmin[0], f0[0] * math.sqrt(n_seg), rel_tol=1e-13)
    assert math.isclose(cmax[0], f0[-1] * math.sqrt(n_seg), rel_tol=1e-13)


# --------------------------------------------------------------------------
# The injected signal stands far above the noise (tiny white workload)
# --------------------------------------------------------------------------
def test_injected_track_stands_out():
    w = synth.WORKLOADS["tiny_white_2p18"]
    rng = np.random.default_rng(0)
    x, inj = synth.make_strain(w, rng)
    P = O.power_table(x, w.dt, w.T_sft, synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft))
    V, s, cmin, cmax = O.svd_basis(synth.make_training_tracks(w, rng), 3)
    t = O.segment_times(w.n_seg, w.T_sft)
    f_true = inj["f0"] + inj["fdot"] * t
    c_true = (f_true @ V.T)[None, :]
    S, *_ = O.eval_stat(P, V, c_true, np.zeros(1), w.T_sft, 0)
    # noise alone: mean 2 * 64 = 128, std 16; signal adds about (2/3) SNR_seg^2 per segment
    assert S[0] - 128 > 10 * 16


# --------------------------------------------------------------------------
# Segment exclusions (Sec. II.B second-order cut, Sec. II.D low f / low fdot)
# --------------------------------------------------------------------------
def _quad_tracks(a, b, c, n_seg, T):
    """f(t) = a + b t + c t^2 / 2 at the segment midpoints, one row per (a, b, c)."""
    t = O.segment_times(n_seg, T)
    return a[:, None] + b[:, None] * t[None, :] + 0.5 * c[:, None] * t[None, :] ** 2, t


def test_segment_validity_second_order_cut_closed_form():
    """For a quadratic track the second difference is exact: z = fddot T^3 / 6 in every
    segment (the ends take the inner value), so the cut is all or nothing at c T^3/6 = 1."""
    T, n_seg = 5.0e4, 40
    c_cut = 6.0 / T ** 3
    c = np.array([0.2, 0.5, 0.9, 1.1, 1.5, 3.0]) * c_cut
    a = np.full(c.size, 5e-3)
    b = np.full(c.size, 1e-11)   # well above the fdot floor
    F, t = _quad_tracks(a, b, c, n_seg, T)
    valid = O.segment_validity(F, T)
    expect = (c * T ** 3 / 6.0 <= 1.0)
    assert np.array_equal(valid, np.repeat(expect[:, None], n_seg, axis=1))


def test_segment_validity_fdot_closed_form():
    """Central differences are exact for quadratics: fdot(t_alpha) = b + c t_alpha inside;
    the end segments use one-sided differences, off by c T / 2."""
    T, n_seg = 1.0e4, 30
    a = np.array([4e-3])
    b = np.array([-1e-13])
    c = np.array([1e-18])          # fdot crosses 1e-13 Hz/s inside the track
    F, t = _quad_tracks(a, b, c, n_seg, T)
    valid = O.segment_validity(F, T)[0]
    fd = b[0] + c[0] * t
    fd[0] = fd[0] + c[0] * T / 2.0
    fd[-1] = fd[-1] - c[0] * T / 2.0
    far = np.abs(fd - 1e-13) > 1e-16
    assert np.array_equal(valid[far], (fd >= 1e-13)[far])
    assert (~valid).any() and valid.any()


def test_segment_validity_low_frequency():
    T, n_seg = 2.0e4, 20
    f0 = np.array([2e-4, 3.1e-4, 3.2e-4, 1e-3])   # 10^-3.5 = 3.162e-4
    F, t = _quad_tracks(f0, np.full(4, 1e-12), np.zeros(4), n_seg, T)
    valid = O.segment_validity(F, T)
    assert np.array_equal(valid, F >= 10.0 ** -3.5)
    assert not valid[0].any() and valid[3].all()


def test_segment_validity_short_tracks():
    """One segment: no derivative (0 < 1e-13), so it is excluded; two segments: one-sided
    differences and no second-order term."""
    F1 = np.array([[5e-3]])
    assert not O.segment_validity(F1, 1e4).any()
    F2 = np.array([[5e-3, 5e-3 + 1e-8]])       # fdot = 1e-12 on both
    assert O.segment_validity(F2, 1e4).all()


def test_statistic_masked_reduces_to_statistic_and_loop():
    rng = np.random.default_rng(3)
    P = rng.exponential(2.0, (9, 40))
    b = rng.integers(-3, 43, (25, 9))
    ones = np.ones_like(b, dtype=bool)
    assert np.allclose(O.statistic_masked(P, b, ones, 1), O.statistic(P, b, 1), rtol=0, atol=1e-12)
    valid = rng.random(b.shape) < 0.6
    loop = np.array([sum(P[a, k] for a in range(9) for k in range(b[t, a] - 2, b[t, a] + 3)
                         if 0 <= k < 40 and valid[t, a]) for t in range(25)])
    assert np.allclose(O.statistic_masked(P, b, valid, 2), loop, rtol=0, atol=1e-12)


def test_eval_stat_masked_drops_only_excluded_segments():
    """A track whose second half is past the cut scores exactly the first half's sum."""
    T, n_seg, n_bin = 1.0e4, 16, 400
    P = np.random.default_rng(4).exponential(2.0, (n_seg, n_bin))
    V = np.eye(n_seg)                       # basis = the track values themselves
    t = O.segment_times(n_seg, T)
    f = 5e-3 + 1e-10 * t
    f[8:] = f[8:] + 0.5 * 1e-9 * (t[8:] - t[7]) ** 2 * 1e3   # strongly curved second half
    S, valid = O.eval_stat_masked(P, V, f[None, :], np.zeros(1), T, 0)
    b = np.floor(f * T + 0.5).astype(int)
    assert valid[0, :7].all() and not valid[0, 9:].all()
    expect = sum(P[a, b[a]] for a in range(n_seg) if valid[0, a])
    assert math.isclose(S[0], expect, rel_tol=1e-15)
