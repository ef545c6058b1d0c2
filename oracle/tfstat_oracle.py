"""Plain FP64 CPU oracle for the semi-coherent time-frequency track statistic.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline (and its ``--impl reference`` arm) use it.  It shares no code with
the CUDA path (no kernels, helpers, tables or constant generators).

What it computes, step by step, each in the plainest form:

* ``sft`` / ``power_table``: the SFTs d~_{alpha,k} of non-overlapping windowed
  segments and the PSD-normalised power 4 Delta f |d~|^2 / S_n (Sec. II.B, the
  detection statistic of Eq. (det_stat) and the inner product beneath it,
  with Delta f = 1/T_SFT), generalised for a window so that noise gives a
  chi^2 with two degrees of freedom and mean 2.
* ``svd_basis``: the SVD track basis f_{i,alpha} = sum_p U_{i,p} S_p V_{p,alpha},
  truncated to K rows of V (Sec. II.C).
* ``track_x`` / ``bins_and_ties``: f_alpha = f_ref + sum_k xi_k V_{k,alpha}
  (Sec. II.C) mapped to the nearest SFT bin.
* ``statistic``: S~ = sum_alpha S_alpha, here with the nearest-bin reading of
  S_alpha plus an optional +-m neighbour sum (Sec. II.B, Eq. det_stat).
* ``topk``: keep the best k tracks (Sec. II.D keeps the best 512 of 1024).
* ``track_freqs`` / ``segment_validity`` / ``statistic_masked``: the per-segment
  exclusions of the search: S_alpha = 0 where the track's second-order
  evolution breaks the linear model, fddot_alpha T_SFT^3 / 6 > 1 (Sec. II.B,
  the T_SFT discussion), and where the track's frequency is below 10^-3.5 Hz
  or its frequency derivative below 1e-13 Hz/s (Sec. II.D).
* ``chirp_template_sft`` / ``chirp_statistic``: the paper's own S_alpha of
  Eq. det_stat with the chirping sinusoid of Sec. II.B as the local template:
  the template's SFT over the 2P + 1 = 201 bins around the track, fdot from
  the finite differences, |sum d~* h~ / S_n|^2 normalised by <h|h>.
* ``chunk_layout`` / ``chunk_eval`` / ``noise_moments``: the plunge-time search
  over data chunks of growing duration with an integer time shift of the
  basis, and the noise mean and standard deviation that normalise each
  duration (Sec. II.D).

Readings where the paper is silent (window, normalisation constant, DC bin,
rounding rule, tie band, out-of-range bins, segment times, quantised
storage) are stated beside each function.

Parity pins: every function here is pinned by tests/test_oracle_pins.py
against closed forms, library routines, brute force or chi^2 moments.
"""
from __future__ import annotations

import math

import numpy as np

TIE_BAND = 1e-9          # |frac(x) - 1/2| <= TIE_BAND is a rounding tie
F8_E4M3_MAX = 448.0

DTYPES = ("f32", "bf16", "f16", "f8e4m3")


# --------------------------------------------------------------------------
# Segmentation (Sec. II.B: segments alpha of duration T_SFT, Delta f = 1/T_SFT)
# --------------------------------------------------------------------------
def sft_layout(n_samples: int, dt: float, T_sft: float):
    """Return (L, n_seg, n_bin): L = T_SFT/dt samples per segment (must be an
    integer), n_seg = floor(n_samples / L) non-overlapping segments (a ragged
    remainder is dropped), n_bin = L//2 + 1 one-sided bins."""
    Lf = T_sft / dt
    L = int(round(Lf))
    if L < 2 or abs(Lf - L) > 1e-9 * max(1.0, Lf):
        raise ValueError("T_sft / dt must be an integer >= 2")
    return L, n_samples // L, L // 2 + 1


def segment_times(n_seg: int, T_sft: float):
    """Reading: t_alpha is the segment midpoint (alpha + 1/2) T_SFT."""
    return (np.arange(n_seg, dtype=np.float64) + 0.5) * T_sft


def window(L: int, kind: str = "hann"):
    """Reading: the paper names no window; 'hann' is the periodic Hann
    w[n] = sin^2(pi n / L); 'rect' is all ones."""
    n = np.arange(L, dtype=np.float64)
    if kind == "hann":
        return np.sin(np.pi * n / L) ** 2
    if kind == "rect":
        return np.ones(L)
    raise ValueError(kind)


# --------------------------------------------------------------------------
# DFT (Sec. II.B: d~_{alpha,k} is the SFT of the data in segment alpha)
# --------------------------------------------------------------------------
def dft_direct(x):
    """X_k = sum_n x[n] exp(-2 pi i n k / L), k = 0..L//2, by the definition (O(L^2))."""
    x = np.asarray(x, dtype=np.float64)
    L = x.shape[-1]
    nb = L // 2 + 1
    out = np.empty(x.shape[:-1] + (nb,), dtype=np.complex128)
    n = np.arange(L, dtype=np.int64)
    for k in range(nb):
        # reduce n k mod L exactly in integers before forming the angle
        ang = -2.0 * np.pi * ((n * k) % L) / L
        out[..., k] = x @ np.exp(1j * ang)
    return out


def sft(strain, dt: float, T_sft: float, window_kind: str = "hann", method: str = "fft"):
    """d~_{alpha,k} = dt sum_n w[n] x[alpha L + n] e^{-2 pi i n k / L} for k = 0..L/2."""
    strain = np.asarray(strain, dtype=np.float64)
    L, n_seg, _ = sft_layout(strain.size, dt, T_sft)
    seg = strain[: n_seg * L].reshape(n_seg, L) * window(L, window_kind)[None, :]
    X = np.fft.rfft(seg, axis=1) if method == "fft" else dft_direct(seg)
    return dt * X


def power_table(strain, dt: float, T_sft: float, psd_bins, window_kind: str = "hann", method: str = "fft"):
    """P[alpha,k] = 4 |d~_{alpha,k}|^2 / (dt * sum_n w[n]^2 * S_n(k/T_SFT))  (FP64).

    Readings: this is the paper's 4 Delta f |d~|^2 / S_n with T_SFT = L dt
    replaced by dt * sum w^2 (equal for the rectangular window) so that
    Gaussian noise gives P ~ chi^2_2 with mean 2 in every interior bin; the
    DC bin is set to 0; a bin whose S_n is not finite and positive gives 0.
    """
    L, n_seg, n_bin = sft_layout(np.asarray(strain).size, dt, T_sft)
    d = sft(strain, dt, T_sft, window_kind, method)
    w = window(L, window_kind)
    sw2 = float(np.sum(w * w))
    S = np.asarray(psd_bins, dtype=np.float64)
    if S.shape != (n_bin,):
        raise ValueError("psd must have n_bin entries")
    ok = np.isfinite(S) & (S > 0)
    denom = np.where(ok, dt * sw2 * np.where(ok, S, 1.0), 1.0)
    P = 4.0 * (d.real ** 2 + d.imag ** 2) / denom[None, :]
    P[:, ~ok] = 0.0
    P[:, 0] = 0.0
    return P


# --------------------------------------------------------------------------
# Reduced-precision storage of the table (the stored values, dequantised)
# --------------------------------------------------------------------------
def _round_to_grid(x, mant_bits: int, emin: int):
    """Round-to-nearest-even of FP64 values onto a binary floating grid with
    ``mant_bits`` explicit fraction bits and minimum normal exponent ``emin``
    (subnormals below 2^emin); no overflow handling."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = (x != 0) & np.isfinite(x)
    ax = np.abs(x[nz])
    e = np.floor(np.log2(ax))
    # guard against log2 rounding at exact powers of two
    e = np.where(2.0 ** e > ax, e - 1, e)
    e = np.where(2.0 ** (e + 1) <= ax, e + 1, e)
    e = np.maximum(e, emin)
    q = 2.0 ** (e - mant_bits)          # spacing of the grid near ax
    out[nz] = np.sign(x[nz]) * np.rint(ax / q) * q   # np.rint is ties-to-even
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out


def round_bf16(x):
    """FP64 -> bfloat16 (8 exponent bits, 7 fraction bits), round to nearest even; overflow -> inf."""
    y = _round_to_grid(x, 7, -126)
    return np.where(np.abs(y) > 3.3895313892515355e38, np.copysign(np.inf, y), y)


def round_f16(x):
    """FP64 -> IEEE binary16 (5 exponent bits, 10 fraction bits), round to nearest even; overflow -> inf."""
    y = _round_to_grid(x, 10, -14)
    return np.where(np.abs(y) > 65504.0, np.copysign(np.inf, y), y)


def round_f8e4m3(x):
    """FP64 -> FP8 E4M3 (4 exponent bits, 3 fraction bits, bias 7, max 448, no inf),
    round to nearest even, saturating at +-448."""
    y = _round_to_grid(x, 3, -6)
    return np.clip(y, -F8_E4M3_MAX, F8_E4M3_MAX)


def f8_row_reference(row):
    """M = min(max P, 256 * 2^e*), e* = lower median of floor(log2 P) over P > 0 (0 if none)."""
    row = np.asarray(row, dtype=np.float64)
    pos = row[row > 0]
    if pos.size == 0:
        return 0.0
    _, ex = np.frexp(pos)                      # pos = mant * 2^ex with mant in [0.5, 1)
    e = np.sort(ex - 1)                        # floor(log2 pos), exact
    e_star = int(e[(pos.size + 1) // 2 - 1])   # the ceil(n/2)-th smallest
    return float(min(pos.max(), 256.0 * 2.0 ** e_star))


def quantise_table(P, dtype: str):
    """Values the table holds in storage ``dtype``, returned dequantised in FP64,
    plus the per-segment FP32 scales (FP8 only, else None).

    f32 / bf16 / f16: P rounded to nearest even in that format.
    f8e4m3: s_alpha = fp32(M_alpha / 448) (1 when M_alpha = 0) with
    M_alpha = min(max_k P[alpha,k], 256 * 2^e*), e* the lower median of
    floor(log2 P[alpha,k]) over the row's positive entries; q = e4m3(P / s_alpha)
    with the division in FP64 and saturation at 448; dequantised as q * s_alpha.
    Reading: the paper fixes no FP8 scale.  A plain max/448 scale fails on the
    one-year PSD, whose f^-4 red noise leaks ~1e8 times the in-band power into
    the lowest bins and would push every in-band value below e4m3's smallest
    subnormal; capping the scale at 256 times a power-of-two median keeps the
    in-band chi^2 values at full FP8 resolution and saturates the rare outliers.
    """
    P = np.asarray(P, dtype=np.float64)
    if dtype == "f32":
        return P.astype(np.float32).astype(np.float64), None
    if dtype == "bf16":
        return round_bf16(P), None
    if dtype == "f16":
        return round_f16(P), None
    if dtype == "f8e4m3":
        M = np.array([f8_row_reference(row) for row in P])
        s = np.where(M > 0, M / F8_E4M3_MAX, 1.0).astype(np.float32)
        q = round_f8e4m3(P / s.astype(np.float64)[:, None])
        # dequantisation is defined as the FP32 product q * s (q is exact in FP32)
        deq = (q.astype(np.float32) * s[:, None]).astype(np.float64)
        return deq, s
    raise ValueError(dtype)


# --------------------------------------------------------------------------
# SVD basis (Sec. II.C: f_{i,alpha} = sum_p U_{i,p} S_p V_{p,alpha})
# --------------------------------------------------------------------------
def svd_basis(F, K: int = 0, tol: float = 1e-7):
    """Uncentred thin SVD of the training tracks F [M, n_seg] (Hz at t_alpha).

    Returns (V_K [K, n_seg] with orthonormal rows, sigma [K], cmin [K], cmax [K])
    where the coefficients of the training tracks are C = F V_K^T and the
    candidate box is their per-coefficient min/max.  K = 0 picks the smallest
    K whose worst training-track relative reconstruction error
    max_alpha |F - C V_K| / max_alpha |F| is <= tol.  Signs are fixed so that
    the entry of largest magnitude in each row of V_K is positive.
    """
    F = np.asarray(F, dtype=np.float64)
    _, s, Vt = np.linalg.svd(F, full_matrices=False)
    if K <= 0:
        K = Vt.shape[0]
        fmax = np.max(np.abs(F), axis=1)
        for k in range(1, Vt.shape[0] + 1):
            R = F - (F @ Vt[:k].T) @ Vt[:k]
            if np.max(np.max(np.abs(R), axis=1) / fmax) <= tol:
                K = k
                break
    V = Vt[:K].copy()
    for k in range(K):
        j = int(np.argmax(np.abs(V[k])))
        if V[k, j] < 0:
            V[k] = -V[k]
    C = F @ V.T
    return V, s[:K].copy(), C.min(axis=0), C.max(axis=0)


def reconstruction_error(F, V):
    """Per-track relative error max_alpha |F - F V^T V| / max_alpha |F|."""
    F = np.asarray(F, dtype=np.float64)
    R = F - (F @ V.T) @ V
    return np.max(np.abs(R), axis=1) / np.max(np.abs(F), axis=1)


# --------------------------------------------------------------------------
# Track -> bin (Sec. II.C: f_alpha = sum_p xi_p V_{p,alpha}, plus an offset f_ref)
# --------------------------------------------------------------------------
def track_x(V, coeffs, f_ref, T_sft: float):
    """x_{t,alpha} = (f_ref[t] + sum_k c[t,k] V[k,alpha]) * T_SFT in FP64.

    The sum runs k = 0..K-1 left to right, each product and sum rounded
    separately (no fused multiply-add), then the frequency is scaled by T_SFT.
    """
    V = np.asarray(V, dtype=np.float64)
    c = np.asarray(coeffs, dtype=np.float64)
    f = np.array(np.asarray(f_ref, dtype=np.float64)[:, None] * np.ones((1, V.shape[1])))
    for k in range(V.shape[0]):
        f = f + c[:, k : k + 1] * V[k][None, :]
    return f * T_sft


def bins_and_ties(x):
    """Reading: bin k is centred at k / T_SFT, so b = floor(x + 1/2); a tie is
    |x - floor(x) - 1/2| <= 1e-9.  A non-finite x maps to no bin (returned as
    a huge sentinel that lies outside every table) and is never a tie."""
    x = np.asarray(x, dtype=np.float64)
    fin = np.isfinite(x)
    xs = np.where(fin, x, 0.0)
    z = np.floor(xs + 0.5)
    big = 2.0 ** 62
    b = np.where(fin, np.clip(z, -big, big), big).astype(np.int64)
    tie = fin & (np.abs(xs - np.floor(xs) - 0.5) <= TIE_BAND)
    return b, tie


# --------------------------------------------------------------------------
# The statistic (Sec. II.B, Eq. det_stat, nearest-bin reading with +-m neighbours)
# --------------------------------------------------------------------------
def statistic(P, b, m: int):
    """S[t] = sum_alpha sum_{j=-m..m} P[alpha, b[t,alpha] + j] in FP64; a bin
    outside [0, n_bin) contributes 0 (no clamping)."""
    P = np.asarray(P, dtype=np.float64)
    n_seg, n_bin = P.shape
    b = np.asarray(b, dtype=np.int64)
    S = np.zeros(b.shape[0], dtype=np.float64)
    rows = np.arange(n_seg)[None, :]
    for j in range(-m, m + 1):
        idx = b + j
        ok = (idx >= 0) & (idx < n_bin)
        vals = P[rows, np.where(ok, idx, 0)]
        S += np.sum(np.where(ok, vals, 0.0), axis=1)
    return S


def statistic_loop(P, b, m: int):
    """The same sum written as plain Python loops (small cases only)."""
    n_seg, n_bin = len(P), len(P[0])
    out = []
    for row in b:
        s = 0.0
        for a in range(n_seg):
            for j in range(-m, m + 1):
                k = int(row[a]) + j
                if 0 <= k < n_bin:
                    s += float(P[a][k])
        out.append(s)
    return np.array(out)


# --------------------------------------------------------------------------
# Segment exclusions (Sec. II.B validity cut on the second-order evolution;
# Sec. II.D low-frequency and low-derivative exclusions)
# --------------------------------------------------------------------------
F_LOW_HZ = 10.0 ** -3.5    # frequencies below this contribute nothing (Sec. II.D)
FDOT_LOW = 1e-13           # nor do frequency derivatives below this (Hz/s)


def track_freqs(V, coeffs, f_ref):
    """f_{t,alpha} = f_ref[t] + sum_k c[t,k] V[k,alpha] in FP64, the sum left to right with
    each product and sum rounded separately (the order of ``track_x`` before the T_SFT factor)."""
    V = np.asarray(V, dtype=np.float64)
    c = np.asarray(coeffs, dtype=np.float64)
    f = np.array(np.asarray(f_ref, dtype=np.float64)[:, None] * np.ones((1, V.shape[1])))
    for k in range(V.shape[0]):
        f = f + c[:, k : k + 1] * V[k][None, :]
    return f


def finite_differences(F, T_sft: float):
    """(fdot, z) [t, alpha] of the tracks F [t, alpha] (Hz at the segment midpoints).

    Readings: the derivatives come from finite differences of the track at the segment
    midpoints (the paper takes them from the track, by numerical differentiation):
    fdot_alpha = (f_{alpha+1} - f_{alpha-1}) / (2 T_SFT) inside, (f_1 - f_0) / T_SFT and
    (f_{n-1} - f_{n-2}) / T_SFT at the ends, 0 for one segment; the second-order term
    z_alpha = fddot_alpha T_SFT^3 / 6 = ((f_{alpha+1} - 2 f_alpha) + f_{alpha-1}) (T_SFT / 6)
    inside, the nearest inner value at the ends, 0 for fewer than three segments.  Every
    step is one IEEE FP64 operation in the order written."""
    F = np.asarray(F, dtype=np.float64)
    N, n = F.shape
    T = float(T_sft)
    fd = np.zeros_like(F)
    z = np.zeros_like(F)
    if n >= 2:
        fd[:, 1:-1] = (F[:, 2:] - F[:, :-2]) / (2.0 * T)
        fd[:, 0] = (F[:, 1] - F[:, 0]) / T
        fd[:, -1] = (F[:, -1] - F[:, -2]) / T
    if n >= 3:
        z[:, 1:-1] = ((F[:, 2:] - 2.0 * F[:, 1:-1]) + F[:, :-2]) * (T / 6.0)
        z[:, 0] = z[:, 1]
        z[:, -1] = z[:, -2]
    return fd, z


def segment_validity(F, T_sft: float):
    """valid[t, alpha]: False where a segment contributes nothing: z > 1, or f < 10^-3.5 Hz,
    or fdot < 1e-13 Hz/s (either low condition suffices), with fdot and z from
    ``finite_differences``."""
    F = np.asarray(F, dtype=np.float64)
    fd, z = finite_differences(F, T_sft)
    return ~((z > 1.0) | (F < F_LOW_HZ) | (fd < FDOT_LOW))


def statistic_masked(P, b, valid, m: int):
    """The statistic with excluded segments contributing 0."""
    P = np.asarray(P, dtype=np.float64)
    n_seg, n_bin = P.shape
    b = np.asarray(b, dtype=np.int64)
    S = np.zeros(b.shape[0], dtype=np.float64)
    rows = np.arange(n_seg)[None, :]
    for j in range(-m, m + 1):
        idx = b + j
        ok = (idx >= 0) & (idx < n_bin) & valid
        vals = P[rows, np.where((idx >= 0) & (idx < n_bin), idx, 0)]
        S += np.sum(np.where(ok, vals, 0.0), axis=1)
    return S


def eval_stat_masked(P, V, coeffs, f_ref, T_sft: float, m: int, chunk: int = 4096):
    """S [N] (FP64) with the segment exclusions, and the validity mask."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    N = coeffs.shape[0]
    S = np.empty(N)
    valid_all = np.empty((N, np.asarray(V).shape[1]), dtype=bool)
    for s0 in range(0, N, chunk):
        s1 = min(N, s0 + chunk)
        F = track_freqs(V, coeffs[s0:s1], f_ref[s0:s1])
        valid = segment_validity(F, T_sft)
        b, _ = bins_and_ties(F * T_sft)
        S[s0:s1] = statistic_masked(P, b, valid, m)
        valid_all[s0:s1] = valid
    return S, valid_all


# --------------------------------------------------------------------------
# The linear-chirp statistic (Sec. II.B: S_alpha of Eq. det_stat with the
# chirping local template, its SFT over the 2P + 1 bins around the track)
# --------------------------------------------------------------------------
CHIRP_P = 100   # the paper's band: 2P + 1 = 201 bins (Sec. II.B)


def chirp_template_sft(f, fdot, T_sft: float, dt: float, bins, window_kind: str = "hann"):
    """h~_k for each listed bin k: the SFT (the window, sampling and DFT of ``sft``) of the
    segment's local waveform exp(i [2 pi f (t - t_a) + pi fdot (t - t_a)^2]), the chirping
    sinusoid of Sec. II.B with unit amplitude and zero phase; t runs over the segment's
    samples t = n dt from its start and t_a = T_SFT / 2 is its midpoint.  f, fdot: [N];
    bins: [N, B] integers in [0, L); returns [N, B] complex."""
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    fdot = np.asarray(fdot, dtype=np.float64).reshape(-1)
    L = int(round(T_sft / dt))
    u = np.arange(L, dtype=np.float64) * dt - 0.5 * T_sft
    w = window(L, window_kind)
    phase = 2.0 * np.pi * f[:, None] * u[None, :] + np.pi * fdot[:, None] * (u * u)[None, :]
    H = dt * np.fft.fft(w[None, :] * np.exp(1j * phase), axis=1)
    return np.take_along_axis(H, np.asarray(bins, dtype=np.int64) % L, axis=1)


def chirp_statistic(d, psd_bins, dt: float, T_sft: float, F, P: int = CHIRP_P, valid=None,
                    window_kind: str = "hann"):
    """S [t] = sum_alpha S_alpha (FP64) with the linear-chirp S_alpha of Eq. det_stat:

        S_alpha = 4 / (dt sum w^2) |sum_k d~*_{alpha,k} h~_{alpha,k} / S_k|^2 / sum_k |h~_{alpha,k}|^2 / S_k

    (the maximised inner product 4 |sum d~* h~ / S_n| Delta f squared over <h|h>, with
    Delta f = 1 / T_SFT generalised for the window as in ``power_table``), h~ from
    ``chirp_template_sft`` at f_alpha = F[t, alpha] and fdot_alpha from
    ``finite_differences``.  Readings: the sum runs over the 2P + 1 bins k = b - P .. b + P
    around the nearest bin b = floor(f_alpha T_SFT + 1/2) that lie in the table, skipping the
    DC bin and bins whose S_n is not finite and positive; S_alpha = 0 when the track's own
    bin b lies outside the table (its frequency is outside the data's band: only the far
    tails of the template would remain), when no bin is left, and where valid[t, alpha] is
    False.  d: the complex SFTs [n_seg, n_bin] of ``sft``."""
    d = np.asarray(d, dtype=np.complex128)
    n_seg, n_bin = d.shape
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[0]
    L = int(round(T_sft / dt))
    w = window(L, window_kind)
    norm = 4.0 / (dt * float(np.sum(w * w)))
    S = np.asarray(psd_bins, dtype=np.float64)
    ok = np.isfinite(S) & (S > 0)
    ok[0] = False
    inv_S = np.where(ok, 1.0 / np.where(ok, S, 1.0), 0.0)
    fd, _ = finite_differences(F, T_sft)
    b, _ = bins_and_ties(F * T_sft)
    j = np.arange(-P, P + 1, dtype=np.int64)
    total = np.zeros(N)
    for a in range(n_seg):
        k = b[:, a][:, None] + j[None, :]                     # [N, 2P+1]
        inside = (k >= 0) & (k < n_bin)
        kk = np.where(inside, k, 0)
        wgt = np.where(inside, inv_S[kk], 0.0)
        h = chirp_template_sft(F[:, a], fd[:, a], T_sft, dt, kk, window_kind)
        num = np.abs(np.sum(np.conj(d[a, kk]) * h * wgt, axis=1)) ** 2
        den = np.sum((h.real ** 2 + h.imag ** 2) * wgt, axis=1)
        Sa = np.where(den > 0, norm * num / np.where(den > 0, den, 1.0), 0.0)
        Sa = np.where((b[:, a] >= 0) & (b[:, a] < n_bin), Sa, 0.0)
        if valid is not None:
            Sa = np.where(valid[:, a], Sa, 0.0)
        total += Sa
    return total


# --------------------------------------------------------------------------
# The plunge-time search over data chunks of growing duration (Sec. II.D)
# --------------------------------------------------------------------------
JULIAN_YEAR_S = 365.25 * 86400.0


def chunk_layout(n_seg: int, T_sft: float, t_min: float = 0.1 * JULIAN_YEAR_S, step: int = 12,
                 n_chunks: int = 48):
    """Segments n_obs of each data chunk: the paper starts at 0.1 yr and adds about 7 days
    (12 SFTs) per chunk, 48 chunks.  Reading: n_obs(c) = floor(t_min / T_SFT) + step c for
    c = 0 .. n_chunks - 1, a Julian year, chunks longer than the data dropped."""
    n0 = int(math.floor(t_min / T_sft))
    return [n0 + step * c for c in range(n_chunks) if 1 <= n0 + step * c <= n_seg]


def chunk_eval(P, V, coeffs_list, f_ref_list, n_obs_list, T_sft: float, m: int):
    """Per chunk c: the statistic (FP64) of its tracks on the data's first n_obs segments,
    with the basis shifted by an integer number of segments so that its plunge (its last
    segment) falls at the chunk's end: basis columns n_seg - n_obs .. n_seg - 1."""
    P = np.asarray(P, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    n_seg = V.shape[1]
    out = []
    for c, f, n in zip(coeffs_list, f_ref_list, n_obs_list):
        S, *_ = eval_stat(P[:n], V[:, n_seg - n:], c, f, T_sft, m, 0)
        out.append(S)
    return out


def noise_moments(n_a: int, m: int, window_kind: str = "hann"):
    """(mean, standard deviation) of the nearest-bin statistic over n_a segments of
    Gaussian noise, the closed form behind the paper's per-duration normalisation
    (Sec. II.D normalises by the noise mean and standard deviation of each duration).
    Each P is chi^2_2 (mean 2, variance 4); two bins of one segment covary by
    4 |rho_d|^2 with rho_d the window's bin correlation at distance d (periodic Hann:
    |rho_1|^2 = 4/9, |rho_2|^2 = 1/36, none beyond; rectangular: none); segments are
    independent.  Windows that leave the table are not accounted for."""
    rho2 = {1: 4.0 / 9.0, 2: 1.0 / 36.0} if window_kind == "hann" else {}
    W = 2 * m + 1
    var_seg = 4.0 * (W + 2.0 * sum((W - d) * rho2.get(d, 0.0) for d in range(1, W)))
    return 2.0 * W * n_a, math.sqrt(var_seg * n_a)


# --------------------------------------------------------------------------
# Top-k (Sec. II.D keeps the highest-scoring half of the population)
# --------------------------------------------------------------------------
def topk(S, k: int):
    """The k largest S by a stable sort on (-S, index): equal values keep the
    lower index first, -0.0 equals +0.0 and NaN ranks below every number."""
    S = np.asarray(S, dtype=np.float64)
    k = min(int(k), S.size)
    nan = np.isnan(S)
    key = np.where(nan, 0.0, -S) + 0.0   # + 0.0 turns -0.0 into +0.0
    order = np.lexsort((np.arange(S.size), key, nan))
    idx = order[:k]
    return idx.astype(np.int64), S[idx]


# --------------------------------------------------------------------------
# The whole statistic call
# --------------------------------------------------------------------------
def eval_stat(P, V, coeffs, f_ref, T_sft: float, m: int, k: int = 0, chunk: int = 4096):
    """S [N] (FP64), top-k (idx, val) and the list of tie (t, alpha) pairs."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    N = coeffs.shape[0]
    S = np.empty(N)
    ties = []
    for s0 in range(0, N, chunk):
        s1 = min(N, s0 + chunk)
        x = track_x(V, coeffs[s0:s1], f_ref[s0:s1], T_sft)
        b, tie = bins_and_ties(x)
        S[s0:s1] = statistic(P, b, m)
        tt, aa = np.nonzero(tie)
        ties.extend(zip((tt + s0).tolist(), aa.tolist()))
    idx, val = topk(S, k) if k > 0 else (np.zeros(0, np.int64), np.zeros(0))
    return S, idx, val, ties


def stat_relative_error(S_test, S_ref):
    """max_t |S_test - S_ref| / |S_ref| (|S_ref| = 0 compares absolutely)."""
    S_test = np.asarray(S_test, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    den = np.where(S_ref != 0, np.abs(S_ref), 1.0)
    return float(np.max(np.abs(S_test - S_ref) / den)) if S_ref.size else 0.0
