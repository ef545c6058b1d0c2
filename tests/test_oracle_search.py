"""Pins of the oracle's plunge-time search (Sec. II.D): the chunk layout against the values
the paper prints, a chunk against the power table of the strain's first segments with the
year's tracks cut to their last segments, and the closed-form noise moments that normalise
each duration against Monte Carlo over noise tables (and the hand values at m = 0 and 1).
"""
import numpy as np
import pytest

import oracle.tfstat_oracle as O


def _golden(name):
    import os

    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_chunk_layout_matches_the_paper():
    g = _golden("paper_chunk_search.txt")
    T = g["T_sft_s"]
    n_year = int(np.floor(O.JULIAN_YEAR_S / T))          # 631 (pinned in paper_segment_counts.txt)
    lay = O.chunk_layout(n_year, T, t_min=g["t_min_yr"] * O.JULIAN_YEAR_S, step=int(g["step_sfts"]),
                         n_chunks=int(g["n_chunks"]))
    assert len(lay) == g["n_chunks"]                     # all 48 chunks fit in the year
    assert lay[0] * T <= g["t_min_yr"] * O.JULIAN_YEAR_S < (lay[0] + 1) * T
    steps = np.diff(lay) * T / 86400.0
    assert np.all(np.abs(steps - g["step_days_approx"]) < 0.1)
    assert lay[-1] <= n_year


def test_chunk_eval_is_the_data_prefix_with_the_shifted_basis():
    """A chunk's table equals the power table of the strain's first n_obs segments, and a
    chunk track equals the last n_obs values of the year's track."""
    rng = np.random.default_rng(7)
    dt, L, n_seg = 1.0, 64, 20
    T = L * dt
    x = rng.standard_normal(L * n_seg)
    psd = np.full(L // 2 + 1, 2.0)
    P = O.power_table(x, dt, T, psd)
    V = np.linalg.qr(rng.standard_normal((n_seg, 3)))[0].T
    c = rng.uniform(-1, 1, (30, 3)) * 20 / T
    f = rng.uniform(5, 25, 30) / T
    for n in (1, 7, 20):
        got = O.chunk_eval(P, V, [c], [f], [n], T, 1)[0]
        Pn = O.power_table(x[: n * L], dt, T, psd)
        Fyear = O.track_freqs(V, c, f)
        b, _ = O.bins_and_ties(Fyear[:, n_seg - n:] * T)
        assert np.allclose(got, O.statistic(Pn, b, 1), rtol=1e-13)


@pytest.mark.parametrize("window_kind", ["hann", "rect"])
def test_noise_moments_against_monte_carlo(window_kind):
    rng = np.random.default_rng(8)
    L, n_seg, Nb = 256, 12, 129
    S = {0: [], 1: [], 2: []}
    for _ in range(300):
        x = rng.standard_normal(L * n_seg)
        P = O.power_table(x, 1.0, float(L), np.full(Nb, 2.0), window_kind=window_kind)
        b = rng.integers(6, Nb - 6, size=(30, n_seg))
        for m in S:
            S[m].append(O.statistic(P, b, m))
    for m in S:
        v = np.concatenate(S[m])
        mu, sd = O.noise_moments(n_seg, m, window_kind)
        assert abs(v.mean() - mu) < 5 * sd / np.sqrt(v.size)
        assert abs(v.std() / sd - 1) < 0.06
    # the hand values at m = 0 and 1 (Hann): variance 4 and 19.333 per segment
    assert np.isclose(O.noise_moments(1, 0)[1] ** 2, 4.0)
    assert np.isclose(O.noise_moments(1, 1)[1] ** 2, 19.0 + 1.0 / 3.0)


def test_splitmix64_published_values():
    """The search's device draws come from SplitMix64; its host definition gives the published
    outputs for seed 1234567: 6457827717110365317, 3203168211198807973, 9817491932198370423
    (Rosetta Code, "Pseudo-random numbers/Splitmix64")."""
    from tests.splitmix import splitmix64_at

    got = [int(x) for x in splitmix64_at(1234567, np.arange(1, 4, dtype=np.uint64))]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_de_draws_are_valid_partners():
    """Every walker's partners are two distinct other walkers of its own chunk; the offsets are
    uniform over the W - 1 others (chi-square over many draws); F lies in [0.3, 1.5)."""
    from tests.splitmix import de_draws

    n_ch, W = 6, 17
    r1s, r2s = [], []
    for it in range(400):
        r1, r2, F = de_draws(99, it, n_ch, W, 0.3, 1.5)
        g = np.arange(n_ch * W)
        assert np.all(r1 // W == g // W) and np.all(r2 // W == g // W)
        assert np.all(r1 != g) and np.all(r2 != g) and np.all(r1 != r2)
        assert F.dtype == np.float32 and np.all(F >= np.float32(0.3)) and np.all(F < np.float32(1.5))
        r1s.append((r1 - g) % W)
        r2s.append((r2 - g) % W)
    for off in (np.concatenate(r1s), np.concatenate(r2s)):
        counts = np.bincount(off, minlength=W)[1:]
        e = off.size / (W - 1)
        chi2 = float(np.sum((counts - e) ** 2 / e))
        assert counts.size == W - 1 and chi2 < 60.0   # 16 degrees of freedom: p ~ 1e-6 at 60
