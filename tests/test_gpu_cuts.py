"""Segment exclusions (tfs_job flag TFS_JOB_SEGMENT_CUTS) against the FP64 oracle.

A segment of a track contributes nothing when its second-order term
fddot T_SFT^3 / 6 exceeds 1 (Sec. II.B), or its frequency lies below
10^-3.5 Hz or its frequency derivative below 1e-13 Hz/s (Sec. II.D), the
derivatives taken by finite differences of the track at the segment midpoints.
The kernel decides each exclusion in FP32 with a rigorous margin and leaves the
close calls to FP64 in the oracle's operation order, so the statistic equals
the oracle's masked statistic within FP32 rounding of the sum (relative 1e-5):
one wrong exclusion moves it by a whole window sum, far more than that.

Tracks: power-law chirps f0 (1 - t / tau)^-p whose plunge (tau) falls just
after the data, so that the last segments break the second-order test, with
f0 reaching below the low-frequency threshold; half of them projected on the
basis, half drawn uniformly from the coefficient box (wiggly tracks whose
derivative changes sign); and tracks scaled or shifted so that one segment sits
on a threshold to within a few ulps.
"""
import numpy as np
import pytest

import oracle.tfstat_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as pkg

    return pkg


def _derivs(F, Tsft):
    """Central-difference fdot and the second-order term, only to place tracks on a threshold."""
    fd = np.zeros_like(F)
    z = np.zeros_like(F)
    n = F.shape[1]
    if n >= 2:
        fd[:, 1:-1] = (F[:, 2:] - F[:, :-2]) / (2 * Tsft)
        fd[:, 0] = (F[:, 1] - F[:, 0]) / Tsft
        fd[:, -1] = (F[:, -1] - F[:, -2]) / Tsft
    if n >= 3:
        z[:, 1:-1] = (F[:, 2:] - 2 * F[:, 1:-1] + F[:, :-2]) * (Tsft / 6)
        z[:, 0], z[:, -1] = z[:, 1], z[:, -2]
    return fd, z


def _plunge_case(rng, n_seg, Tsft, K, N, n_near, f0=(5e-5, 3e-3), tau=(1.0003, 3.0)):
    """Basis [K][n_seg], coefficients [N'][K], f_ref [N'] (N' = N + 3 n_near); f0 in Hz, tau in
    units of the observation's duration."""
    t = (np.arange(n_seg) + 0.5) * Tsft
    D = n_seg * Tsft

    def tracks(M):
        fa = rng.uniform(*f0, M)
        ta = D * rng.uniform(*tau, M)
        p = rng.uniform(0.25, 0.4, M)
        return fa[:, None] * (1.0 - t[None, :] / ta[:, None]) ** (-p[:, None])

    _, _, Vt = np.linalg.svd(tracks(600), full_matrices=False)
    V = Vt[:K].copy()
    c_proj = tracks(N - N // 2) @ V.T
    lo, hi = c_proj.min(axis=0), c_proj.max(axis=0)
    c_box = lo + (hi - lo) * rng.uniform(0, 1, (N // 2, K))
    c = np.concatenate([c_proj, c_box])
    f = np.zeros(N)
    # on a threshold: one segment's f at 10^-3.5 Hz, fdot at 1e-13 Hz/s, or z at 1
    src = c_proj[rng.integers(0, c_proj.shape[0], 3 * n_near)]
    F0 = O.track_freqs(V, src, np.zeros(src.shape[0]))
    fd, z = _derivs(F0, Tsft)
    a = rng.integers(1, max(2, n_seg - 1), 3 * n_near) % n_seg
    rows = np.arange(3 * n_near)
    near_c, near_f = src.copy(), np.zeros(3 * n_near)
    s0, s1 = slice(0, n_near), slice(n_near, 2 * n_near)
    s2 = slice(2 * n_near, 3 * n_near)
    near_f[s0] = O.F_LOW_HZ - F0[rows[s0], a[s0]]
    scale = np.where(fd[rows[s1], a[s1]] > 0, O.FDOT_LOW / np.where(fd[rows[s1], a[s1]] > 0, fd[rows[s1], a[s1]], 1), 1)
    near_c[s1] *= scale[:, None]
    zz = z[rows[s2], a[s2]]
    near_c[s2] *= np.where(zz > 0, 1.0 / np.where(zz > 0, zz, 1), 1)[:, None]
    return V, np.concatenate([c, near_c]), np.concatenate([f, near_f])


def _power(rng, n_seg, n_bin):
    P = rng.exponential(2.0, (n_seg, n_bin))
    P[:, :3] = 0.0
    return P


def _run(T, torch, specs, seed):
    """One eval_batch call over every spec, each job twice: with and without the cuts."""
    rng = np.random.default_rng(seed)
    cases, jobs = [], []
    for (dtype, n_seg, n_bin, Tsft, K, N, m, n_near, *kw) in specs:
        V, c, f = _plunge_case(rng, n_seg, Tsft, K, N, n_near, **(kw[0] if kw else {}))
        P = _power(rng, n_seg, n_bin)
        table = T.table_from_power(P, Tsft, dtype)
        basis = T.basis_from_host(V)
        dc = torch.tensor(c, device="cuda")
        df = torch.tensor(f, device="cuda")
        cases.append(dict(V=V, c=c, f=f, table=table, Tsft=Tsft, m=m))
        for cut in (True, False):
            jobs.append(T.Job(table, basis, dc, df, m=m, segment_cuts=cut))
    order = rng.permutation(len(jobs))  # cut and plain jobs interleaved in the batch
    T.eval_batch([jobs[i] for i in order])
    torch.cuda.synchronize()
    return cases, jobs


def _check(cases, jobs):
    why = np.zeros(3, dtype=np.int64)
    for i, d in enumerate(cases):
        Pq, _ = d["table"].to_host()
        S_cut, valid = O.eval_stat_masked(Pq, d["V"], d["c"], d["f"], d["Tsft"], d["m"])
        S_all, *_ = O.eval_stat(Pq, d["V"], d["c"], d["f"], d["Tsft"], d["m"], 0)
        got_cut = jobs[2 * i].stat.cpu().numpy().astype(np.float64)
        got_all = jobs[2 * i + 1].stat.cpu().numpy().astype(np.float64)
        assert O.stat_relative_error(got_cut, S_cut) <= 1e-5, i
        assert O.stat_relative_error(got_all, S_all) <= 1e-5, i
        F = O.track_freqs(d["V"], d["c"], d["f"])
        fd, z = _derivs(F, d["Tsft"])
        why += [(z > 1).sum(), (F < O.F_LOW_HZ).sum(), (fd < O.FDOT_LOW).sum()]
        if valid.shape[1] >= 10:
            assert 0.02 < 1 - valid.mean() < 0.98, (i, valid.mean())  # the cuts change the statistic
    return why


def test_segment_cuts_equal_the_masked_oracle(T):
    torch = pytest.importorskip("torch")
    specs = [
        # dtype, n_seg, n_bin, Tsft,  K, N,    m, near
        ("f32", 120, 2000, 5.0e4, 6, 3000, 1, 100),
        ("f32", 120, 2000, 5.0e4, 3, 2000, 0, 60),
        ("f32", 90, 1500, 5.0e4, 8, 2000, 2, 60),
        ("f32", 60, 2500, 5.0e4, 13, 1500, 1, 40),
        ("f32", 64, 2500, 5.0e4, 20, 1000, 3, 40),
        ("bf16", 100, 2000, 5.0e4, 6, 2000, 1, 60),
        ("f16", 80, 1800, 5.0e4, 4, 1500, 2, 40),
        ("f8e4m3", 120, 2000, 5.0e4, 6, 1500, 1, 40),
        # narrow families: every tile's band fits the staged slot (the complete-band path)
        ("f32", 120, 600, 5.0e4, 6, 3000, 1, 60, dict(f0=(2.5e-4, 4e-4), tau=(1.0003, 1.01))),
        ("bf16", 90, 600, 5.0e4, 8, 2000, 2, 40, dict(f0=(2.8e-4, 3.6e-4), tau=(1.0003, 1.02))),
        ("f32", 60, 600, 5.0e4, 13, 1500, 0, 40, dict(f0=(2.5e-4, 4e-4), tau=(1.0003, 1.01))),
    ]
    cases, jobs = _run(T, torch, specs, seed=11)
    why = _check(cases, jobs)
    assert (why > 0).all(), why  # every rule excludes something


def test_segment_cuts_short_and_wide(T):
    """One segment (fdot = 0: everything excluded), two segments (no second-order term),
    a long observation, and a band wider than the staged slot."""
    torch = pytest.importorskip("torch")
    specs = [
        ("f32", 2, 600, 5.0e4, 2, 500, 1, 10),
        ("f32", 3, 600, 5.0e4, 3, 500, 0, 10),
        ("f32", 631, 1200, 5.0e4, 6, 1200, 1, 30),
        ("f32", 40, 40000, 5.0e4, 5, 800, 2, 20, dict(f0=(5e-4, 3e-2))),
    ]
    cases, jobs = _run(T, torch, specs, seed=12)
    _check(cases, jobs)
    rng = np.random.default_rng(13)
    P = _power(rng, 1, 500)
    table = T.table_from_power(P, 5.0e4, "f32")
    V = np.ones((1, 1))
    c = rng.uniform(0.0, 500 / 5.0e4, (300, 1))
    job = T.Job(table, T.basis_from_host(V), torch.tensor(c, device="cuda"), None, m=1, segment_cuts=True)
    T.eval_batch([job])
    torch.cuda.synchronize()
    assert (job.stat.cpu().numpy() == 0).all()


def test_segment_cuts_full_size_sampled(T):
    """Ten million one-year tracks with the exclusions, in the benchmark's launch configuration
    (`bench.py --segment-cuts`); 4000 sampled tracks and the top 32 against the masked oracle."""
    torch = pytest.importorskip("torch")
    from paper_2510_20891_gb300 import synth

    w = synth.WORKLOADS["oneyear_daily_fp32"]
    rng = np.random.default_rng(0)
    x, _ = synth.make_strain(w, rng)
    psd = synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft)
    P64 = O.power_table(x, w.dt, w.T_sft, psd)
    V, s, lo, hi = O.svd_basis(synth.make_training_tracks(w, rng), w.K)
    N = w.n_tracks
    coeffs = synth.uniform_coeffs(N, lo, hi, np.random.default_rng(8))
    table = T.table_from_power(P64, w.T_sft, "f32")
    job = T.Job(table, T.basis_from_host(V), torch.from_numpy(coeffs).cuda(), None, m=1, topk=32,
                segment_cuts=True)
    T.eval_batch([job])
    torch.cuda.synchronize()
    stat = job.stat.cpu().numpy().astype(np.float64)
    sample = np.random.default_rng(9).choice(N, 4000, replace=False)
    S, valid = O.eval_stat_masked(P64, V, coeffs[sample], np.zeros(sample.size), w.T_sft, 1)
    assert O.stat_relative_error(stat[sample], S) <= 1e-5
    assert 0 < 1 - valid.mean() < 0.5
    gi, _ = O.topk(stat, 32)
    assert np.array_equal(job.top_idx.cpu().numpy(), gi)
    St, _ = O.eval_stat_masked(P64, V, coeffs[gi], np.zeros(gi.size), w.T_sft, 1)
    assert O.stat_relative_error(job.top_val.cpu().numpy().astype(np.float64), St) <= 1e-5
