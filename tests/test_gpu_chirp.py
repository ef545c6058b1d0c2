"""The paper's linear-chirp statistic on the GPU (tfs_build_chirp_table, tfs_eval_chirp_stat)
against the FP64 oracle (``chirp_statistic``: the template's SFT as the L-point DFT of the
sampled Hann-windowed chirp, every sum in FP64).

The GPU evaluates the template as the Fourier integral of the windowed chirp at 256
points (aliasing below about 1e-7 of the template's peak for the drifts tested here, up to
60 bins per segment), the data bins in FP32 and the sums in
FP32 per segment, so the statistic agrees with the oracle within 2e-5 relative per track
(max over tracks), stated here; the bins are the oracle's FP64 bins (made observable with
P = 0 and tracks exactly on half-integer x).
"""
import numpy as np
import pytest

import oracle.tfstat_oracle as O

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as pkg

    return pkg


def _strain(rng, n_seg, L, dt, chirp=None, colored=False):
    n = n_seg * L
    x = rng.standard_normal(n)
    nb = L // 2 + 1
    psd = np.full(nb, 2.0 * dt)
    if colored:
        # red noise below 0.05 Hz (levelled off below 0.01 Hz), the same law for the strain
        shape_of = lambda f: 1.0 + (0.05 / np.maximum(f, 0.01)) ** 2
        psd = psd * shape_of(np.arange(nb) / (L * dt))
        X = np.fft.rfft(x) * np.sqrt(shape_of(np.arange(n // 2 + 1) / (n * dt)))
        x = np.fft.irfft(X, n)
    if chirp is not None:
        f0, fdot, A = chirp
        t = np.arange(n) * dt
        x = x + A * np.cos(2 * np.pi * (f0 * t + 0.5 * fdot * t * t))
    return x, psd


def _basis(n_seg, K):
    t = np.linspace(-1, 1, n_seg)
    return np.linalg.qr(np.vander(t, K, increasing=True))[0].T.copy()


def _tracks(rng, V, N, n_bin, Tsft, beta_max):
    """Coefficients whose tracks span the band with drifts up to beta_max bins per segment."""
    K, n_seg = V.shape
    f = rng.uniform(-0.05, 1.05, N) * n_bin / Tsft
    c = np.zeros((N, K))
    c[:, 0] = f / V[0, 0]                          # constant basis row
    if K > 1:
        slope = rng.uniform(-beta_max, beta_max, N) / Tsft ** 2   # fdot
        c[:, 1] = slope * Tsft / (V[1, 1] - V[1, 0])
    if K > 2:
        c[:, 2:] = rng.standard_normal((N, K - 2)) * 0.3 / Tsft
    return c


def _run(T, torch, table, basis, c, f=None, P=100, cuts=False, topk=0):
    dc = torch.tensor(c, device="cuda")
    df = torch.tensor(f, device="cuda") if f is not None else None
    stat, ti, tv = T.eval_chirp_stat(table, basis, dc, df, P=P, segment_cuts=cuts, topk=topk)
    torch.cuda.synchronize()
    return stat.cpu().numpy().astype(np.float64), ti, tv


def test_chirp_table_matches_oracle(T):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    dt, L, n_seg = 1.0, 1024, 6
    x, psd = _strain(rng, n_seg, L, dt, colored=True)
    psd[7] = np.inf
    ct = T.build_chirp_table(x, dt, L * dt, psd)
    z, wt = ct.to_host()
    d = O.sft(x, dt, L * dt)
    w = O.window(L)
    ok = np.isfinite(psd) & (psd > 0)
    ok[0] = False
    s_ref = ct.s_ref
    assert s_ref == np.sort(psd[ok])[ok.sum() // 2]  # the median usable S_n (upper middle)
    want = np.sqrt(4.0 / (dt * np.sum(w * w) * s_ref)) * d * np.where(ok, s_ref / np.where(ok, psd, 1), 0)[None, :]
    assert np.max(np.abs(z - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.allclose(wt, np.where(ok, s_ref / np.where(ok, psd, 1), 0), rtol=1e-7)
    assert z[:, 0].tolist() == [0j] * n_seg and np.all(z[:, 7] == 0)


@pytest.mark.parametrize("K,P,cuts,colored", [(3, 100, False, False), (6, 100, True, True), (2, 20, False, True),
                                              (4, 111, False, False)])
def test_chirp_statistic_matches_oracle(T, K, P, cuts, colored):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10 + K + P)
    dt, L, n_seg = 2.0, 1024, 10
    Tsft = L * dt
    n_bin = L // 2 + 1
    x, psd = _strain(rng, n_seg, L, dt, chirp=(150.3 / Tsft, 4.0 / Tsft ** 2, 0.3), colored=colored)
    V = _basis(n_seg, K)
    c = _tracks(rng, V, 700, n_bin, Tsft, 60.0)
    f = rng.uniform(-2, 2, 700) / Tsft
    ct = T.build_chirp_table(x, dt, Tsft, psd)
    got, *_ = _run(T, torch, ct, T.basis_from_host(V), c, f, P=P, cuts=cuts)
    F = O.track_freqs(V, c, f)
    valid = O.segment_validity(F, Tsft) if cuts else None
    want = O.chirp_statistic(O.sft(x, dt, Tsft), psd, dt, Tsft, F, P=P, valid=valid)
    assert O.stat_relative_error(got, want) <= TOL
    if cuts:
        assert 0.05 < 1 - valid.mean() < 0.95


def test_chirp_bins_are_the_oracles(T):
    """P = 0: one bin per segment, so a different bin changes the statistic outright; tracks
    sit exactly on half-integer x (ties round up) and on both sides of them."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    dt, L, n_seg = 1.0, 512, 5
    Tsft = L * dt
    x, psd = _strain(rng, n_seg, L, dt)
    V = np.full((1, n_seg), 1.0 / np.sqrt(n_seg))
    k = rng.integers(2, 250, 300)
    off = np.tile([0.5, 0.5 - 1e-12, 0.5 + 1e-12, 0.25, -0.5], 60)
    c = ((k + off) / Tsft / V[0, 0])[:, None]
    ct = T.build_chirp_table(x, dt, Tsft, psd)
    for P in (0, 1):
        got, *_ = _run(T, torch, ct, T.basis_from_host(V), c, P=P)
        F = O.track_freqs(V, c, np.zeros(300))
        want = O.chirp_statistic(O.sft(x, dt, Tsft), psd, dt, Tsft, F, P=P)
        assert O.stat_relative_error(got, want) <= TOL


def test_chirp_recovers_an_injection_and_topk(T):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    dt, L, n_seg = 1.0, 2048, 8
    Tsft = L * dt
    n_bin = L // 2 + 1
    f0, fdot = 400.2 / Tsft, 12.0 / Tsft ** 2
    x, psd = _strain(rng, n_seg, L, dt, chirp=(f0, fdot, 0.08))
    V = _basis(n_seg, 2)
    ta = O.segment_times(n_seg, Tsft)
    Ftrue = f0 + fdot * ta
    ctrue = np.linalg.lstsq(V.T, Ftrue, rcond=None)[0]
    c = np.concatenate([ctrue[None, :], _tracks(rng, V, 999, n_bin, Tsft, 30.0)])
    ct = T.build_chirp_table(x, dt, Tsft, psd)
    got, ti, tv = _run(T, torch, ct, T.basis_from_host(V), c, topk=16)
    F = O.track_freqs(V, c, np.zeros(1000))
    want = O.chirp_statistic(O.sft(x, dt, Tsft), psd, dt, Tsft, F)
    assert O.stat_relative_error(got, want) <= TOL
    assert int(ti[0].item()) == 0 and got[0] > 2.5 * np.median(got)
    gi, _ = O.topk(got, 16)
    assert np.array_equal(ti.cpu().numpy(), gi)


def test_chirp_edges(T):
    """One segment (fdot = 0), two segments, tracks wholly outside the table, N = 0."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    dt, L = 1.0, 512
    Tsft = L * dt
    for n_seg in (1, 2):
        x, psd = _strain(rng, n_seg, L, dt)
        V = _basis(n_seg, 1) if n_seg == 1 else _basis(n_seg, 2)
        # tracks across and beyond the band, drifting at most 60 bins per segment (the
        # documented range of the template is |fdot| T^2 <= 100)
        Ft = rng.uniform(-0.5, 1.5, (200, 1)) * 257 / Tsft + rng.uniform(-30, 30, (200, 1)) / Tsft * \
            np.arange(n_seg)[None, :]
        c = np.ascontiguousarray(np.linalg.lstsq(V.T, Ft.T, rcond=None)[0].T)
        ct = T.build_chirp_table(x, dt, Tsft, psd)
        got, *_ = _run(T, torch, ct, T.basis_from_host(V), c)
        F = O.track_freqs(V, c, np.zeros(200))
        want = O.chirp_statistic(O.sft(x, dt, Tsft), psd, dt, Tsft, F)
        assert O.stat_relative_error(got, want) <= TOL
        assert (want == 0).any() and (want > 0).any()
    empty = torch.zeros((0, V.shape[0]), dtype=torch.float64, device="cuda")
    stat, _, _ = T.eval_chirp_stat(ct, T.basis_from_host(V), empty)
    assert stat.numel() == 0


def test_chirp_batch_equals_single_calls_and_views(T):
    """Jobs of different tables, bases, P and cuts in one launch give exactly what each gives
    alone (one warp per track: nothing depends on the neighbours); a view of a table's first
    rows equals the table built from the strain's first segments."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    dt, L = 1.0, 1024
    Tsft = L * dt
    jobs, singles = [], []
    tables = []
    for n_seg, K, P, cuts in [(9, 3, 100, False), (12, 4, 50, True), (5, 2, 111, False), (9, 2, 0, True)]:
        x, psd = _strain(rng, n_seg, L, dt, chirp=(200.2 / Tsft, 3.0 / Tsft ** 2, 0.2))
        ct = T.build_chirp_table(x, dt, Tsft, psd)
        tables.append((x, psd, ct))
        V = _basis(n_seg, K)
        b = T.basis_from_host(V)
        c = torch.tensor(_tracks(rng, V, int(rng.integers(1, 600)), L // 2 + 1, Tsft, 40.0), device="cuda")
        jobs.append(T.ChirpJob(ct, b, c, None, P=P, segment_cuts=cuts))
        singles.append(T.eval_chirp_stat(ct, b, c, None, P=P, segment_cuts=cuts)[0])
    T.eval_chirp_batch(jobs)
    torch.cuda.synchronize()
    for j, s1 in zip(jobs, singles):
        assert np.array_equal(j.stat.cpu().numpy().view(np.uint32), s1.cpu().numpy().view(np.uint32))
    x, psd, ct = tables[1]
    v = T.ctable_view(ct, 0, 7)
    pre = T.build_chirp_table(x[: 7 * L], dt, Tsft, psd)
    zv, wv = v.to_host()
    zp, wp = pre.to_host()
    assert np.array_equal(zv, zp) and np.array_equal(wv, wp)


def test_chirp_full_size_sampled(T):
    """The benchmark's one-year configuration (`bench.py --workload chirp`: 2 x 10^5 tracks,
    P = 100, table from the strain on the device); 12 sampled tracks against the oracle."""
    torch = pytest.importorskip("torch")
    from paper_2510_20891_gb300 import synth

    w = synth.WORKLOADS["oneyear_daily_fp32"]
    rng = np.random.default_rng(0)
    x, _ = synth.make_strain(w, rng)
    psd = synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft)
    V, s, lo, hi = O.svd_basis(synth.make_training_tracks(w, rng), w.K)
    N = 200_000
    coeffs = synth.uniform_coeffs(N, lo, hi, np.random.default_rng(5))
    ct = T.build_chirp_table(torch.from_numpy(x).cuda(), w.dt, w.T_sft, psd)
    stat, ti, tv = T.eval_chirp_stat(ct, T.basis_from_host(V), torch.from_numpy(coeffs).cuda(), topk=16)
    torch.cuda.synchronize()
    got = stat.cpu().numpy().astype(np.float64)
    sample = np.concatenate([np.random.default_rng(6).choice(N, 8, replace=False), ti.cpu().numpy()[:4]])
    F = O.track_freqs(V, coeffs[sample], np.zeros(sample.size))
    want = O.chirp_statistic(O.sft(x, w.dt, w.T_sft), psd, w.dt, w.T_sft, F)
    assert O.stat_relative_error(got[sample], want) <= TOL
    gi, _ = O.topk(got, 16)
    assert np.array_equal(ti.cpu().numpy(), gi)
