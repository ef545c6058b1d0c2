"""The plunge-time search (Sec. II.D) on the GPU: chunk views and shifted bases evaluated in
one batched launch against the oracle's chunk_eval; the differential-evolution kernels
against numpy and the device draws against the generator's host definition; the population
driver against the oracle's statistic of its result."""
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


def _dataset(rng, n_seg=60, n_bin=700, Tsft=2.0e4, K=4):
    P = rng.exponential(2.0, (n_seg, n_bin))
    t = (np.arange(n_seg) + 0.5) * Tsft
    D = n_seg * Tsft
    f0 = rng.uniform(2, 6, 500) * 100 / Tsft
    tau = D * rng.uniform(1.001, 1.2, 500)
    F = f0[:, None] * (1 - t[None, :] / tau[:, None]) ** -0.3
    V = np.linalg.svd(F, full_matrices=False)[2][:K].copy()
    c = F @ V.T
    return P, V, c.min(axis=0), c.max(axis=0), Tsft


def test_chunks_in_one_batch_equal_the_oracle(T):
    torch = pytest.importorskip("torch")
    from paper_2510_20891_gb300 import search

    rng = np.random.default_rng(1)
    P, V, lo, hi, Tsft = _dataset(rng)
    sizes = [10 + 4 * i for i in range(13)]
    for dtype in ("f32", "bf16"):
        table = T.table_from_power(P, Tsft, dtype)
        cs = search.ChunkSearch(table, T.basis_from_host(V), sizes)
        coeffs = [lo + (hi - lo) * rng.random((int(rng.integers(1, 900)), V.shape[0])) for _ in sizes]
        f_ref = [rng.uniform(-1, 1, c.shape[0]) / Tsft for c in coeffs]
        jobs = cs.evaluate([torch.tensor(c, device="cuda") for c in coeffs],
                           [torch.tensor(f, device="cuda") for f in f_ref], m=1, topk=5)
        torch.cuda.synchronize()
        Pq, _ = table.to_host()
        want = O.chunk_eval(Pq, V, coeffs, f_ref, sizes, Tsft, 1)
        for j, w in zip(jobs, want):
            got = j.stat.cpu().numpy().astype(np.float64)
            assert O.stat_relative_error(got, w) <= 1e-5
            gi, _ = O.topk(got, 5)
            assert np.array_equal(j.top_idx.cpu().numpy(), gi)
        if dtype == "f32":
            # a view gives what a table of the same rows gives
            n = sizes[5]
            alone = T.eval_stat(T.table_from_power(Pq[:n], Tsft, "f32"), cs.bases[5], coeffs[5], f_ref[5], m=1).stat
            assert O.stat_relative_error(alone.astype(np.float64), want[5]) <= 1e-5


def test_views_reject_bad_ranges_and_servers(T):
    rng = np.random.default_rng(2)
    P, V, *_ = _dataset(rng, n_seg=20)
    table = T.table_from_power(P, 2.0e4, "f32")
    basis = T.basis_from_host(V)
    for seg0, n in ((-1, 5), (0, 0), (15, 6)):
        with pytest.raises(T.TfsError):
            T.table_view(table, seg0, n)
        with pytest.raises(T.TfsError):
            T.basis_view(basis, seg0, n)
    v = T.table_view(table, 3, 10)
    srv = T.Server(1 << 30)
    with pytest.raises(T.TfsError):
        srv.add_dataset(v, T.basis_view(basis, 3, 10))
    srv.close()
    U, *_ = T.basis_view(basis, 4, 9).to_host()
    assert np.array_equal(U, V[:, 4:13])


def test_de_kernels_against_numpy(T):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    N, K = 3000, 6
    c = rng.standard_normal((N, K))
    r1 = rng.integers(0, N, N).astype(np.int32)
    r2 = rng.integers(0, N, N).astype(np.int32)
    F = rng.uniform(0.3, 1.5, N).astype(np.float32)
    lo, hi = -np.full(K, 1.5), np.full(K, 1.5)
    d = lambda a: torch.tensor(a, device="cuda")
    cd, ct, ip = d(c), torch.empty((N, K), dtype=torch.float64, device="cuda"), torch.empty(N, dtype=torch.int32,
                                                                                         device="cuda")
    L = T.lib()
    r1d, r2d, Fd, lod, hid = d(r1), d(r2), d(F), d(lo), d(hi)
    T.check(L.tfs_de_propose(cd.data_ptr(), N, K, r1d.data_ptr(), r2d.data_ptr(), Fd.data_ptr(), lod.data_ptr(),
                             hid.data_ptr(), ct.data_ptr(), ip.data_ptr(), None))
    want = c + F.astype(np.float64)[:, None] * (c[r1] - c[r2])
    assert np.array_equal(ct.cpu().numpy(), want)
    assert np.array_equal(ip.cpu().numpy(), np.all((want >= lo) & (want <= hi), axis=1).astype(np.int32))
    s = rng.standard_normal(N).astype(np.float32)
    s_trial = rng.standard_normal(N).astype(np.float32)
    sd, std_ = d(s), d(s_trial)
    T.check(L.tfs_de_accept(cd.data_ptr(), sd.data_ptr(), ct.data_ptr(), std_.data_ptr(), ip.data_ptr(), N, K, None))
    acc = (ip.cpu().numpy() == 1) & (s_trial > s)
    assert np.array_equal(cd.cpu().numpy(), np.where(acc[:, None], want, c))
    assert np.array_equal(sd.cpu().numpy(), np.where(acc, s_trial, s))


def test_de_draw_is_the_published_generator(T):
    """tfs_de_draw against the host definition of the same SplitMix64 draws, bit for bit, over
    three iterations (the device counter advances once per call), with a ragged chunk count."""
    torch = pytest.importorskip("torch")
    from tests.splitmix import de_draws

    L = T.lib()
    for n_ch, W, seed in ((5, 3, 1), (48, 512, 123456789123), (7, 1000, (1 << 63) - 25)):
        n = n_ch * W
        it = torch.zeros(1, dtype=torch.int32, device="cuda")
        r1 = torch.empty(n, dtype=torch.int32, device="cuda")
        r2 = torch.empty(n, dtype=torch.int32, device="cuda")
        F = torch.empty(n, dtype=torch.float32, device="cuda")
        for i in range(3):
            T.check(L.tfs_de_draw(seed, it.data_ptr(), n_ch, W, 0.3, 1.5, r1.data_ptr(), r2.data_ptr(), F.data_ptr(),
                                  None))
            w1, w2, wF = de_draws(seed, i, n_ch, W, 0.3, 1.5)
            assert np.array_equal(r1.cpu().numpy(), w1)
            assert np.array_equal(r2.cpu().numpy(), w2)
            assert np.array_equal(F.cpu().numpy().view(np.uint32), wF.view(np.uint32))
        assert int(it.item()) == 3
    with pytest.raises(T.TfsError):
        T.check(L.tfs_de_draw(1, it.data_ptr(), 4, 2, 0.3, 1.5, r1.data_ptr(), r2.data_ptr(), F.data_ptr(), None))


def test_de_driver_results_are_the_oracles(T):
    """A short search over 6 chunks: the reported best of every chunk is the oracle's statistic
    of the returned coefficients and at least the initial best; graph replay and plain calls
    give the same search."""
    torch = pytest.importorskip("torch")
    from paper_2510_20891_gb300 import search

    rng = np.random.default_rng(4)
    P, V, lo, hi, Tsft = _dataset(rng, n_seg=40, K=3)
    sizes = [12, 18, 24, 30, 36, 40]
    table = T.table_from_power(P, Tsft, "f32")
    cs = search.ChunkSearch(table, T.basis_from_host(V), sizes)
    de0 = search.DESearch(cs, lo, hi, m=1, n_init=256, n_walkers=64, f_start=(4e-3, 2e-2), seed=5)
    r0 = de0.run(n_iter=0, U_full=V)
    de = search.DESearch(cs, lo, hi, m=1, n_init=256, n_walkers=64, f_start=(4e-3, 2e-2), seed=5)
    r = de.run(n_iter=40, U_full=V)
    assert r.evaluations == len(sizes) * (256 + 40 * 64)
    assert np.all(r.stat >= r0.stat)
    assert np.any(r.stat > r0.stat)
    for i, n in enumerate(sizes):
        want = O.chunk_eval(P, V, [r.coeffs[i][None, :]], [np.zeros(1)], [n], Tsft, 1)[0][0]
        assert abs(r.stat[i] - want) <= 1e-5 * want
    rp = search.DESearch(cs, lo, hi, m=1, n_init=256, n_walkers=64, f_start=(4e-3, 2e-2), seed=5,
                         graph=False).run(n_iter=40, U_full=V)
    assert np.array_equal(rp.stat, r.stat)
    mom = np.array([O.noise_moments(n, 1) for n in sizes])
    assert np.allclose(r.normalised, (r.stat - mom[:, 0]) / mom[:, 1])


def test_de_driver_with_the_linear_chirp_statistic(T):
    """The same driver on the paper's own statistic (chirp table views, one chirp launch per
    iteration, the paper's exclusions): its results are the oracle's masked linear-chirp
    statistic of the returned coefficients."""
    torch = pytest.importorskip("torch")
    from paper_2510_20891_gb300 import search

    rng = np.random.default_rng(9)
    dt, L, n_seg, K = 4.0, 1024, 24, 3
    Tsft = L * dt
    t = (np.arange(n_seg) + 0.5) * Tsft
    D = n_seg * Tsft
    F = rng.uniform(40, 150, 400)[:, None] / Tsft * (1 - t[None, :] / (D * rng.uniform(1.001, 1.3, 400))[:, None]) ** -0.3
    V = np.linalg.svd(F, full_matrices=False)[2][:K].copy()
    c = F @ V.T
    lo, hi = c.min(axis=0), c.max(axis=0)
    x = rng.standard_normal(n_seg * L)
    psd = np.full(L // 2 + 1, 2.0 * dt)
    ct = T.build_chirp_table(x, dt, Tsft, psd)
    sizes = [8, 12, 16, 20, 24]
    cs = search.ChunkSearch(None, T.basis_from_host(V), sizes, chirp_table=ct)
    r = search.DESearch(cs, lo, hi, n_init=128, n_walkers=32, f_start=(40 / Tsft, 150 / Tsft), seed=3,
                        segment_cuts=True, statistic="chirp").run(n_iter=10, U_full=V)
    assert r.evaluations == len(sizes) * (128 + 10 * 32)
    d = O.sft(x, dt, Tsft)
    for i, n in enumerate(sizes):
        Fi = O.track_freqs(V[:, n_seg - n:], r.coeffs[i][None, :], np.zeros(1))
        want = O.chirp_statistic(d[:n], psd, dt, Tsft, Fi, valid=O.segment_validity(Fi, Tsft))[0]
        assert abs(r.stat[i] - want) <= 2e-5 * abs(want)
