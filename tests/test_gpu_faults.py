"""Failures made on the host, never on the GPU: a NaN in the strain, a request whose wait
expires, a server with no room, malformed shapes.  Each is reported through the status
codes (or, for the NaN, carried into the statistic and ranked last by the top-k), and the
context stays usable afterwards."""
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


def test_nan_in_the_strain(T):
    """A NaN sample poisons its segment's spectrum; tracks that read it get a NaN statistic
    (as the oracle does), tracks outside the band are unaffected, and the top-k ranks NaN last."""
    rng = np.random.default_rng(1)
    dt, L, n_seg = 1.0, 256, 8
    x = rng.standard_normal(L * n_seg)
    x[3 * L + 17] = np.nan
    psd = np.full(L // 2 + 1, 2.0)
    table = T.build_sfts(x, dt, L * dt, psd, "hann", "f32")
    U = np.linalg.qr(rng.standard_normal((n_seg, 2)))[0].T.copy()
    basis = T.basis_from_host(U)
    c = rng.uniform(-1, 1, (500, 2)) * 10 / (L * dt)
    f = rng.uniform(10, 110, 500) / (L * dt)
    f[::2] += 400 / (L * dt)  # every other track stays above the band: it never reads the NaN row
    r = T.eval_stat(table, basis, c, f, m=1, topk=20)
    Pq, _ = table.to_host()
    want, *_ = O.eval_stat(O.power_table(x, dt, L * dt, psd), U, c, f, L * dt, 1, 0)
    got = r.stat.astype(np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(want)) and np.isnan(got).any()
    ok = ~np.isnan(want)
    assert O.stat_relative_error(got[ok], want[ok]) <= 1e-5
    assert not np.isnan(r.top_val).any()
    gi, _ = O.topk(got, 20)
    assert np.array_equal(r.top_idx, gi)
    # the context is fine afterwards
    x[3 * L + 17] = 0.0
    T.build_sfts(x, dt, L * dt, psd, "hann", "f32")


def test_server_expired_wait_and_no_room(T):
    rng = np.random.default_rng(2)
    P = rng.exponential(2.0, (30, 500))
    U = np.linalg.qr(rng.standard_normal((30, 3)))[0].T.copy()
    basis = T.basis_from_host(U)
    srv = T.Server(64 << 20)
    ds = srv.add_dataset(T.table_from_power(P, 1e4, "f32"), basis)
    c = rng.uniform(-1, 1, (300000, 3)) * 0.01
    f = rng.uniform(0.005, 0.04, 300000)
    ticket = srv.submit(ds, c, f, m=1, topk=4)
    rc = T.lib().tfs_server_wait(srv._h, ticket, 0, None, None, None)  # expires at once or succeeds
    assert rc in (0, -4)
    if rc == -4:  # the ticket survives an expired wait and completes
        stat, ti, tv = srv.wait(ticket, 60000)
        assert stat.shape == (300000,) and ti.shape == (4,)
    with pytest.raises(T.TfsError) as e:   # more than the whole budget: refused, not queued
        srv.submit(ds, rng.uniform(-1, 1, (4_000_000, 3)), rng.uniform(0, 0.05, 4_000_000))
    assert e.value.code == -2
    with pytest.raises(ValueError):        # malformed: coefficients of the wrong width
        srv.submit(ds, rng.uniform(-1, 1, (10, 5)), rng.uniform(0, 0.05, 10))
    srv.close()


def test_device_wait_timeout_and_recovery(T):
    """A bounded device wait that runs out, made deterministic on the host: the statistic
    kernel's staging warp is held back on a signal that nothing sends, with a 2 ms limit on
    every wait.  The synchronous call returns TFS_ERR_TIMEOUT and the batched call sets its
    device status; the kernel lets its in-flight copies land before it returns, so the next
    ordinary calls on the same context match the oracle."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    n_seg, n_bin, T_sft, K, N = 41, 700, 1.0e4, 3, 6000
    P = rng.exponential(2.0, (n_seg, n_bin))
    U = np.linalg.qr(rng.standard_normal((n_seg, K)))[0].T.copy()
    table = T.table_from_power(P, T_sft, "f32")
    basis = T.basis_from_host(U)
    c = rng.uniform(-1, 1, (N, K)) * 30 / T_sft
    f = rng.uniform(50, 650, N) / T_sft
    S, *_ = O.eval_stat(P.astype(np.float32).astype(np.float64), U, c, f, T_sft, 1, 0)
    first = T.eval_stat(table, basis, c, f, m=1)  # builds the cached per-segment data and window sums
    assert O.stat_relative_error(first.stat.astype(np.float64), S) <= 1e-5
    dc = torch.from_numpy(c).cuda()
    df = torch.from_numpy(f).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    T.set_wait_limit(2_000_000, hold=True)
    try:
        with pytest.raises(T.TfsError) as e:
            T.eval_stat(table, basis, c, f, m=1)
        assert e.value.code == -4
        job = T.Job(table, basis, dc, df, m=1)
        T.eval_batch([job], dev_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 1
    finally:
        T.set_wait_limit(0, hold=False)
    again = T.eval_stat(table, basis, c, f, m=1, topk=8)
    assert np.array_equal(again.stat.view(np.uint32), first.stat.view(np.uint32))
    job = T.Job(table, basis, dc, df, m=1)
    T.eval_batch([job], dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert O.stat_relative_error(job.stat.cpu().numpy().astype(np.float64), S) <= 1e-5
