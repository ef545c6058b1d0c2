"""Serving runtime (tfs_server_*): resident datasets under a device-memory budget,
requests admitted and batched as they arrive, overlapping on the device.

Every served result must match the FP64 oracle's statistic of the same stored
table within the parity tolerance (relative 1e-5), and tfs_eval_stat on the same
dataset and tracks alone within 1e-6 (the bins are identical; only the FP32
summation can differ, because the tiles a request's tracks share decide which
pairs the FP32 filter leaves to the exact path), whether the request ran alone
or in a mix with others, with tables resident or evicted and reloaded; the
top-k must be the top of the returned statistic.
"""
import math
import threading

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


SHAPES = [  # dtype, n_seg, n_bin, Tsft, K
    ("f32", 365, 2049, 86400.0, 6),
    ("bf16", 120, 4001, 2.0e4, 4),
    ("f16", 60, 1001, 5.0e4, 8),
    ("f8e4m3", 200, 3001, 1.0e4, 3),
]


def _datasets(T, seed):
    """Each dataset twice: one table for the server (handed over) and one to evaluate alone."""
    rng = np.random.default_rng(seed)
    out = []
    for dtype, n_seg, n_bin, Tsft, K in SHAPES:
        P = rng.exponential(2.0, (n_seg, n_bin))
        U = np.linalg.qr(rng.standard_normal((n_seg, K)))[0].T.copy()
        out.append(dict(P=P, U=U, Tsft=Tsft, K=K, n_seg=n_seg, n_bin=n_bin, dtype=dtype,
                        basis=T.basis_from_host(U), alone=T.table_from_power(P, Tsft, dtype)))
    return out


def _tracks(rng, d, N):
    f = rng.uniform(-0.01, 1.01, N) * d["n_bin"] / d["Tsft"]
    c = rng.uniform(-1, 1, (N, d["K"])) * 0.05 * d["n_bin"] / d["Tsft"] * math.sqrt(d["n_seg"] / d["K"])
    return c, f


def _requests(rng, data, n):
    reqs = []
    for i in range(n):
        di = int(rng.integers(0, len(data)))
        N = int(10 ** rng.uniform(0, 4.3))
        c, f = _tracks(rng, data[di], N)
        reqs.append(dict(ds=di, c=c, f=f, m=int(rng.integers(0, 3)), topk=int(rng.integers(0, 9))))
    return reqs


def _check(T, data, r, stat, ti, tv):
    d = data[r["ds"]]
    if "Pq" not in d:
        d["Pq"] = d["alone"].to_host()[0]  # the stored (dequantised) values, FP64
    want, *_ = O.eval_stat(d["Pq"], d["U"], r["c"], r["f"], d["Tsft"], r["m"], 0)
    assert O.stat_relative_error(stat.astype(np.float64), want) <= 1e-5
    ref = T.eval_stat(d["alone"], d["basis"], r["c"], r["f"], m=r["m"]).stat
    assert O.stat_relative_error(stat.astype(np.float64), ref.astype(np.float64)) <= 1e-6
    if r["topk"]:
        gi, _ = O.topk(stat.astype(np.float64), r["topk"])
        assert np.array_equal(ti, gi)
        assert np.array_equal(tv, stat[gi])


def _serve(T, srv, ids, reqs, threads=4):
    """Submit from several threads at once; wait for every ticket."""
    tickets = [None] * len(reqs)

    def sub(k):
        for i in range(k, len(reqs), threads):
            r = reqs[i]
            tickets[i] = srv.submit(ids[r["ds"]], r["c"], r["f"], m=r["m"], topk=r["topk"])

    th = [threading.Thread(target=sub, args=(k,)) for k in range(threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return [srv.wait(t, 60000) for t in tickets]


def test_served_results_equal_alone_under_concurrency(T):
    data = _datasets(T, 1)
    srv = T.Server(8 << 30)
    ids = [srv.add_dataset(T.table_from_power(d["P"], d["Tsft"], d["dtype"]), d["basis"]) for d in data]
    rng = np.random.default_rng(2)
    reqs = _requests(rng, data, 48)
    res = _serve(T, srv, ids, reqs)
    for r, (stat, ti, tv) in zip(reqs, res):
        _check(T, data, r, stat, ti, tv)
    st = srv.stats()
    assert st["completed"] == 48 and st["failed"] == 0
    assert st["tracks_completed"] == sum(r["c"].shape[0] for r in reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    # 48 requests from 4 threads at once: while one batch runs the others queue, so batches carry
    # several requests (continuous batching, not a queue served one at a time)
    assert st["batches"] >= 1 and st["mean_jobs_per_batch"] > 1.0
    assert st["evictions"] == 0
    srv.close()


def test_same_result_alone_and_in_the_mix(T):
    """One request served alone, then again inside a burst of 30 others."""
    data = _datasets(T, 3)
    srv = T.Server(8 << 30)
    ids = [srv.add_dataset(T.table_from_power(d["P"], d["Tsft"], d["dtype"]), d["basis"]) for d in data]
    rng = np.random.default_rng(4)
    probe = _requests(rng, data, 1)[0]
    alone = srv.wait(srv.submit(ids[probe["ds"]], probe["c"], probe["f"], m=probe["m"], topk=probe["topk"]))
    mix = _requests(rng, data, 30)
    mix.insert(15, probe)
    res = _serve(T, srv, ids, mix)
    inmix = res[15]
    assert O.stat_relative_error(inmix[0].astype(np.float64), alone[0].astype(np.float64)) <= 1e-6
    _check(T, data, probe, *inmix)
    _check(T, data, probe, *alone)
    srv.close()


def test_budget_evicts_and_reloads_tables(T):
    """A budget that holds about two of the four tables: serving all four must evict
    idle tables and bring them back, with unchanged results."""
    data = _datasets(T, 5)
    tables = [T.table_from_power(d["P"], d["Tsft"], d["dtype"]) for d in data]
    # a resident dataset holds its table and, once evaluated with m = 1, its FP32 window sums
    sizes = sorted(t.nbytes + t.n_seg * ((t.n_bin + 2 + 31) // 32 * 32) * 4 for t in tables)
    budget = sizes[-1] + sizes[-2] + (256 << 10)
    srv = T.Server(budget, max_batch_jobs=8)
    ids = [srv.add_dataset(t, d["basis"]) for t, d in zip(tables, data)]
    rng = np.random.default_rng(6)
    reqs = []
    for rep in range(3):
        for di in range(len(data)):
            c, f = _tracks(rng, data[di], int(rng.integers(100, 3000)))
            reqs.append(dict(ds=di, c=c, f=f, m=1, topk=3))
    res = _serve(T, srv, ids, reqs, threads=1)
    for r, (stat, ti, tv) in zip(reqs, res):
        _check(T, data, r, stat, ti, tv)
    st = srv.stats()
    assert st["evictions"] > 0 and st["loads"] > 0
    assert st["resident_bytes"] <= budget
    srv.close()


def test_results_into_a_callers_buffer(T):
    """wait(stat=buf) fills the first N elements of the caller's (larger, reused) buffer with the
    same values a fresh array gets, and leaves the rest alone."""
    data = _datasets(T, 9)[:2]
    srv = T.Server(8 << 30)
    ids = [srv.add_dataset(T.table_from_power(d["P"], d["Tsft"], d["dtype"]), d["basis"]) for d in data]
    rng = np.random.default_rng(10)
    buf = np.full(50000, -7.0, np.float32)
    for di, N in ((0, 20000), (1, 777), (0, 50000)):
        c, f = _tracks(rng, data[di], N)
        fresh = srv.wait(srv.submit(ids[di], c, f, m=1, topk=4))
        buf[:] = -7.0
        got = srv.wait(srv.submit(ids[di], c, f, m=1, topk=4), stat=buf)
        assert got[0].base is buf or got[0] is buf or np.shares_memory(got[0], buf)
        assert np.array_equal(got[0], fresh[0]) and np.array_equal(got[1], fresh[1])
        assert np.all(buf[N:] == -7.0)
    with pytest.raises(ValueError):
        srv.wait(srv.submit(ids[0], c[:10], f[:10]), stat=np.empty(5, np.float32))
    srv.close()


def test_rejections(T):
    data = _datasets(T, 7)[:1]
    srv = T.Server(64 << 20)
    ds = srv.add_dataset(T.table_from_power(data[0]["P"], data[0]["Tsft"], "f32"), data[0]["basis"])
    c, f = _tracks(np.random.default_rng(8), data[0], 4_000_000)   # 4e6 x 6 x 8 B > 64 MB
    with pytest.raises(T.TfsError) as e:
        srv.submit(ds, c, f)
    assert e.value.code == -2
    with pytest.raises(T.TfsError) as e:
        srv.submit(ds + 5, c[:10], f[:10])
    assert e.value.code == -6
    L = T.lib()
    assert L.tfs_server_wait(srv._h, 123456, 0, None, None, None) == -6
    srv.close()
