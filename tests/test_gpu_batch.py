"""Batched evaluation (tfs_eval_batch): many datasets of different shapes in one
persistent launch per table dtype.

A job's bins do not depend on how its tracks are grouped into tiles, but
which pairs the FP32 filter leaves to the FP64 fix-up sum does (the decision
limit and the base bin are warp-uniform, the staged band is per tile), so the
statistic of a job inside a batch equals tfs_eval_stat on the job alone within
FP32 rounding of the sum (relative 1e-6), and each job is checked against the
FP64 oracle on the same stored table (relative 1e-5, the parity tolerance).  The same call repeated
gives bit-identical results, and so does a CUDA-graph replay against an
uncaptured call.
"""
import math

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


def _dataset(T, rng, n_seg, n_bin, Tsft, dtype, K):
    """Random chi^2_2-like power table and an orthonormal basis [K][n_seg]."""
    P = rng.exponential(2.0, size=(n_seg, n_bin))
    P[:, 0] = 0.0
    table = T.table_from_power(P, Tsft, dtype)
    U = np.linalg.qr(rng.standard_normal((n_seg, K)))[0].T.copy()
    return table, T.basis_from_host(U), U


def _tracks(rng, N, K, n_seg, n_bin, Tsft, n_ties=0):
    """f_ref across the band (a few tracks leave the table), coefficients spreading
    each track over ~5% of the bins; the first n_ties tracks sit exactly on a
    half-integer x in every segment (c = 0, Tsft a power of two)."""
    f_ref = rng.uniform(-0.02, 1.02, N) * n_bin / Tsft
    scale = 0.05 * n_bin / Tsft * math.sqrt(n_seg) / math.sqrt(K)
    c = rng.uniform(-1.0, 1.0, (N, K)) * scale
    for t in range(min(n_ties, N)):
        c[t] = 0.0
        f_ref[t] = (rng.integers(1, n_bin - 1) + 0.5) / Tsft
    return c, f_ref


SPECS = [
    # dtype,  n_seg, n_bin,  Tsft,     K,  N,     m, topk, ties
    ("f32", 17, 300, 4096.0, 3, 5000, 1, 10, 5),
    ("f32", 365, 2049, 86400.0, 6, 40000, 0, 0, 0),
    ("bf16", 64, 1001, 1.0e4, 4, 777, 2, 5, 0),
    ("f32", 100, 500, 2.0e4, 8, 0, 1, 3, 0),
    ("f16", 33, 8641, 5.0e4, 2, 1, 7, 1, 0),
    ("f8e4m3", 50, 700, 1.0e5, 13, 3000, 1, 1024, 0),
    ("f32", 40, 400, 8192.0, 20, 2000, 3, 7, 3),
    ("f32", 2500, 300, 1024.0, 3, 3000, 1, 0, 2),
    ("bf16", 7, 64, 512.0, 1, 10000, 0, 16, 4),
]


def _make_jobs(T, torch, specs, seed):
    rng = np.random.default_rng(seed)
    out = []
    for (dtype, n_seg, n_bin, Tsft, K, N, m, topk, ties) in specs:
        table, basis, U = _dataset(T, rng, n_seg, n_bin, Tsft, dtype, K)
        c, f = _tracks(rng, N, K, n_seg, n_bin, Tsft, ties)
        out.append(dict(table=table, basis=basis, U=U, c=c, f=f, m=m, topk=topk, Tsft=Tsft,
                        dc=torch.tensor(c.reshape(N, K), device="cuda"),
                        df=torch.tensor(f, device="cuda")))
    return out


def _alone(T, torch, d):
    r = T.eval_stat(d["table"], d["basis"], d["dc"], d["df"], m=d["m"], topk=d["topk"])
    torch.cuda.synchronize()
    return r


def _batch(T, torch, data, dev_status=None):
    jobs = [T.Job(d["table"], d["basis"], d["dc"], d["df"], m=d["m"], topk=d["topk"],
                  stat=torch.full((d["dc"].shape[0],), float("nan"), device="cuda")) for d in data]
    T.eval_batch(jobs, dev_status=dev_status)
    torch.cuda.synchronize()
    return jobs


def _same(torch, job, alone, exact=True):
    a = alone.stat.cpu().numpy()
    b = job.stat.cpu().numpy()
    if exact:
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), np.flatnonzero(a != b)[:5]
        if job.topk:
            assert np.array_equal(alone.top_idx.cpu().numpy(), job.top_idx.cpu().numpy())
            assert np.array_equal(alone.top_val.cpu().numpy().view(np.uint32),
                                  job.top_val.cpu().numpy().view(np.uint32))
    else:
        assert O.stat_relative_error(b.astype(np.float64), a.astype(np.float64)) <= 1e-6
    if job.topk and b.size:
        ref_idx, _ = O.topk(b.astype(np.float64), job.topk)
        assert np.array_equal(job.top_idx.cpu().numpy(), ref_idx)


def _check_vs_alone(T, torch, data, jobs):
    for d, j in zip(data, jobs):
        _same(torch, j, _alone(T, torch, d), exact=False)


def test_batch_equals_each_job_alone_and_the_oracle(T):
    torch = pytest.importorskip("torch")
    data = _make_jobs(T, torch, SPECS, seed=5)
    jobs = _batch(T, torch, data)
    _check_vs_alone(T, torch, data, jobs)
    for d, j in zip(data, jobs):
        if d["c"].shape[0] == 0:
            continue
        Pq, _ = d["table"].to_host()
        S, idx, val, _ = O.eval_stat(Pq, d["U"], d["c"], d["f"], d["Tsft"], d["m"], d["topk"])
        got = j.stat.cpu().numpy().astype(np.float64)
        assert O.stat_relative_error(got, S) <= 1e-5


def test_batch_larger_than_one_launch(T):
    """70 jobs: more than one launch's 64, mixed dtypes."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    specs = []
    for i in range(70):
        dt = ["f32", "bf16", "f16"][i % 3]
        specs.append((dt, int(rng.integers(8, 90)), int(rng.integers(40, 900)), float(2 ** rng.integers(8, 14)),
                      int(rng.integers(1, 9)), int(rng.integers(0, 3000)), int(rng.integers(0, 3)),
                      int(rng.integers(0, 4)), 1))
    data = _make_jobs(T, torch, specs, seed=10)
    jobs = _batch(T, torch, data)
    _check_vs_alone(T, torch, data, jobs)
    again = _batch(T, torch, data)  # the same call twice: deterministic
    for j, k in zip(jobs, again):
        assert np.array_equal(j.stat.cpu().numpy().view(np.uint32), k.stat.cpu().numpy().view(np.uint32))


def test_batch_in_a_cuda_graph(T):
    """Capture once (after one uncaptured call builds the cached per-segment data), then
    replay on new coefficients written in place: each replay equals a fresh call."""
    torch = pytest.importorskip("torch")
    data = _make_jobs(T, torch, SPECS[:3] + SPECS[5:7], seed=21)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    jobs = [T.Job(d["table"], d["basis"], d["dc"], d["df"], m=d["m"], topk=d["topk"]) for d in data]
    T.eval_batch(jobs, dev_status=status)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            T.eval_batch(jobs, dev_status=status, stream=s.cuda_stream)
    torch.cuda.synchronize()
    rng = np.random.default_rng(22)
    for rep in range(3):
        for d in data:
            N, K = d["dc"].shape
            c, f = _tracks(rng, N, K, d["U"].shape[1], d["table"].n_bin, d["Tsft"], 2)
            d["dc"].copy_(torch.tensor(c.reshape(N, K)))
            d["df"].copy_(torch.tensor(f))
        status.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        fresh = _batch(T, torch, data)
        for j, k in zip(jobs, fresh):
            _same(torch, j, _AsResult(k), exact=True)
        _check_vs_alone(T, torch, data, jobs)


class _AsResult:
    """A batch Job seen through the result fields that _same reads."""

    def __init__(self, job):
        self.stat, self.top_idx, self.top_val = job.stat, job.top_idx, job.top_val


def test_autotuned_launch_shape(T):
    """The tuner returns a shape that fits, later calls of that kind use it, and the results
    stay within the parity tolerance of the oracle."""
    torch = pytest.importorskip("torch")
    data = _make_jobs(T, torch, SPECS[:3] + SPECS[5:6], seed=31)
    jobs = [T.Job(d["table"], d["basis"], d["dc"], d["df"], m=d["m"], topk=d["topk"]) for d in data]
    shape, ms, ms0 = T.autotune(jobs, reps=2)
    assert shape["pcap"] in (512, 1024, 2048, 3072, 4096) and shape["tile_div"] in (1, 2, 4, 8) and ms > 0
    assert shape["slots"] in (2, 3, 4, 6, 8) and shape["group"] in (1, 4, 8, 16, 32) and 0 < ms <= ms0
    assert shape["tile_class"] in (0, 1, 2)
    jobs2 = _batch(T, torch, data)
    for d, j in zip(data, jobs2):
        Pq, _ = d["table"].to_host()
        S, *_ = O.eval_stat(Pq, d["U"], d["c"], d["f"], d["Tsft"], d["m"], 0)
        assert O.stat_relative_error(j.stat.cpu().numpy().astype(np.float64), S) <= 1e-5
    T.lib().tfs_tuning_clear()



def test_table_save_and_load_round_trip(T, tmp_path):
    """A saved table comes back bit for bit (every dtype), so its statistic is identical."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(41)
    for dtype in ("f32", "bf16", "f16", "f8e4m3"):
        table, basis, U = _dataset(T, rng, 37, 900, 2.0e4, dtype, 4)
        path = str(tmp_path / f"t_{dtype}.npz")
        table.save(path)
        back = T.table_load(path)
        assert (back.n_seg, back.n_bin, back.dtype, back.T_sft) == (table.n_seg, table.n_bin, table.dtype, table.T_sft)
        P0, s0 = table.to_host()
        P1, s1 = back.to_host()
        assert np.array_equal(P0, P1) and (s0 is None or np.array_equal(s0, s1))
        c, f = _tracks(rng, 2000, 4, 37, 900, 2.0e4)
        a = T.eval_stat(table, basis, c, f, m=1).stat
        b = T.eval_stat(back, basis, c, f, m=1).stat
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_topk_batch_equals_each_array_alone(T):
    """The segmented top-k (tfs_topk_batch): 70 arrays (two pass sets) of ragged sizes across the
    4096-element chunks, with NaN, -0, -inf and heavy ties; each result is the oracle's top-k of
    that array and, bit for bit, tfs_topk's result on the array alone."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(61)
    sizes = [0, 1, 2, 5, 4095, 4096, 4097, 8191, 12288, 100000, 1000003] * 6 + [3, 70000, 1, 4096]
    ks = [int(rng.choice([0, 1, 7, 128, 1024])) for _ in sizes]
    arrs, hosts = [], []
    for n in sizes:
        v = rng.integers(0, 40, n).astype(np.float32) * 0.25
        if n > 20:
            v[rng.choice(n, 5, replace=False)] = np.nan
            v[rng.choice(n, 5, replace=False)] = -0.0
            v[rng.choice(n, 3, replace=False)] = -np.inf
        hosts.append(v)
        arrs.append(torch.from_numpy(v).cuda())
    outs = T.topk_batch(arrs, ks)
    torch.cuda.synchronize()
    assert len(outs) == len(sizes)
    for v, a, k, (idx, val) in zip(hosts, arrs, ks, outs):
        m = min(k, v.size)
        assert idx.numel() == m and val.numel() == m
        if m == 0:
            continue
        ri, rv = O.topk(v.astype(np.float64), m)
        assert np.array_equal(idx.cpu().numpy(), ri)
        assert np.array_equal(val.cpu().numpy().astype(np.float64), rv, equal_nan=True)
        i1, v1 = T.topk(a, m)
        assert np.array_equal(i1.cpu().numpy(), idx.cpu().numpy())
        assert np.array_equal(v1.cpu().numpy().view(np.uint32), val.cpu().numpy().view(np.uint32))


def test_batch_of_64_jobs_launches_few_kernels(T):
    """A 64-job batched call with a top-k per job: one statistic launch and one set of 13
    top-k passes (not 13 per job), each job's top-k the top of its own statistic."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(62)
    table, basis, U = _dataset(T, rng, 40, 600, 1.0e4, "f32", 4)
    jobs = []
    for i in range(64):
        N = int(rng.integers(1, 3000))
        c, f = _tracks(rng, N, 4, 40, 600, 1.0e4)
        jobs.append(T.Job(table, basis, torch.tensor(c, device="cuda"), torch.tensor(f, device="cuda"), m=1,
                          topk=int(rng.integers(1, 40))))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    T.eval_batch(jobs, dev_status=status)  # warm: cached per-segment data and window sums
    torch.cuda.synchronize()
    k0 = T.lib().tfs_kernel_launches()
    T.eval_batch(jobs, dev_status=status)
    torch.cuda.synchronize()
    launches = T.lib().tfs_kernel_launches() - k0
    assert int(status.item()) == 0
    assert launches <= 16, launches
    for j in jobs:
        s = j.stat.cpu().numpy().astype(np.float64)
        ri, _ = O.topk(s, j.topk)
        assert np.array_equal(j.top_idx.cpu().numpy(), ri)


def _force_tile_class(T, tmp_path, table, K, multi, cls, cuts=False):
    """Load a tuning entry that forces the tile class of launches of this kind (the key the library
    derives: table dtype, coefficient slots, log2 of the row pitch and of the segments, batch)."""
    kp = next(v for v in (2, 4, 6, 8, 16, 32) if K <= v)
    dt = {"f32": 0, "bf16": 1, "f16": 2, "f8e4m3": 3}[table.dtype]
    row = (table.n_bin + 31) // 32 * 32
    key = f"{dt}:{kp}:{math.ceil(math.log2(row))}:{math.ceil(math.log2(max(table.n_seg, 1)))}:{int(multi)}"
    if cuts:
        key += ":c"
    path = tmp_path / "force.json"
    path.write_text('{"%s": [0, 0, 0, 0, %d]}' % (key, cls))
    T.lib().tfs_tuning_clear()
    T.tuning_load(str(path))


@pytest.mark.parametrize("dtype,K,m", [("f32", 3, 0), ("f32", 6, 1), ("bf16", 8, 3), ("f8e4m3", 5, 1), ("f16", 2, 2)])
def test_both_tile_classes_match_the_oracle(T, tmp_path, dtype, K, m):
    """The large (12 or 9 tracks per thread) and the small (4) tile classes give the same bins
    and, within FP32 rounding of the sum (1e-6), the same statistic; both match the oracle."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(71 + K + m)
    n_seg, n_bin, Tsft, N = 97, 1200, 2.0e4, 30000
    table, basis, U = _dataset(T, rng, n_seg, n_bin, Tsft, dtype, K)
    c, f = _tracks(rng, N, K, n_seg, n_bin, Tsft, 3)
    Pq, _ = table.to_host()
    S, *_ = O.eval_stat(Pq, U, c, f, Tsft, m, 0)
    got = []
    try:
        for cls in (1, 2):
            _force_tile_class(T, tmp_path, table, K, False, cls)
            r = T.eval_stat(table, basis, c, f, m=m, ties_capacity=64)
            assert O.stat_relative_error(r.stat.astype(np.float64), S) <= 1e-5
            got.append(r)
    finally:
        T.lib().tfs_tuning_clear()
    a, b = got
    assert a.tie_count == b.tie_count
    assert O.stat_relative_error(a.stat.astype(np.float64), b.stat.astype(np.float64)) <= 1e-6
