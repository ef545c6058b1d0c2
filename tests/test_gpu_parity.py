"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances (stated per check):
* bins: bit-exact for every (track, segment), ties included;
* statistic: max relative error over tracks <= 1e-5 against the oracle on the
  same stored table (FP32 accumulation of at most ~5000 non-negative terms in
  two levels of <= 32 + 50 additions: <= 90 * 2^-24 = 5.4e-6); against the
  exact FP64 table, additionally the storage rounding: <= 1e-5 (f32),
  4e-3 (bf16, 2^-9), 2e-3 (f16, 2^-11), 6.5e-2 (f8e4m3, 2^-4 plus subnormals);
* tables: f32 elements within 2^-24 relative plus the FP64 FFT error
  (1e-12 of the row's largest value); other dtypes equal to the oracle's
  rounding except at rounding boundaries (one unit in the last place, in at
  most 1e-4 of the elements);
* top-k: the exact top-k of the statistic values (ties by lower index).
"""
import math

import numpy as np
import pytest

import oracle.tfstat_oracle as O
from paper_2510_20891_gb300 import synth

pytestmark = pytest.mark.gpu

STAT_TOL_P64 = {"f32": 1e-5, "bf16": 4e-3, "f16": 2e-3, "f8e4m3": 6.5e-2}
STAT_TOL_SAME_TABLE = 1e-5
INT_MIN, INT_MAX = -(2 ** 31), 2 ** 31 - 1


@pytest.fixture(scope="session")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_20891_gb300 import build as B

    B.build()
    import paper_2510_20891_gb300 as pkg

    return pkg


def oracle_bins_mapped(x, m, n_bin):
    """Oracle bins with the ABI's sentinels for windows wholly outside the table."""
    b, tie = O.bins_and_ties(x)
    out = b.copy()
    out[b + m < 0] = INT_MIN
    out[b - m >= n_bin] = INT_MAX
    out[~np.isfinite(x)] = INT_MAX
    return out.astype(np.int64), tie


def dataset(name, seed=0):
    w = synth.WORKLOADS[name]
    rng = np.random.default_rng(seed)
    x, inj = synth.make_strain(w, rng)
    psd = synth.psd_bins(w.psd_fn(), w.n_bin, w.T_sft)
    F = synth.make_training_tracks(w, rng)
    P64 = O.power_table(x, w.dt, w.T_sft, psd)
    V, s, cmin, cmax = O.svd_basis(F, w.K)
    return dict(w=w, x=x, psd=psd, F=F, P64=P64, V=V, s=s, cmin=cmin, cmax=cmax, inj=inj)


@pytest.fixture(scope="session")
def tiny():
    return dataset("tiny_white_2p18")


@pytest.fixture(scope="session")
def oneyear():
    return dataset("oneyear_daily_fp32")


# --------------------------------------------------------------------------- tables
def _check_table(T, table, P64, dtype):
    got, sc = table.to_host()
    assert got.shape == P64.shape
    if dtype == "f32":
        ref = P64
        tol = 2.0 ** -24 * np.abs(ref) + 1e-12 * np.max(np.abs(ref), axis=1, keepdims=True)
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])
        return
    ref, ref_sc = O.quantise_table(P64, dtype)
    if dtype == "f8e4m3":
        assert np.allclose(sc, ref_sc, rtol=2.0 ** -23)
    diff = got != ref
    frac = diff.mean()
    assert frac <= 1e-4, frac
    if diff.any():
        # a rounding-boundary disagreement is one unit in the last place of the format
        rel = np.abs(got[diff] - ref[diff]) / np.maximum(np.abs(ref[diff]), 1e-300)
        ulp = {"bf16": 2.0 ** -7, "f16": 2.0 ** -10, "f8e4m3": 2.0 ** -3}[dtype]
        assert np.all(rel <= ulp * 1.01), rel.max()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f8e4m3"])
def test_build_sfts_tiny(T, tiny, dtype):
    w = tiny["w"]
    table = T.build_sfts(tiny["x"], w.dt, w.T_sft, tiny["psd"], "hann", dtype)
    assert (table.n_seg, table.n_bin) == (64, 2049)
    _check_table(T, table, tiny["P64"], dtype)


def test_build_sfts_oneyear_red_noise(T, oneyear):
    w = oneyear["w"]
    table = T.build_sfts(oneyear["x"], w.dt, w.T_sft, oneyear["psd"], "hann", "f32")
    assert (table.n_seg, table.n_bin) == (365, 8641)
    _check_table(T, table, oneyear["P64"], "f32")


@pytest.mark.parametrize("L", [4, 6, 12, 30, 250, 2000, 4000, 4096, 10000, 17280, 20000, 40000])
@pytest.mark.parametrize("window", ["hann", "rect"])
def test_build_sfts_lengths(T, L, window):
    rng = np.random.default_rng(L)
    n_seg = 3
    x = rng.standard_normal(n_seg * L + 7)          # a ragged tail that must be dropped
    psd = np.full(L // 2 + 1, 2.0)
    psd[1] = np.inf
    P64 = O.power_table(x, 1.0, float(L), psd, window)
    table = T.build_sfts(x, 1.0, float(L), psd, window, "f32")
    _check_table(T, table, P64, "f32")


def test_build_sfts_closed_form(T):
    L, A, k0 = 4096, 0.05, 40
    n = np.arange(4 * L)
    x = A * np.cos(2 * np.pi * k0 * n / L + 0.3)
    table = T.build_sfts(x, 1.0, float(L), np.full(L // 2 + 1, 2.0), "hann", "f32")
    P, _ = table.to_host()
    assert np.allclose(P[:, k0], 3.4133333333333333, rtol=1e-6)
    assert np.allclose(P[:, k0 + 1], 0.8533333333333333, rtol=1e-6)


def test_table_rebuild_equals_build(T, tiny):
    w = tiny["w"]
    table = T.build_sfts(tiny["x"], w.dt, w.T_sft, tiny["psd"], "hann", "bf16")
    x2 = np.random.default_rng(9).standard_normal(w.n_samples)
    T.check(T.lib().tfs_table_rebuild(table.handle, x2.ctypes.data, x2.size, 0, None))
    fresh = T.build_sfts(x2, w.dt, w.T_sft, tiny["psd"], "hann", "bf16")
    assert np.array_equal(table.to_host()[0], fresh.to_host()[0])


@pytest.mark.parametrize("dtype", ["f32", "f8e4m3"])
def test_statistic_after_rebuild_uses_the_new_strain(T, tiny, dtype):
    """The statistic reads per-table window sums built on the first evaluation with each m: a
    rebuild from new strain must refresh them (for every m used so far), so the statistic after
    the rebuild equals that of a fresh table of the new strain and the oracle's."""
    w = tiny["w"]
    coeffs = synth.uniform_coeffs(3000, tiny["cmin"], tiny["cmax"], np.random.default_rng(11))
    table = T.build_sfts(tiny["x"], w.dt, w.T_sft, tiny["psd"], "hann", dtype)
    basis = T.basis_from_host(tiny["V"])
    before = {m: T.eval_stat(table, basis, coeffs, None, m=m).stat for m in (1, 3)}
    x2 = np.random.default_rng(12).standard_normal(w.n_samples)
    x2 += synth.chirp_signal(w.n_samples, w.dt, 5.2e-3, 1e-9, 0.2)
    T.check(T.lib().tfs_table_rebuild(table.handle, x2.ctypes.data, x2.size, 0, None))
    fresh = T.build_sfts(x2, w.dt, w.T_sft, tiny["psd"], "hann", dtype)
    Pq = fresh.to_host()[0]
    for m in (1, 3):
        got = T.eval_stat(table, basis, coeffs, None, m=m).stat
        assert not np.array_equal(got, before[m])
        assert np.array_equal(got, T.eval_stat(fresh, basis, coeffs, None, m=m).stat)
        ref, *_ = O.eval_stat(Pq, tiny["V"], coeffs, np.zeros(len(coeffs)), w.T_sft, m, 0)
        assert O.stat_relative_error(got, ref) <= STAT_TOL_SAME_TABLE


def test_table_rebuild_host_strain_on_a_stream(T, tiny):
    """Host strain and a stream: the call returns once the strain has been copied (the buffer
    may be overwritten at once) and the transform completes on the stream."""
    torch = pytest.importorskip("torch")
    w = tiny["w"]
    table = T.build_sfts(tiny["x"], w.dt, w.T_sft, tiny["psd"], "hann", "f32")
    x2 = np.random.default_rng(10).standard_normal(w.n_samples)
    keep = x2.copy()
    s = torch.cuda.Stream()
    T.check(T.lib().tfs_table_rebuild(table.handle, x2.ctypes.data, x2.size, 0, s.cuda_stream))
    x2[:] = np.nan
    s.synchronize()
    fresh = T.build_sfts(keep, w.dt, w.T_sft, tiny["psd"], "hann", "f32")
    assert np.array_equal(table.to_host()[0], fresh.to_host()[0])


# --------------------------------------------------------------------------- basis
def _basis_tol(s, k):
    gap = min([abs(s[k] - s[j]) for j in range(len(s)) if j != k] + [s[k]])
    return 1e-12 * s[0] / gap + 1e-12


@pytest.mark.parametrize("name", ["tiny_white_2p18", "oneyear_daily_fp32"])
def test_build_basis_parity(T, name):
    w = synth.WORKLOADS[name]
    F = synth.make_training_tracks(w, np.random.default_rng(3))
    V, s, cmin, cmax = O.svd_basis(F, w.K)
    b = T.build_basis(F, w.K)
    U, sg, lo, hi = b.to_host()
    assert U.shape == V.shape
    assert np.allclose(sg, s, rtol=1e-9)
    for k in range(w.K):
        assert np.max(np.abs(U[k] - V[k])) <= _basis_tol(s, k), k
    assert np.allclose(U @ U.T, np.eye(w.K), atol=1e-12)
    scale = np.max(np.abs(F)) * math.sqrt(w.n_seg)
    assert np.max(np.abs(lo - cmin)) <= 1e-9 * scale and np.max(np.abs(hi - cmax)) <= 1e-9 * scale


def test_build_basis_auto_k(T):
    w = synth.WORKLOADS["tiny_white_2p18"]
    F = synth.make_training_tracks(w, np.random.default_rng(4))
    b = T.build_basis(F, 0, 1e-10)
    assert b.K == 3 == O.svd_basis(F, 0, 1e-10)[0].shape[0]
    w2 = synth.WORKLOADS["oneyear_daily_fp32"]
    F2 = synth.make_training_tracks(w2, np.random.default_rng(4), 800)
    for tol in (1e-3, 1e-5):
        assert T.build_basis(F2, 0, tol).K == O.svd_basis(F2, 0, tol)[0].shape[0]


# --------------------------------------------------------------------------- statistic
def _eval_and_check(T, P64, V, coeffs, f_ref, Tsft, m, dtype, topk=0, check_bins=True):
    table = T.table_from_power(P64, Tsft, dtype)
    basis = T.basis_from_host(V)
    res = T.eval_stat(table, basis, coeffs, f_ref, m=m, topk=topk, ties_capacity=4096)
    fr = np.zeros(len(coeffs)) if f_ref is None else f_ref
    Pq, sq = O.quantise_table(P64, dtype)
    Sq, idx, val, ties = O.eval_stat(Pq, V, coeffs, fr, Tsft, m, topk)
    # FP8 storage saturates at 448 s_alpha by definition: compare with the exact table so saturated
    Pref = np.minimum(P64, 448.0 * sq.astype(np.float64)[:, None]) if dtype == "f8e4m3" else P64
    S64, *_ = O.eval_stat(Pref, V, coeffs, fr, Tsft, m, 0)
    e_same = O.stat_relative_error(res.stat, Sq)
    e_64 = O.stat_relative_error(res.stat, S64)
    assert e_same <= STAT_TOL_SAME_TABLE, e_same
    assert e_64 <= STAT_TOL_P64[dtype], e_64
    assert res.tie_count == len(ties)
    # the report holds min(count, capacity) distinct pairs: all of them when they fit, else a
    # subset of the oracle's ties (which ones depends on the order the device found them)
    assert len(res.ties) == min(len(ties), 4096) and len(set(res.ties)) == len(res.ties)
    if len(ties) <= 4096:
        assert sorted(res.ties) == sorted(ties)
    else:
        assert set(res.ties) <= set(ties)
    if topk:
        gi, gv = O.topk(res.stat, topk)
        assert np.array_equal(res.top_idx, gi)
        assert np.array_equal(res.top_val, res.stat[gi])
    if check_bins:
        bins = np.empty((len(coeffs), P64.shape[0]), dtype=np.int32)
        T.check(T.lib().tfs_eval_bins(table.handle, basis.handle, np.ascontiguousarray(coeffs).ctypes.data,
                                      None if f_ref is None else f_ref.ctypes.data, len(coeffs), m,
                                      bins.ctypes.data, 0, None))
        ob, _ = oracle_bins_mapped(O.track_x(V, coeffs, fr, Tsft), m, P64.shape[1])
        mism = np.argwhere(bins.astype(np.int64) != ob)
        assert mism.size == 0, (mism[:5], bins[tuple(mism[0])], ob[tuple(mism[0])])
    return res, e_same, e_64


@pytest.mark.parametrize("m", [0, 1])
def test_eval_stat_tiny(T, tiny, m):
    w = tiny["w"]
    coeffs = synth.uniform_coeffs(w.n_tracks, tiny["cmin"], tiny["cmax"], np.random.default_rng(5))
    _eval_and_check(T, tiny["P64"], tiny["V"], coeffs, None, w.T_sft, m, "f32", topk=128)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f8e4m3"])
def test_eval_stat_oneyear_dtypes(T, oneyear, dtype):
    w = oneyear["w"]
    N = 3 * 2048 + 777                       # several tiles and a ragged tail
    coeffs = synth.uniform_coeffs(N, oneyear["cmin"], oneyear["cmax"], np.random.default_rng(6))
    res, e_same, e_64 = _eval_and_check(T, oneyear["P64"], oneyear["V"], coeffs, None, w.T_sft, 1, dtype,
                                        topk=64, check_bins=(dtype == "f32"))
    print(f"{dtype}: max rel err vs same table {e_same:.2e}, vs FP64 table {e_64:.2e}")


def test_eval_stat_full_size_sampled(T, oneyear):
    """Ten million tracks in the benchmark's launch configuration (device memory,
    top-128); a sample of 20000 tracks is recomputed by the oracle."""
    torch = pytest.importorskip("torch")
    w = oneyear["w"]
    N = w.n_tracks
    rng = np.random.default_rng(7)
    coeffs = synth.uniform_coeffs(N, oneyear["cmin"], oneyear["cmax"], rng)
    table = T.table_from_power(oneyear["P64"], w.T_sft, "f32")
    basis = T.basis_from_host(oneyear["V"])
    dc = torch.from_numpy(coeffs).cuda()
    res = T.eval_stat(table, basis, dc, None, m=1, topk=128)
    torch.cuda.synchronize()
    stat = res.stat.cpu().numpy()
    sample = rng.choice(N, 20000, replace=False)
    Pq, _ = O.quantise_table(oneyear["P64"], "f32")
    S, *_ = O.eval_stat(Pq, oneyear["V"], coeffs[sample], np.zeros(sample.size), w.T_sft, 1)
    assert O.stat_relative_error(stat[sample], S) <= STAT_TOL_SAME_TABLE
    gi, _ = O.topk(stat, 128)
    assert np.array_equal(res.top_idx.cpu().numpy(), gi)
    St, *_ = O.eval_stat(Pq, oneyear["V"], coeffs[gi], np.zeros(gi.size), w.T_sft, 1)
    assert O.stat_relative_error(res.top_val.cpu().numpy(), St) <= STAT_TOL_SAME_TABLE


@pytest.mark.parametrize("extra", [1, 13 * 4608 - 5, 151 * 4608])
def test_eval_stat_last_round_split(T, oneyear, extra):
    """One round of full tiles over the SMs (152 x 384 x 12 tracks at K = 6) plus a tail: the
    tail's tiles split their segments over several tiles (partial sums added in segment order)
    so that the last round spreads over the SMs.  Tracks on both sides of the boundary, the
    first ones and the last ones match the oracle and, within FP32 rounding of the sums, the
    same tracks evaluated in a launch of their own."""
    torch = pytest.importorskip("torch")
    w = oneyear["w"]
    full = 152 * 384 * 12
    N = full + extra
    rng = np.random.default_rng(27)
    coeffs = synth.uniform_coeffs(N, oneyear["cmin"], oneyear["cmax"], rng)
    table = T.table_from_power(oneyear["P64"], w.T_sft, "f32")
    basis = T.basis_from_host(oneyear["V"])
    dc = torch.from_numpy(coeffs).cuda()
    res = T.eval_stat(table, basis, dc, None, m=1, topk=16)
    torch.cuda.synchronize()
    stat = res.stat.cpu().numpy()
    pick = np.unique(np.concatenate([np.arange(0, 3000), np.arange(full - 3000, min(N, full + 3000)),
                                     np.arange(max(0, N - 3000), N)]))
    Pq, _ = O.quantise_table(oneyear["P64"], "f32")
    S, *_ = O.eval_stat(Pq, oneyear["V"], coeffs[pick], np.zeros(pick.size), w.T_sft, 1)
    assert O.stat_relative_error(stat[pick].astype(np.float64), S) <= STAT_TOL_SAME_TABLE
    tail = T.eval_stat(table, basis, dc[full:], None, m=1).stat.cpu().numpy()
    assert O.stat_relative_error(stat[full:].astype(np.float64), tail.astype(np.float64)) <= 1e-6
    gi, _ = O.topk(stat.astype(np.float64), 16)
    assert np.array_equal(res.top_idx.cpu().numpy(), gi)


def test_eval_stat_full_size_host_chunks(T, oneyear):
    """Ten million tracks from host buffers (the end-to-end configuration): the coefficients
    and offsets go up in chunks, each evaluated as soon as it has arrived, and the values come
    back chunk by chunk.  Bins are those of one launch; the statistic agrees with the
    device-pointer call within FP32 rounding (the tiling decides which pairs take the FP64
    fix-up), a sample matches the oracle, and the top-k is that of the returned values."""
    torch = pytest.importorskip("torch")
    w = oneyear["w"]
    N = w.n_tracks
    rng = np.random.default_rng(17)
    coeffs = synth.uniform_coeffs(N, oneyear["cmin"], oneyear["cmax"], rng)
    f_ref = rng.uniform(-0.5, 0.5, N) / w.T_sft
    table = T.table_from_power(oneyear["P64"], w.T_sft, "f32")
    basis = T.basis_from_host(oneyear["V"])
    res = T.eval_stat(table, basis, coeffs, f_ref, m=1, topk=128)
    dev = T.eval_stat(table, basis, torch.from_numpy(coeffs).cuda(), torch.from_numpy(f_ref).cuda(), m=1, topk=128)
    torch.cuda.synchronize()
    assert O.stat_relative_error(res.stat.astype(np.float64), dev.stat.cpu().numpy().astype(np.float64)) <= 1e-5
    sample = rng.choice(N, 20000, replace=False)
    Pq, _ = O.quantise_table(oneyear["P64"], "f32")
    S, *_ = O.eval_stat(Pq, oneyear["V"], coeffs[sample], f_ref[sample], w.T_sft, 1)
    assert O.stat_relative_error(res.stat[sample].astype(np.float64), S) <= STAT_TOL_SAME_TABLE
    gi, _ = O.topk(res.stat.astype(np.float64), 128)
    assert np.array_equal(res.top_idx, gi)
    assert np.array_equal(res.top_val, res.stat[gi])
    # top-k alone (no per-track output), on a stream of its own: the same launches, the same
    # answer, in host memory when the call returns
    ti = np.empty(128, np.int64)
    tv = np.empty(128, np.float32)
    s = torch.cuda.Stream()
    T.check(T.lib().tfs_eval_stat(table.handle, basis.handle, coeffs.ctypes.data, f_ref.ctypes.data, N, 1, 128,
                                  None, ti.ctypes.data, tv.ctypes.data, None, 0, s.cuda_stream))
    assert np.array_equal(ti, gi) and np.array_equal(tv, res.top_val)


def test_injected_track_stands_out(T, tiny):
    """Strain -> GPU table -> statistic of the true track: far above the noise
    distribution of m = 1 (mean 2*64*3, variance 19.33*64)."""
    w = tiny["w"]
    t = O.segment_times(w.n_seg, w.T_sft)
    f_true = tiny["inj"]["f0"] + tiny["inj"]["fdot"] * t
    c_true = f_true @ tiny["V"].T
    coeffs = synth.uniform_coeffs(5000, tiny["cmin"], tiny["cmax"], np.random.default_rng(8))
    coeffs[1234] = c_true
    table = T.build_sfts(tiny["x"], w.dt, w.T_sft, tiny["psd"], "hann", "f32")
    res = T.eval_stat(table, T.basis_from_host(tiny["V"]), coeffs, None, m=1, topk=4)
    mean, sd = 2 * 64 * 3, math.sqrt(19.333 * 64)
    assert res.stat[1234] > mean + 8 * sd
    assert res.top_val[0] >= res.stat[1234]


# --------------------------------------------------------------------------- edge cases
def _rand_problem(n_seg, n_bin, K, N, seed, T_sft=4096.0):
    rng = np.random.default_rng(seed)
    P = rng.exponential(2.0, (n_seg, n_bin))
    V = rng.standard_normal((K, n_seg)) / math.sqrt(n_seg)
    coeffs = rng.standard_normal((N, K)) * (n_bin / T_sft) * 0.3
    f_ref = rng.uniform(0, n_bin / T_sft, N)
    return P, V, coeffs, f_ref


@pytest.mark.parametrize("K", [1, 2, 3, 5, 7, 8, 12, 20, 32])
def test_eval_stat_basis_sizes(T, K):
    P, V, c, f = _rand_problem(40, 300, K, 3000, K)
    _eval_and_check(T, P, V, c, f, 4096.0, 1, "f32", topk=10)


@pytest.mark.parametrize("m", [0, 2, 7, 64])
def test_eval_stat_neighbour_widths(T, m):
    P, V, c, f = _rand_problem(33, 257, 4, 2500, 100 + m)
    _eval_and_check(T, P, V, c, f, 4096.0, m, "f32", topk=5)


@pytest.mark.parametrize("n_seg", [1, 2, 31, 32, 33, 65])
def test_eval_stat_segment_counts(T, n_seg):
    P, V, c, f = _rand_problem(n_seg, 129, 3, 2100, 200 + n_seg)
    _eval_and_check(T, P, V, c, f, 4096.0, 1, "bf16", topk=3)


@pytest.mark.parametrize("N", [0, 1, 2047, 2048, 2049])
def test_eval_stat_track_counts(T, N):
    P, V, c, f = _rand_problem(8, 100, 3, max(N, 1), 300 + N)
    c, f = c[:N], f[:N]
    if N == 0:
        table = T.table_from_power(P, 4096.0, "f32")
        res = T.eval_stat(table, T.basis_from_host(V), np.zeros((0, 3)), None, m=1)
        assert res.stat.size == 0
        return
    _eval_and_check(T, P, V, c, f, 4096.0, 1, "f32", topk=min(N, 7))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f8e4m3"])
@pytest.mark.parametrize("m", [1, 2, 3, 8, 9])
@pytest.mark.parametrize("n_bin", [64, 700, 1001, 1016, 1024, 1025])
def test_eval_stat_table_edges(T, dtype, m, n_bin):
    """Tracks crowding both ends of the table, many leaving it: the windows that
    reach past bin 0 or past the last bin (window sums built with zeros outside
    the table), for band ends at every position of the builders' 16-byte vectors
    and of a warp's lanes, widths that fit the left zero pad (2m <= 16) and
    widths that do not."""
    rng = np.random.default_rng(1000 * m + n_bin)
    n_seg, K, N, Tsft = 24, 3, 3000, 4096.0
    P = rng.exponential(2.0, (n_seg, n_bin))
    V = np.linalg.qr(rng.standard_normal((n_seg, K)))[0].T.copy()
    side = rng.integers(0, 2, N)
    f_ref = np.where(side == 0, rng.uniform(-3.0 * m - 4, 3.0 * m + 4, N),
                     n_bin + rng.uniform(-3.0 * m - 4, 3.0 * m + 4, N)) / Tsft
    c = rng.uniform(-1.0, 1.0, (N, K)) * 3.0 / Tsft
    _eval_and_check(T, P, V, c, f_ref, Tsft, m, dtype, topk=5)


def test_eval_stat_exact_ties_everywhere(T):
    """Every pair lands exactly on a half-integer: all pairs take the FP64 path,
    the per-segment queues overflow and the tie report lists every pair."""
    n_seg, n_bin, Tsft = 6, 64, 4096.0
    P = np.random.default_rng(1).exponential(2.0, (n_seg, n_bin))
    V = np.zeros((1, n_seg))
    N = 3000
    k = np.random.default_rng(2).integers(0, n_bin - 1, N)
    f_ref = (k + 0.5) / Tsft
    coeffs = np.zeros((N, 1))
    res, _, _ = _eval_and_check(T, P, V, coeffs, f_ref, Tsft, 0, "f32")
    assert res.tie_count == N * n_seg


def test_eval_stat_out_of_range_and_nonfinite(T):
    P, V, c, f = _rand_problem(10, 50, 2, 400, 9)
    f[:50] = -1.0                    # far below bin 0
    f[50:100] = 1e3                  # far above the table
    c[100:110, 0] = np.nan           # not finite: contributes 0
    c[110:120, 1] = 1e9              # huge coefficients: the FP64 path for every segment
    f[120:130] = -0.2 / 4096.0       # straddling bin 0
    f[130:140] = (49.6) / 4096.0     # straddling the last bin
    res, _, _ = _eval_and_check(T, P, V, c, f, 4096.0, 1, "f32")
    assert np.all(res.stat[:100] == 0) and np.all(res.stat[100:110] == 0)


# --------------------------------------------------------------------------- top-k
@pytest.mark.parametrize("N", [1, 5, 4096, 4097, 1_000_003])
@pytest.mark.parametrize("k", [1, 7, 128, 1024])
def test_topk_parity(T, N, k):
    rng = np.random.default_rng(N + k)
    v = rng.integers(0, 50, N).astype(np.float32) * 0.5
    if N > 10:
        v[rng.choice(N, 5, replace=False)] = np.nan
        v[rng.choice(N, 5, replace=False)] = -0.0
        v[rng.choice(N, 3, replace=False)] = -np.inf
    idx, val = T.topk(v, k)
    ri, rv = O.topk(v.astype(np.float64), k)
    assert np.array_equal(idx, ri)
    assert np.array_equal(val.astype(np.float64), rv, equal_nan=True)


@pytest.mark.parametrize("N", [9, 5000, 300_001])
def test_topk_boundary_ties(T, N):
    """Equal values at the k-th place: when all of them are among the k (k = 4, 9, 10 here) one pass
    collects them without ranks, when some are left out (k = 6) the lowest indices are taken; in
    both the output orders equal values by lower index."""
    rng = np.random.default_rng(N)
    v = (rng.permutation(N).astype(np.float32) + 1.0) / (N + 1.0)   # distinct values in (0, 1)
    top = rng.choice(N, 9, replace=False)
    v[top[:4]] = 3.0                                                # four equal maxima
    v[top[4:]] = 2.0                                                # five equal values below them
    for k in (4, 6, 9, 10):
        idx, val = T.topk(v, k)
        ri, rv = O.topk(v.astype(np.float64), k)
        assert np.array_equal(idx, ri), k
        assert np.array_equal(val.astype(np.float64), rv), k


def test_topk_device_distinct_values(T):
    torch = pytest.importorskip("torch")
    v = torch.randn(3_000_001, device="cuda")
    idx, val = T.topk(v, 1000)
    vh = v.cpu().numpy()
    ri, _ = O.topk(vh.astype(np.float64), 1000)
    assert np.array_equal(idx.cpu().numpy(), ri)
