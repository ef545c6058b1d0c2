"""GB300-native semi-coherent time-frequency track statistic (arXiv:2510.20891).

A thin ctypes binding over ``libtfstat.so`` (include/tfstat.h): every step of
the computation runs in the library's CUDA kernels; this module only
marshals arguments.  Functions keep the C names without the ``tfs_`` prefix:

* ``build_sfts(strain, dt, T_sft, psd, window="hann", dtype="f32")`` -> ``Table``
* ``table_from_power(P, T_sft, dtype="f32")`` -> ``Table``
* ``build_basis(tracks, K=0, tol=1e-7)`` -> ``Basis``;  ``basis_from_host(U)`` -> ``Basis``
* ``eval_stat(table, basis, coeffs, f_ref=None, m=0, topk=0, ...)`` -> ``EvalResult``
* ``eval_batch([Job(table, basis, coeffs, ...), ...], dev_status=None)`` -> the jobs, outputs filled
* ``Server(budget_bytes)``: ``add_dataset(table, basis)``, ``submit(ds, coeffs, ...)`` -> ticket,
  ``wait(ticket, stat=None)`` -> (stat, top_idx, top_val), ``stats()``
* ``autotune(jobs)`` -> (launch shape, ms, default ms); ``tuning_save(path)`` / ``tuning_load(path)``
* ``topk(values, k)`` -> (idx, val)

Array arguments are numpy arrays (host memory: the call copies in and out
and returns when done) or CUDA torch tensors (device memory: work is
enqueued on the current torch stream).  The library must be built first
(``paper_2510_20891_gb300.build.build()``); nothing falls back to the CPU.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import _lib
from ._lib import LIB_PATH, TfsError, check, lib  # noqa: F401

DTYPES = {"f32": 0, "bf16": 1, "f16": 2, "f8e4m3": 3}
WINDOWS = {"rect": 0, "hann": 1}
MEM_HOST, MEM_DEVICE = 0, 1


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _torch():
    import torch

    return torch


def _stream_ptr(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    """The address of a C-contiguous array or tensor (the library reads row-major layouts)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays passed to the library must be C-contiguous (np.ascontiguousarray)")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous (.contiguous())")
    return ctypes.c_void_p(a.data_ptr())


class Table:
    """Device-resident normalised power table P[alpha][k] (owned by the library)."""

    def __init__(self, handle):
        self._h = handle
        n_seg, n_bin, stride = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        dt, T = ctypes.c_int(), ctypes.c_double()
        check(lib().tfs_table_info(self._h, ctypes.byref(n_seg), ctypes.byref(n_bin), ctypes.byref(dt),
                                   ctypes.byref(T), ctypes.byref(stride)))
        self.n_seg, self.n_bin, self.row_stride = n_seg.value, n_bin.value, stride.value
        self.dtype = {v: k for k, v in DTYPES.items()}[dt.value]
        self.T_sft = T.value

    @property
    def handle(self):
        return self._h

    @property
    def nbytes(self) -> int:
        return int(lib().tfs_table_bytes(self._h))

    def to_host(self):
        """Dequantised values as FP64 [n_seg, n_bin] and the FP8 scales (or None)."""
        P = np.empty((self.n_seg, self.n_bin), dtype=np.float64)
        sc = np.empty(self.n_seg, dtype=np.float32) if self.dtype == "f8e4m3" else None
        check(lib().tfs_table_to_host(self._h, _ptr(P), _ptr(sc) if sc is not None else None))
        return P, sc

    def save(self, path: str):
        """Write the stored table exactly as held (.npz: raw elements, FP8 scales, shape, T_sft)."""
        es = {"f32": 4, "bf16": 2, "f16": 2, "f8e4m3": 1}[self.dtype]
        raw = np.empty(self.n_seg * self.row_stride * es, dtype=np.uint8)
        sc = np.empty(self.n_seg, dtype=np.float32)
        check(lib().tfs_table_export(self._h, _ptr(raw), _ptr(sc) if self.dtype == "f8e4m3" else None))
        np.savez(path, raw=raw, scales=sc if self.dtype == "f8e4m3" else np.zeros(0, np.float32),
                 meta=np.array([self.n_seg, self.n_bin, self.row_stride, DTYPES[self.dtype]], dtype=np.int64),
                 T_sft=np.array([self.T_sft]))

    def free(self):
        if self._h:
            lib().tfs_table_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Basis:
    """Device-resident track basis U [K][n_seg] (FP64) plus its training statistics."""

    def __init__(self, handle):
        self._h = handle
        K, n = ctypes.c_int(), ctypes.c_int64()
        check(lib().tfs_basis_info(self._h, ctypes.byref(K), ctypes.byref(n)))
        self.K, self.n_seg = K.value, n.value

    @property
    def handle(self):
        return self._h

    def to_host(self):
        """(U [K, n_seg], sigma [K], cmin [K], cmax [K]) as FP64 numpy arrays."""
        U = np.empty((self.K, self.n_seg))
        s, lo, hi = np.empty(self.K), np.empty(self.K), np.empty(self.K)
        check(lib().tfs_basis_to_host(self._h, _ptr(U), _ptr(s), _ptr(lo), _ptr(hi)))
        return U, s, lo, hi

    def free(self):
        if self._h:
            lib().tfs_basis_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_sfts(strain, dt: float, T_sft: float, psd, window: str = "hann", dtype: str = "f32", stream=None) -> Table:
    """Strain -> normalised power table (tfs_build_sfts)."""
    h = ctypes.c_void_p()
    if _is_torch_cuda(strain):
        torch = _torch()
        psd_t = psd if _is_torch_cuda(psd) else torch.as_tensor(np.asarray(psd, np.float64), device=strain.device)
        assert strain.dtype == torch.float64 and psd_t.dtype == torch.float64
        check(lib().tfs_build_sfts(_ptr(strain), strain.numel(), float(dt), float(T_sft), WINDOWS[window],
                                   _ptr(psd_t), DTYPES[dtype], MEM_DEVICE, _stream_ptr(stream), ctypes.byref(h)))
    else:
        s, p = _f64(strain), _f64(psd)
        check(lib().tfs_build_sfts(_ptr(s), s.size, float(dt), float(T_sft), WINDOWS[window], _ptr(p),
                                   DTYPES[dtype], MEM_HOST, None, ctypes.byref(h)))
    return Table(h)


def table_from_power(P, T_sft: float, dtype: str = "f32") -> Table:
    """Wrap an FP64 power table [n_seg, n_bin] (tfs_table_from_power)."""
    P = _f64(P)
    h = ctypes.c_void_p()
    check(lib().tfs_table_from_power(_ptr(P), P.shape[0], P.shape[1], float(T_sft), DTYPES[dtype], MEM_HOST, None,
                                     ctypes.byref(h)))
    return Table(h)


def build_basis(tracks, K: int = 0, tol: float = 1e-7) -> Basis:
    """Training tracks [M, n_seg] -> SVD basis (tfs_build_basis)."""
    F = _f64(tracks)
    h = ctypes.c_void_p()
    check(lib().tfs_build_basis(_ptr(F), F.shape[0], F.shape[1], int(K), float(tol), MEM_HOST, None,
                                ctypes.byref(h)))
    return Basis(h)


def basis_from_host(U) -> Basis:
    U = _f64(np.atleast_2d(U))
    h = ctypes.c_void_p()
    check(lib().tfs_basis_from_host(_ptr(U), U.shape[0], U.shape[1], ctypes.byref(h)))
    return Basis(h)


def table_load(path: str) -> Table:
    """A table written by Table.save, bit for bit (tfs_table_import)."""
    z = np.load(path)
    n_seg, n_bin, row_stride, dt = (int(v) for v in z["meta"])
    raw = np.ascontiguousarray(z["raw"])
    sc = np.ascontiguousarray(z["scales"]) if z["scales"].size else None
    h = ctypes.c_void_p()
    check(lib().tfs_table_import(_ptr(raw), _ptr(sc) if sc is not None else None, n_seg, n_bin,
                                 float(z["T_sft"][0]), dt, ctypes.byref(h)))
    t = Table(h)
    if t.row_stride != row_stride:
        raise ValueError("saved row stride does not match this library's layout")
    return t


def table_view(table: Table, seg0: int, n_seg: int) -> Table:
    """Rows seg0 .. seg0 + n_seg - 1 of `table`, sharing its device memory (tfs_table_view)."""
    h = ctypes.c_void_p()
    check(lib().tfs_table_view(table.handle, int(seg0), int(n_seg), ctypes.byref(h)))
    v = Table(h)
    v._parent = table  # the view's memory belongs to the parent
    return v


def basis_view(basis: Basis, seg0: int, n_seg: int) -> Basis:
    """Columns seg0 .. seg0 + n_seg - 1 of every basis row, as a new basis (tfs_basis_view)."""
    h = ctypes.c_void_p()
    check(lib().tfs_basis_view(basis.handle, int(seg0), int(n_seg), ctypes.byref(h)))
    return Basis(h)


class _TieReport(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("n_stored", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("track", ctypes.c_void_p), ("seg", ctypes.c_void_p)]


class ChirpTable:
    """Device-resident linear-chirp table (scaled complex spectra of a Hann-windowed strain)."""

    def __init__(self, handle):
        self._h = handle
        n_seg, n_bin = ctypes.c_int64(), ctypes.c_int64()
        T, dt, s_ref = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().tfs_ctable_info(self._h, ctypes.byref(n_seg), ctypes.byref(n_bin), ctypes.byref(T),
                                    ctypes.byref(dt), ctypes.byref(s_ref)))
        self.n_seg, self.n_bin, self.T_sft, self.dt, self.s_ref = n_seg.value, n_bin.value, T.value, dt.value, s_ref.value

    @property
    def handle(self):
        return self._h

    def to_host(self):
        """(z [n_seg, n_bin] complex64, wt [n_bin] float32)."""
        z = np.empty((self.n_seg, self.n_bin, 2), dtype=np.float32)
        wt = np.empty(self.n_bin, dtype=np.float32)
        check(lib().tfs_ctable_to_host(self._h, _ptr(z), _ptr(wt)))
        return z[..., 0] + 1j * z[..., 1], wt

    def free(self):
        if self._h:
            lib().tfs_ctable_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


CHIRP_P = 100  # TFS_CHIRP_P: the paper's 2P + 1 = 201 bins
CHIRP_M = 256  # TFS_CHIRP_M: samples of the template's Fourier integral per segment


def build_chirp_table(strain, dt: float, T_sft: float, psd, stream=None) -> ChirpTable:
    """Strain -> linear-chirp table (tfs_build_chirp_table; Hann window)."""
    h = ctypes.c_void_p()
    if _is_torch_cuda(strain):
        torch = _torch()
        psd_t = psd if _is_torch_cuda(psd) else torch.as_tensor(np.asarray(psd, np.float64), device=strain.device)
        check(lib().tfs_build_chirp_table(_ptr(strain), strain.numel(), float(dt), float(T_sft), _ptr(psd_t),
                                          MEM_DEVICE, _stream_ptr(stream), ctypes.byref(h)))
    else:
        s, p = _f64(strain), _f64(psd)
        check(lib().tfs_build_chirp_table(_ptr(s), s.size, float(dt), float(T_sft), _ptr(p), MEM_HOST, None,
                                          ctypes.byref(h)))
    return ChirpTable(h)


def eval_chirp_stat(ctable: ChirpTable, basis: Basis, coeffs, f_ref=None, P: int = CHIRP_P,
                    segment_cuts: bool = False, topk: int = 0, stat=None, top_idx=None, top_val=None,
                    stream=None):
    """The paper's linear-chirp statistic of a batch of tracks (tfs_eval_chirp_stat).

    coeffs (and f_ref) are CUDA tensors; returns (stat, top_idx, top_val) as CUDA tensors,
    asynchronous on `stream`."""
    torch = _torch()
    N = coeffs.shape[0]
    dev = coeffs.device
    if stat is None:
        stat = torch.empty(N, dtype=torch.float32, device=dev)
    kk = min(topk, N)
    if topk > 0 and top_idx is None:
        top_idx = torch.empty(kk, dtype=torch.int64, device=dev)
        top_val = torch.empty(kk, dtype=torch.float32, device=dev)
    check(lib().tfs_eval_chirp_stat(ctable.handle, basis.handle, _ptr(coeffs),
                                    _ptr(f_ref) if f_ref is not None else None, N, int(P),
                                    _lib.JOB_SEGMENT_CUTS if segment_cuts else 0, _ptr(stat), int(topk),
                                    _ptr(top_idx) if topk else None, _ptr(top_val) if topk else None,
                                    _stream_ptr(stream)))
    return stat, top_idx, top_val


def ctable_view(ctable: ChirpTable, seg0: int, n_seg: int) -> ChirpTable:
    """Rows seg0 .. seg0 + n_seg - 1 of a chirp table, sharing its memory (tfs_ctable_view)."""
    h = ctypes.c_void_p()
    check(lib().tfs_ctable_view(ctable.handle, int(seg0), int(n_seg), ctypes.byref(h)))
    v = ChirpTable(h)
    v._parent = ctable
    return v


@dataclasses.dataclass
class ChirpJob:
    """One job of a batched linear-chirp evaluation (struct tfs_chirp_job); CUDA tensors."""

    table: ChirpTable
    basis: Basis
    coeffs: object
    f_ref: object = None
    P: int = CHIRP_P
    segment_cuts: bool = False
    stat: object = None


def eval_chirp_batch(jobs, stream=None):
    """The linear-chirp statistic of many jobs in one launch (tfs_eval_chirp_batch); a Job's
    missing stat is allocated here.  Asynchronous on `stream`."""
    torch = _torch()
    arr = (_lib.TfsChirpJob * len(jobs))()
    for i, j in enumerate(jobs):
        N = j.coeffs.shape[0]
        if j.stat is None:
            j.stat = torch.empty(N, dtype=torch.float32, device=j.coeffs.device)
        arr[i] = _lib.TfsChirpJob(j.table.handle, j.basis.handle, _ptr(j.coeffs),
                                  _ptr(j.f_ref) if j.f_ref is not None else None, N, int(j.P),
                                  _lib.JOB_SEGMENT_CUTS if j.segment_cuts else 0, _ptr(j.stat))
    check(lib().tfs_eval_chirp_batch(arr, len(jobs), _stream_ptr(stream)))
    return jobs


@dataclasses.dataclass
class EvalResult:
    stat: object            # [N] float32 (numpy, or torch on the device)
    top_idx: object         # [min(topk, N)] int64
    top_val: object         # [min(topk, N)] float32
    tie_count: int | None   # total ties (None if not requested)
    ties: list              # up to ties_capacity (track, segment) pairs


def eval_stat(table: Table, basis: Basis, coeffs, f_ref=None, m: int = 0, topk: int = 0, ties_capacity: int = -1,
              stat=None, top_idx=None, top_val=None, stream=None) -> EvalResult:
    """Statistic of a batch of tracks, its top-k and the rounding ties (tfs_eval_stat).

    ties_capacity < 0 skips the tie report (no synchronisation for device inputs).
    """
    want_ties = ties_capacity >= 0
    cap = max(ties_capacity, 0)
    tt = np.zeros(max(cap, 1), dtype=np.int64)
    ts = np.zeros(max(cap, 1), dtype=np.int32)
    rep = _TieReport(0, 0, cap, tt.ctypes.data, ts.ctypes.data)
    rep_p = ctypes.byref(rep) if want_ties else None
    if _is_torch_cuda(coeffs):
        torch = _torch()
        N = coeffs.shape[0]
        dev = coeffs.device
        if stat is None:
            stat = torch.empty(N, dtype=torch.float32, device=dev)
        kk = min(topk, N)
        if topk > 0 and top_idx is None:
            top_idx = torch.empty(kk, dtype=torch.int64, device=dev)
            top_val = torch.empty(kk, dtype=torch.float32, device=dev)
        check(lib().tfs_eval_stat(table.handle, basis.handle, _ptr(coeffs), _ptr(f_ref) if f_ref is not None else None,
                                  N, m, topk, _ptr(stat), _ptr(top_idx) if topk else None,
                                  _ptr(top_val) if topk else None, rep_p, MEM_DEVICE, _stream_ptr(stream)))
    else:
        c = _f64(coeffs).reshape(-1, basis.K)
        N = c.shape[0]
        fr = _f64(f_ref) if f_ref is not None else None
        stat = np.empty(N, dtype=np.float32)
        kk = min(topk, N)
        top_idx = np.empty(kk, dtype=np.int64)
        top_val = np.empty(kk, dtype=np.float32)
        check(lib().tfs_eval_stat(table.handle, basis.handle, _ptr(c), _ptr(fr) if fr is not None else None, N, m,
                                  topk, _ptr(stat), _ptr(top_idx) if topk else None, _ptr(top_val) if topk else None,
                                  rep_p, MEM_HOST, None))
    ties = list(zip(tt[: rep.n_stored].tolist(), ts[: rep.n_stored].tolist())) if want_ties else []
    return EvalResult(stat, top_idx, top_val, int(rep.count) if want_ties else None, ties)


@dataclasses.dataclass
class Job:
    """One dataset of a batched evaluation (struct tfs_job); tensors on the CUDA device."""

    table: Table
    basis: Basis
    coeffs: object
    f_ref: object = None
    m: int = 0
    topk: int = 0
    stat: object = None
    top_idx: object = None
    top_val: object = None
    segment_cuts: bool = False  # TFS_JOB_SEGMENT_CUTS: the paper's segment exclusions


def eval_batch(jobs, dev_status=None, stream=None):
    """Statistic (and top-k) of many datasets in one persistent launch per dtype (tfs_eval_batch).

    Outputs missing from a Job (stat, top-k) are allocated here and set on it.  With a device int32
    `dev_status` the call is asynchronous and capturable into a CUDA graph; without one it waits.
    """
    arr = _job_array(jobs)
    check(lib().tfs_eval_batch(arr, len(jobs), _ptr(dev_status) if dev_status is not None else None,
                               _stream_ptr(stream)))
    return jobs


def _job_array(jobs):
    torch = _torch()
    arr = (_lib.TfsJob * len(jobs))()
    for i, j in enumerate(jobs):
        N = j.coeffs.shape[0]
        dev = j.coeffs.device
        if j.stat is None:
            j.stat = torch.empty(N, dtype=torch.float32, device=dev)
        if j.topk > 0 and j.top_idx is None:
            kk = min(j.topk, N)
            j.top_idx = torch.empty(kk, dtype=torch.int64, device=dev)
            j.top_val = torch.empty(kk, dtype=torch.float32, device=dev)
        arr[i] = _lib.TfsJob(j.table.handle, j.basis.handle, _ptr(j.coeffs),
                             _ptr(j.f_ref) if j.f_ref is not None else None, N, j.m, j.topk,
                             _ptr(j.stat), _ptr(j.top_idx) if j.topk else None,
                             _ptr(j.top_val) if j.topk else None,
                             _lib.JOB_SEGMENT_CUTS if j.segment_cuts else 0, 0)
    return arr


def autotune(jobs, reps: int = 3, stream=None):
    """Choose the statistic kernel's launch shape for `jobs` by coordinate descent over its five
    axes and keep it for launches of this kind (tfs_autotune_batch); returns
    ({"pcap": .., "tile_div": .., "slots": .., "group": ..}, ms per batch, ms per batch with the
    default shape)."""
    arr = _job_array(jobs)
    best = _lib.TfsTuning()
    ms = ctypes.c_double()
    ms0 = ctypes.c_double()
    check(lib().tfs_autotune_batch(arr, len(jobs), int(reps), ctypes.byref(best), ctypes.byref(ms),
                                   ctypes.byref(ms0), _stream_ptr(stream)))
    return ({"pcap": best.pcap, "tile_div": best.tile_div, "slots": best.slots, "group": best.group,
             "tile_class": best.tile_class}, ms.value, ms0.value)


def set_wait_limit(limit_ns: int = 0, hold: bool = False):
    """Limit of the statistic kernel's device waits (0: the default 2 s); hold=True makes its next
    launches time out deterministically (tfs_set_wait_limit; for failure-detection tests)."""
    check(lib().tfs_set_wait_limit(int(limit_ns), 1 if hold else 0))


def tuning_save(path: str):
    check(lib().tfs_tuning_save(path.encode()))


def tuning_load(path: str):
    check(lib().tfs_tuning_load(path.encode()))


class Server:
    """Serving runtime (tfs_server_*): resident datasets under a device-memory budget,
    requests batched as they arrive.  Thread-safe; submit() returns a ticket, wait()
    returns (stat, top_idx, top_val) as numpy arrays."""

    def __init__(self, budget_bytes: int, max_batch_jobs: int = 64):
        self._h = ctypes.c_void_p()
        check(lib().tfs_server_create(int(budget_bytes), int(max_batch_jobs), ctypes.byref(self._h)))
        self._bases = []      # bases must outlive the server
        self._inputs = {}     # host inputs must stay alive until their ticket is waited for
        self._shape = {}
        self._lock = __import__("threading").Lock()

    def add_dataset(self, table: Table, basis: Basis) -> int:
        """Hand `table` over to the server (it frees it) and return the dataset id."""
        ds = ctypes.c_int()
        check(lib().tfs_server_add_dataset(self._h, table.handle, basis.handle, ctypes.byref(ds)))
        table._h = None
        self._bases.append(basis)
        return ds.value

    def submit(self, ds: int, coeffs, f_ref=None, m: int = 0, topk: int = 0) -> int:
        c = _f64(coeffs)
        fr = _f64(f_ref) if f_ref is not None else None
        if 0 <= ds < len(self._bases):
            K = self._bases[ds].K
            if c.ndim != 2 or c.shape[1] != K:
                raise ValueError(f"coefficients must be [N, {K}] for dataset {ds}, got {c.shape}")
            if fr is not None and fr.shape != (c.shape[0],):
                raise ValueError("f_ref must have one entry per track")
        N = c.shape[0]
        t = ctypes.c_int64()
        check(lib().tfs_server_submit(self._h, int(ds), _ptr(c), _ptr(fr) if fr is not None else None, N, int(m),
                                      int(topk), ctypes.byref(t)))
        with self._lock:
            self._inputs[t.value] = (c, fr)
            self._shape[t.value] = (N, min(int(topk), N))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1, stat=None):
        """(stat, top_idx, top_val) of a ticket.  `stat` may be the caller's own float32 buffer of
        at least N elements (reused from request to request); the values fill its first N."""
        with self._lock:
            N, kk = self._shape[ticket]
        if stat is None:
            stat = np.empty(N, dtype=np.float32)
        else:
            if not (isinstance(stat, np.ndarray) and stat.dtype == np.float32 and stat.ndim == 1
                    and stat.flags.c_contiguous and stat.size >= N):
                raise ValueError(f"stat must be a contiguous float32 vector of at least {N} elements")
            stat = stat[:N]
        ti = np.empty(kk, dtype=np.int64)
        tv = np.empty(kk, dtype=np.float32)
        rc = lib().tfs_server_wait(self._h, int(ticket), int(timeout_ms), _ptr(stat), _ptr(ti) if kk else None,
                                   _ptr(tv) if kk else None)
        if rc != -4:  # TIMEOUT keeps the ticket
            with self._lock:
                self._inputs.pop(ticket, None)
                self._shape.pop(ticket, None)
        check(rc)
        return stat, ti, tv

    def stats(self) -> dict:
        st = _lib.TfsServerStats()
        check(lib().tfs_server_get_stats(self._h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in st._fields_}

    def close(self):
        if self._h:
            lib().tfs_server_free(self._h)
            self._h = None
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def topk(values, k: int, stream=None):
    """Indices and values of the k largest entries (tfs_topk)."""
    if _is_torch_cuda(values):
        torch = _torch()
        N = values.numel()
        kk = min(k, N)
        idx = torch.empty(kk, dtype=torch.int64, device=values.device)
        val = torch.empty(kk, dtype=torch.float32, device=values.device)
        check(lib().tfs_topk(_ptr(values), N, k, _ptr(idx), _ptr(val), MEM_DEVICE, _stream_ptr(stream)))
        return idx, val
    v = np.ascontiguousarray(values, dtype=np.float32)
    kk = min(k, v.size)
    idx = np.empty(kk, dtype=np.int64)
    val = np.empty(kk, dtype=np.float32)
    check(lib().tfs_topk(_ptr(v), v.size, k, _ptr(idx), _ptr(val), MEM_HOST, None))
    return idx, val


def topk_batch(arrays, ks, stream=None):
    """Top-k of many CUDA float32 arrays at once (tfs_topk_batch): one set of passes covers up to
    64 arrays; returns [(idx, val), ...], each equal to topk() of that array alone."""
    torch = _torch()
    n = len(arrays)
    outs = []
    vals = (ctypes.c_void_p * max(n, 1))()
    Ns = (ctypes.c_int64 * max(n, 1))()
    kk = (ctypes.c_int * max(n, 1))()
    oi = (ctypes.c_void_p * max(n, 1))()
    ov = (ctypes.c_void_p * max(n, 1))()
    for i, (a, k) in enumerate(zip(arrays, ks)):
        if not (_is_torch_cuda(a) and a.dtype == torch.float32 and a.is_contiguous()):
            raise ValueError("topk_batch takes contiguous CUDA float32 tensors")
        m = min(int(k), a.numel())
        idx = torch.empty(m, dtype=torch.int64, device=a.device)
        val = torch.empty(m, dtype=torch.float32, device=a.device)
        outs.append((idx, val))
        vals[i], Ns[i], kk[i] = _ptr(a).value, a.numel(), int(k)
        oi[i], ov[i] = _ptr(idx).value if m else None, _ptr(val).value if m else None
    check(lib().tfs_topk_batch(vals, Ns, kk, n, oi, ov, _stream_ptr(stream)))
    return outs
