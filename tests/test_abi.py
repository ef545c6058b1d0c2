"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
symbol include/tfstat.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import subprocess

import pytest

from paper_2510_20891_gb300 import _lib
from paper_2510_20891_gb300 import build as B


@pytest.fixture(scope="module")
def L():
    B.build()
    return _lib.lib()


def test_header_declares_the_boundary_calls():
    syms = _lib.header_symbols()
    for name in ("tfs_build_sfts", "tfs_build_basis", "tfs_eval_stat", "tfs_topk"):
        assert name in syms


def test_library_exports_every_header_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in _lib.header_symbols() if s not in exported]
    assert not missing, missing
    for s in _lib.header_symbols():
        assert hasattr(L, s)


def test_binding_declares_exactly_the_header(L):
    assert set(_lib.SIGNATURES) == set(_lib.header_symbols())


def test_binding_constants_equal_the_header():
    import os
    import re

    import paper_2510_20891_gb300 as T

    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "tfstat.h")).read()
    defs = dict(re.findall(r"#define (TFS_[A-Z0-9_]+) (-?\d+)", hdr))
    assert int(defs["TFS_CHIRP_P"]) == T.CHIRP_P
    assert int(defs["TFS_CHIRP_M"]) == T.CHIRP_M


def test_library_targets_sm103a(L):
    out = subprocess.run(["cuobjdump", "--list-elf", _lib.LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_version_and_error_string(L):
    assert L.tfs_version() == 10000
    assert L.tfs_last_error() is not None


def test_host_validation_without_device(L):
    P = ctypes.c_void_p
    # null handles and shapes are rejected before any CUDA call
    assert L.tfs_eval_stat(None, None, None, None, 0, 0, 0, None, None, None, None, 0, None) == -1
    assert b"null" in L.tfs_last_error()
    buf = (ctypes.c_float * 4)()
    idx = (ctypes.c_int64 * 4)()
    val = (ctypes.c_float * 4)()
    assert L.tfs_topk(ctypes.cast(buf, P), 0, 4, ctypes.cast(idx, P), ctypes.cast(val, P), 0, None) == -1
    assert L.tfs_topk(ctypes.cast(buf, P), 4, 2000, ctypes.cast(idx, P), ctypes.cast(val, P), 0, None) == -1
    x = (ctypes.c_double * 64)()
    out = P()
    # T_sft / dt = 7 is not even and 2,3,5-smooth
    assert L.tfs_build_sfts(ctypes.cast(x, P), 64, 1.0, 7.0, 1, ctypes.cast(x, P), 0, 0, None, ctypes.byref(out)) == -1
    assert L.tfs_build_sfts(ctypes.cast(x, P), 64, 1.0, 14.0, 1, ctypes.cast(x, P), 0, 0, None, ctypes.byref(out)) == -1
    assert b"prime factors" in L.tfs_last_error()
    assert L.tfs_build_basis(ctypes.cast(x, P), 8, 8, 40, 0.0, 0, None, ctypes.byref(out)) == -1
    assert L.tfs_basis_from_host(ctypes.cast(x, P), 0, 8, ctypes.byref(out)) == -1
    # batched evaluation: job list and per-job handles are checked before any CUDA call
    assert L.tfs_eval_batch(None, 1, None, None) == -1
    jobs = (_lib.TfsJob * 2)()
    assert L.tfs_eval_batch(jobs, 0, None, None) == -1
    assert L.tfs_eval_batch(jobs, 5000, None, None) == -1
    assert L.tfs_eval_batch(jobs, 2, None, None) == -1
    assert b"job 0" in L.tfs_last_error()
    # the linear-chirp calls validate before any CUDA call
    out = P()
    x = (ctypes.c_double * 1024)()
    assert L.tfs_build_chirp_table(ctypes.cast(x, P), 1024, 1.0, 256.0, ctypes.cast(x, P), 0, None,
                                   ctypes.byref(out)) == -1          # L = 256 < 512
    assert L.tfs_eval_chirp_stat(None, None, None, None, 0, 100, 0, None, 0, None, None, None) == -1
    assert L.tfs_ctable_info(None, None, None, None, None, None) == -1
    assert L.tfs_ctable_free(None) == 0
    assert L.tfs_eval_chirp_batch(None, 1, None) == -1
    assert L.tfs_table_export(None, None, None) == -1
    assert L.tfs_table_import(ctypes.cast(x, P), None, 4, 10, 1.0, 3, ctypes.byref(out)) == -1  # FP8 without scales
    assert L.tfs_table_import(ctypes.cast(x, P), None, 0, 10, 1.0, 0, ctypes.byref(out)) == -1
    assert L.tfs_ctable_view(None, 0, 1, ctypes.byref(out)) == -1
    assert ctypes.sizeof(_lib.TfsChirpJob) == 7 * 8 and _lib.TfsChirpJob.P.offset == 40
    # the search's device draws: fewer than 3 walkers, an empty interval or no counter
    it = (ctypes.c_int32 * 1)()
    assert L.tfs_de_draw(1, ctypes.cast(it, P), 4, 2, 0.3, 1.5, None, None, None, None) == -1
    assert L.tfs_de_draw(1, ctypes.cast(it, P), 4, 8, 1.5, 0.3, None, None, None, None) == -1
    assert L.tfs_de_draw(1, None, 4, 8, 0.3, 1.5, None, None, None, None) == -1
    assert L.tfs_de_draw(1, ctypes.cast(it, P), 4, 8, 0.3, 1.5, None, None, None, None) == -1  # null outputs


def test_tuning_cache_round_trip(L, tmp_path):
    """The tuner's cache: load a JSON object, save it back, reject malformed entries (host only)."""
    src = tmp_path / "tune.json"
    src.write_text('{\n  "0:6:14:9:0": [1024, 2, 4, 16, 0],\n  "1:8:12:12:1": [4096, 1, 8, 2, 2]\n}\n')
    assert L.tfs_tuning_clear() == 0
    assert L.tfs_tuning_load(str(src).encode()) == 0
    out = tmp_path / "out.json"
    assert L.tfs_tuning_save(str(out).encode()) == 0
    import json

    assert json.loads(out.read_text()) == {"0:6:14:9:0": [1024, 2, 4, 16, 0], "1:8:12:12:1": [4096, 1, 8, 2, 2]}
    bad = tmp_path / "bad.json"
    for txt in ('{"0:6:14:9:0": [1024]}', '{"0:6:14:9:0": [1024, 2, 4, 16]}', '{"0:6:14:9:0": [1024, 2, 9, 16, 0]}',
                '{"0:6:14:9:0": [1024, 2, 4, 33, 0]}', '{"0:6:14:9:0": [1024, 2, 4, 32, 3]}'):
        bad.write_text(txt)
        assert L.tfs_tuning_load(str(bad).encode()) == -1
    assert L.tfs_tuning_load(str(tmp_path / "missing.json").encode()) == -6
    assert L.tfs_tuning_clear() == 0
    assert L.tfs_autotune_batch(None, 0, 3, None, None, None, None) == -1
    assert L.tfs_set_wait_limit(0, 2) == -1


def test_server_validation_without_device(L):
    out = ctypes.c_void_p()
    assert L.tfs_server_create(0, 64, ctypes.byref(out)) == -1
    assert L.tfs_server_create(1 << 30, 0, ctypes.byref(out)) == -1
    t = ctypes.c_int64()
    assert L.tfs_server_submit(None, 0, None, None, 10, 0, 0, ctypes.byref(t)) == -1
    assert L.tfs_server_wait(None, 1, 0, None, None, None) == -1
    assert L.tfs_server_get_stats(None, None) == -1
    assert L.tfs_server_free(None) == 0


def test_server_stats_struct_matches_the_header():
    assert ctypes.sizeof(_lib.TfsServerStats) == 10 * 8 + 4 * 8


def test_job_struct_matches_the_header():
    """struct tfs_job: 8-byte fields except m and topk (int32 each), no padding."""
    assert ctypes.sizeof(_lib.TfsJob) == 10 * 8
    assert _lib.TfsJob.flags.offset == 72 and _lib.TfsJob.reserved.offset == 76
    assert _lib.TfsJob.m.offset == 40 and _lib.TfsJob.topk.offset == 44 and _lib.TfsJob.stat.offset == 48


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()


def test_binding_refuses_non_contiguous_arrays():
    """Every pointer the binding hands over must address a row-major array: a transposed view
    (the natural result of a least-squares solve, for example) is refused, not misread."""
    import numpy as np
    import pytest

    from paper_2510_20891_gb300 import _ptr

    a = np.zeros((4, 3))
    _ptr(a)
    with pytest.raises(ValueError):
        _ptr(a.T)
