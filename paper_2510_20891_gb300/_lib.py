"""Loading libtfstat.so and declaring its C signatures (include/tfstat.h)."""
from __future__ import annotations

import ctypes
import os
import re

LIB_PATH = os.environ.get("TFS_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtfstat.so")
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tfstat.h")

_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double

SIGNATURES = {
    "tfs_version": (I, []),
    "tfs_last_error": (ctypes.c_char_p, []),
    "tfs_build_sfts": (I, [P, I64, D, D, I, P, I, I, P, P]),
    "tfs_table_from_power": (I, [P, I64, I64, D, I, I, P, P]),
    "tfs_table_info": (I, [P, P, P, P, P, P]),
    "tfs_table_to_host": (I, [P, P, P]),
    "tfs_table_bytes": (I64, [P]),
    "tfs_table_free": (I, [P]),
    "tfs_build_basis": (I, [P, I64, I64, I, D, I, P, P]),
    "tfs_basis_from_host": (I, [P, I, I64, P]),
    "tfs_basis_info": (I, [P, P, P]),
    "tfs_basis_to_host": (I, [P, P, P, P, P]),
    "tfs_basis_free": (I, [P]),
    "tfs_eval_stat": (I, [P, P, P, P, I64, I, I, P, P, P, P, I, P]),
    "tfs_topk": (I, [P, I64, I, P, P, I, P]),
    "tfs_table_rebuild": (I, [P, P, I64, I, P]),
    "tfs_eval_bins": (I, [P, P, P, P, I64, I, P, I, P]),
    "tfs_kernel_launches": (ctypes.c_longlong, []),
    "tfs_topk_noalloc": (I, [P, I64, I, P, P, P]),
    "tfs_topk_batch": (I, [P, P, P, I, P, P, P]),
    "tfs_eval_batch": (I, [P, I, P, P]),
    "tfs_autotune_batch": (I, [P, I, I, P, P, P, P]),
    "tfs_set_wait_limit": (I, [I64, I]),
    "tfs_tuning_save": (I, [ctypes.c_char_p]),
    "tfs_tuning_load": (I, [ctypes.c_char_p]),
    "tfs_tuning_clear": (I, []),
    "tfs_server_create": (I, [I64, I, P]),
    "tfs_server_add_dataset": (I, [P, P, P, P]),
    "tfs_server_submit": (I, [P, I, P, P, I64, I, I, P]),
    "tfs_server_wait": (I, [P, I64, I, P, P, P]),
    "tfs_server_get_stats": (I, [P, P]),
    "tfs_server_free": (I, [P]),
    "tfs_table_view": (I, [P, I64, I64, P]),
    "tfs_table_export": (I, [P, P, P]),
    "tfs_table_import": (I, [P, P, I64, I64, D, I, P]),
    "tfs_basis_view": (I, [P, I64, I64, P]),
    "tfs_de_propose": (I, [P, I64, I, P, P, P, P, P, P, P, P]),
    "tfs_de_accept": (I, [P, P, P, P, P, I64, I, P]),
    "tfs_de_draw": (I, [ctypes.c_uint64, P, I64, I, ctypes.c_float, ctypes.c_float, P, P, P, P]),
    "tfs_build_chirp_table": (I, [P, I64, D, D, P, I, P, P]),
    "tfs_ctable_view": (I, [P, I64, I64, P]),
    "tfs_eval_chirp_batch": (I, [P, I, P]),
    "tfs_measure_l2_read": (I, [I64, I, P]),
    "tfs_ctable_info": (I, [P, P, P, P, P, P]),
    "tfs_ctable_to_host": (I, [P, P, P]),
    "tfs_ctable_free": (I, [P]),
    "tfs_eval_chirp_stat": (I, [P, P, P, P, I64, I, I, P, I, P, P, P]),
}


class TfsTuning(ctypes.Structure):
    """struct tfs_tuning (include/tfstat.h)."""

    _fields_ = [("pcap", ctypes.c_int32), ("tile_div", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("group", ctypes.c_int32), ("tile_class", ctypes.c_int32)]


class TfsServerStats(ctypes.Structure):
    """struct tfs_server_stats (include/tfstat.h)."""

    _fields_ = [(n, I64) for n in ("submitted", "completed", "failed", "tracks_completed", "evictions", "loads",
                                   "batches", "used_bytes", "resident_bytes", "budget_bytes")] + \
               [(n, ctypes.c_double) for n in ("mean_jobs_per_batch", "p50_ms", "p99_ms", "mean_ms")]


class TfsJob(ctypes.Structure):
    """struct tfs_job (include/tfstat.h): one dataset of a batched statistic launch."""

    _fields_ = [
        ("table", P),
        ("basis", P),
        ("coeffs", P),
        ("f_ref", P),
        ("N", I64),
        ("m", ctypes.c_int32),
        ("topk", ctypes.c_int32),
        ("stat", P),
        ("top_idx", P),
        ("top_val", P),
        ("flags", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


JOB_SEGMENT_CUTS = 1  # TFS_JOB_SEGMENT_CUTS


class TfsChirpJob(ctypes.Structure):
    """struct tfs_chirp_job (include/tfstat.h): one job of a batched linear-chirp launch."""

    _fields_ = [
        ("table", P),
        ("basis", P),
        ("coeffs", P),
        ("f_ref", P),
        ("N", I64),
        ("P", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("stat", P),
    ]

ERR_NAMES = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "BUSY", -6: "NOT_FOUND"}


class TfsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tfstat error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


def header_symbols(path: str = HEADER) -> list[str]:
    """Names of the functions declared in include/tfstat.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tfs_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """The loaded library (raises if it has not been built: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2510_20891_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != 0:
        msg = lib().tfs_last_error()
        raise TfsError(rc, msg.decode() if msg else "")
    return rc
