"""ctypes view of the C ABI in include/rotseq.h (argument marshalling only).

The shared library must have been built (``paper_2412_01852_gb300.build.build()``
or ``__graft_entry__.build()``).  There is no fallback: if the library is
missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

i64 = ctypes.c_int64
vp = ctypes.c_void_p
ci = ctypes.c_int
sz = ctypes.c_size_t

# name -> (restype, argtypes); must match include/rotseq.h
SIGNATURES = {
    "rot_version": (ci, []),
    "rot_status_string": (ctypes.c_char_p, [ci]),
    "rot_last_error": (ctypes.c_char_p, []),
    "rot_apply": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_apply_f32": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_device_status": (ci, []),
    "rot_device_code_status": (ci, [ci]),
    "rot_selftest_wait_timeout": (ci, [ci, vp]),
    "rot_apply_host": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_apply_reflectors": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_apply_left": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_apply_noalloc": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "rot_apply_noalloc_prepare": (ci, []),
    "rot_packed_elems": (i64, [i64, i64]),
    "rot_pack": (ci, [i64, i64, vp, i64, vp, vp]),
    "rot_unpack": (ci, [i64, i64, vp, vp, i64, vp]),
    "rot_pack_f32": (ci, [i64, i64, vp, i64, vp, vp]),
    "rot_unpack_f32": (ci, [i64, i64, vp, vp, i64, vp]),
    "rot_apply_packed": (ci, [i64, i64, i64, vp, vp, i64, vp, i64, vp]),
    "rot_apply_packed_f32": (ci, [i64, i64, i64, vp, vp, i64, vp, i64, vp]),
    "rot_trace_start": (ci, []),
    "rot_trace_stop": (ci, [vp, ci, ctypes.POINTER(ci)]),
    "rot_launch_count": (ctypes.c_int64, []),
    "rot_measure_fp64_peak": (ci, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "rot_measure_fp64_mix": (ci, [ci, ci, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "rot_measure_tc_issue": (ci, [ci, ci, ci, ci, ctypes.POINTER(ctypes.c_double)]),
    "rot_batch_plan_create": (ci, [ci, vp, vp, ctypes.POINTER(vp)]),
    "rot_batch_plan_execute": (ci, [vp, vp]),
    "rot_batch_plan_info": (ci, [vp, vp]),
    "rot_batch_plan_destroy": (ci, [vp]),
    "rot_apply_batched": (ci, [ci, vp, vp]),
    "rot_apply_tuned": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp]),
    "rot_batch_autotune": (ci, [ci, vp, vp, vp, ctypes.POINTER(ctypes.c_float)]),
    "rot_form_blocks_count": (i64, [i64, i64, ci, ci]),
    "rot_form_blocks": (ci, [i64, i64, vp, i64, vp, i64, ci, ci, vp, vp]),
    "rot_form_blocks_f32": (ci, [i64, i64, vp, i64, vp, i64, ci, ci, vp, vp]),
    "rot_apply_gemm": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, ci, ci, ci, vp]),
    "rot_apply_gemm_workspace_size": (ci, [i64, i64, i64, ci, ci, ci, ctypes.POINTER(sz)]),
    "rot_apply_gemm_ws": (ci, [i64, i64, i64, vp, i64, vp, i64, vp, i64, ci, ci, ci, vp, sz, vp]),
    "rot_batched_workspace_size": (ci, [ci, vp, ctypes.POINTER(sz)]),
    "rot_apply_batched_ws": (ci, [ci, vp, vp, sz, vp]),
    "rot_server_create": (ci, [vp, ctypes.POINTER(vp)]),
    "rot_server_register": (ci, [vp, i64, i64, vp, i64, ctypes.POINTER(ci)]),
    "rot_server_submit": (ci, [vp, ci, i64, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_uint64)]),
    "rot_server_wait": (ci, [vp, ctypes.c_uint64, ci]),
    "rot_server_wait_latency": (ci, [vp, ctypes.c_uint64, ci, ctypes.POINTER(ctypes.c_double)]),
    "rot_server_stats": (ci, [vp, vp, ci]),
    "rot_server_destroy": (ci, [vp]),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("streams", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_fused_k", ctypes.c_int),
                ("wide_rows", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("inflight", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("mean_batch", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("rotation_rows", ctypes.c_int64), ("busy_s", ctypes.c_double),
                ("rotation_rows_per_s", ctypes.c_double), ("arena_used_bytes", ctypes.c_size_t)]


class Tuning(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("NB", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("fp64_products", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("S", ctypes.c_void_p), ("lds", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int), ("work_items", ctypes.c_int64),
                ("rotation_rows", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
                ("tuning", Tuning)]


class TraceRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ms", ctypes.c_float), ("work", ctypes.c_int64)]


KERNEL_KINDS = {1: "wave_f64", 2: "wave_f32", 3: "wave_batched", 4: "form_blocks", 5: "gemm_apply", 6: "reflect_f64",
                7: "pipe_f32", 8: "pipe_f64"}
GEMM_MODES = {"dmma": 0, "bf16": 1, "f16": 2, "bf16-q32": 3, "f16-q32": 4}


class RotError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        detail = ""
        try:
            detail = load().rot_last_error().decode()
        except Exception:
            pass
        super().__init__("%s%s%s" % (where + ": " if where else "", status_string(code),
                                     " [" + detail + "]" if detail else ""))


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    "the CUDA library %s is not built; run paper_2412_01852_gb300.build.build() "
                    "(there is no CPU fallback)" % path)
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(code) -> str:
    try:
        return load().rot_status_string(int(code)).decode()
    except Exception:
        return "rot_status %d" % int(code)


def check(code, where=""):
    if int(code) != 0:
        raise RotError(code, where)


def header_functions(path=None):
    """Names of the functions declared in include/rotseq.h (used by the ABI test)."""
    if path is None:
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "rotseq.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text)
    return sorted(set(n for n in names if n.startswith("rot_")))
