"""Python binding of the C ABI with the same names, taking torch CUDA tensors.

Only marshalling happens here: shapes, leading dimensions, raw device
pointers and the current CUDA stream are passed to the library; every step of
the computation runs in its kernels.  Matrices are column-major: a tensor of
shape (rows, cols) with stride(0) == 1; ``colmajor`` and ``empty_colmajor``
make such tensors.
"""
from __future__ import annotations

import torch

from . import _native


def empty_colmajor(rows, cols, dtype=torch.float64, device="cuda"):
    """Uninitialised column-major (rows x cols) tensor (leading dimension = rows)."""
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy of a 2-D tensor (same values)."""
    out = empty_colmajor(t.shape[0], t.shape[1], dtype=t.dtype, device=t.device)
    out.copy_(t)
    return out


def _ld(t: torch.Tensor, rows: int) -> int:
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.shape[0] > 1 and t.shape[1] > 1 and t.stride(0) != 1:
        raise ValueError("expected a column-major tensor (stride(0) == 1)")
    if t.shape[1] > 1:
        return max(int(t.stride(1)), max(1, rows))
    return max(1, rows)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes_void(stream.cuda_stream)


def ctypes_void(h):
    return int(h) if h else None


def _ptr(t):
    return t.data_ptr() if t.numel() > 0 else None


def _args(A, C, S, dtype):
    for name, t in (("A", A), ("C", C), ("S", S)):
        if t.dtype != dtype:
            raise TypeError("%s must be %s" % (name, dtype))
        if t.numel() > 0 and not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
    m, n = A.shape
    nm1 = max(n - 1, 0)
    if C.shape != S.shape or (n >= 2 and C.shape[0] != nm1):
        raise ValueError("C and S must both be (n-1) x k")
    k = C.shape[1] if n >= 2 else (C.shape[1] if C.dim() == 2 else 0)
    return (m, n, k, _ptr(A), _ld(A, m), _ptr(C), _ld(C, nm1), _ptr(S), _ld(S, nm1))


def rot_apply(A, C, S, stream=None):
    """Algorithm 2 in FP64 on device tensors, in place on A (column-major)."""
    lib = _native.load()
    _native.check(lib.rot_apply(*_args(A, C, S, torch.float64), _stream_handle(stream)), "rot_apply")
    return A


def rot_apply_f32(A, C, S, stream=None):
    """Algorithm 2 in FP32 on device tensors, in place on A (column-major)."""
    lib = _native.load()
    _native.check(lib.rot_apply_f32(*_args(A, C, S, torch.float32), _stream_handle(stream)),
                  "rot_apply_f32")
    return A


# ---- packed resident layout ------------------------------------------------------

def packed_elems(m, n):
    """Elements of the packed buffer of an m x n matrix (32-row strips)."""
    return int(_native.load().rot_packed_elems(int(m), int(n)))


def pack(A, stream=None):
    """Column-major device tensor A (m x n) -> a new 1-D tensor in the packed
    layout (strip s of 32 rows is a 32 x n column-major panel)."""
    lib = _native.load()
    m, n = A.shape
    P = torch.empty(packed_elems(m, n), dtype=A.dtype, device=A.device)
    fn = lib.rot_pack if A.dtype == torch.float64 else lib.rot_pack_f32
    _native.check(fn(m, n, _ptr(A), _ld(A, m), _ptr(P), _stream_handle(stream)), "rot_pack")
    return P


def unpack(P, A, stream=None):
    """Packed P into the column-major device tensor A (m x n), in place."""
    lib = _native.load()
    m, n = A.shape
    if P.numel() < packed_elems(m, n) or P.dtype != A.dtype:
        raise ValueError("P must hold packed_elems(m, n) elements of A's dtype")
    fn = lib.rot_unpack if A.dtype == torch.float64 else lib.rot_unpack_f32
    _native.check(fn(m, n, _ptr(P), _ptr(A), _ld(A, m), _stream_handle(stream)), "rot_unpack")
    return A


def rot_apply_packed(P, m, n, C, S, stream=None):
    """rot_apply (FP64) or rot_apply_f32 (FP32, by P's dtype) on a packed matrix."""
    lib = _native.load()
    k = C.shape[1] if C.dim() == 2 else 0
    if P.numel() < packed_elems(m, n):
        raise ValueError("P must hold packed_elems(m, n) elements")
    if not P.is_cuda or not C.is_cuda or not S.is_cuda:
        raise ValueError("device tensors expected")
    if C.dtype != P.dtype or S.dtype != P.dtype:
        raise ValueError("C and S must have P's dtype")
    fn = lib.rot_apply_packed if P.dtype == torch.float64 else lib.rot_apply_packed_f32
    _native.check(fn(int(m), int(n), int(k), _ptr(P), _ptr(C), _ld(C, max(1, n - 1)), _ptr(S),
                     _ld(S, max(1, n - 1)), _stream_handle(stream)), "rot_apply_packed")
    return P


def rot_device_status():
    """Synchronize; raise RotError if a kernel recorded a device-side failure."""
    lib = _native.load()
    _native.check(lib.rot_device_status(), "rot_device_status")


def rot_apply_host(A, C, S, stream=None):
    """rot_apply on host numpy arrays (column-major FP64); copies in, runs, copies A back.

    A is updated in place and must be a Fortran-ordered float64 array.
    """
    import numpy as np
    lib = _native.load()
    for name, a in (("A", A), ("C", C), ("S", S)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and
                (a.flags.f_contiguous or a.ndim < 2 or a.shape[0] <= 1)):
            raise TypeError("%s must be a Fortran-ordered float64 numpy array" % name)
    m, n = A.shape
    k = C.shape[1] if C.ndim == 2 else 0
    nm1 = max(n - 1, 1)
    _native.check(lib.rot_apply_host(m, n, k, A.ctypes.data or None, max(1, m),
                                     C.ctypes.data or None, nm1, S.ctypes.data or None, nm1,
                                     _stream_handle(stream)), "rot_apply_host")
    return A


def trace_start():
    _native.check(_native.load().rot_trace_start(), "rot_trace_start")


def trace_stop(capacity=4096):
    """Stop tracing; list of (kernel kind name, ms, rotation-row updates)."""
    import ctypes
    lib = _native.load()
    recs = (_native.TraceRecord * capacity)()
    cnt = ctypes.c_int(0)
    _native.check(lib.rot_trace_stop(ctypes.cast(recs, ctypes.c_void_p), capacity, ctypes.byref(cnt)),
                  "rot_trace_stop")
    return [(_native.KERNEL_KINDS.get(r.kind, str(r.kind)), float(r.ms), int(r.work))
            for r in recs[:min(cnt.value, capacity)]]


def launch_count():
    return int(_native.load().rot_launch_count())


def measure_fp64_peak():
    """(GFLOP/s counting 2 per DFMA, ms per probe launch) on the current device."""
    import ctypes
    g = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    _native.check(_native.load().rot_measure_fp64_peak(ctypes.byref(g), ctypes.byref(ms)),
                  "rot_measure_fp64_peak")
    return g.value, ms.value


FP64_MIX_KINDS = {"dfma": 0, "dmul": 1, "rotation": 2, "rotation_smem": 3, "rotation_fma_smem": 4,
                  "dfma_smem": 5}


def measure_fp64_mix(kind, warps_per_cta, ctas_per_sm):
    """(FP64 lane-operations per second, ms per probe launch) of one register-only
    instruction mix ('dfma', 'dmul', 'rotation', 'rotation_smem') at the given
    launch shape on the current device."""
    import ctypes
    r = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    _native.check(_native.load().rot_measure_fp64_mix(FP64_MIX_KINDS[kind], int(warps_per_cta),
                                                      int(ctas_per_sm), ctypes.byref(r),
                                                      ctypes.byref(ms)), "rot_measure_fp64_mix")
    return r.value, ms.value


def measure_tc_issue(m, n, accumulators, mmas=3000):
    """Mean ns per tcgen05.mma of shape m x n x 16 (BF16) over `accumulators`
    independent accumulators, one issuing thread per SM."""
    import ctypes
    ns = ctypes.c_double(0)
    _native.check(_native.load().rot_measure_tc_issue(int(m), int(n), int(accumulators), int(mmas),
                                                      ctypes.byref(ns)), "rot_measure_tc_issue")
    return ns.value


# ---- batches of independent problems ---------------------------------------------

def _problem_array(problems):
    arr = (_native.Problem * max(len(problems), 1))()
    for i, (A, C, S) in enumerate(problems):
        m, n, k, pa, lda, pc, ldc, ps, lds = _args(A, C, S, torch.float64)
        arr[i] = _native.Problem(m, n, k, pa, lda, pc, ldc, ps, lds)
    return arr


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, dict):
        t = (t.get("K", 0), t.get("NB", 0), t.get("ctas_per_sm", 0), t.get("fp64_products", 0))
    return _native.Tuning(*t)


class BatchPlan:
    """One persistent launch over many independent (A, C, S) problems.

    ``problems`` is a list of (A, C, S) column-major FP64 CUDA tensors.  The
    plan keeps references to them; ``execute`` queues the whole batch on a
    stream (capturable in a CUDA graph).
    """

    def __init__(self, problems, tuning=None):
        import ctypes
        self._lib = _native.load()
        self._keep = list(problems)
        arr = _problem_array(self._keep)
        h = ctypes.c_void_p()
        t = _tuning(tuning)
        _native.check(self._lib.rot_batch_plan_create(
            len(self._keep), ctypes.cast(arr, ctypes.c_void_p),
            ctypes.cast(ctypes.pointer(t), ctypes.c_void_p) if t is not None else None,
            ctypes.byref(h)), "rot_batch_plan_create")
        self._h = h

    def execute(self, stream=None):
        _native.check(self._lib.rot_batch_plan_execute(self._h, _stream_handle(stream)),
                      "rot_batch_plan_execute")

    def info(self):
        import ctypes
        inf = _native.BatchInfo()
        _native.check(self._lib.rot_batch_plan_info(self._h, ctypes.cast(ctypes.pointer(inf), ctypes.c_void_p)),
                      "rot_batch_plan_info")
        return {"problems": inf.problems, "work_items": inf.work_items,
                "rotation_rows": inf.rotation_rows, "workspace_bytes": inf.workspace_bytes,
                "tuning": {"K": inf.tuning.K, "NB": inf.tuning.NB, "ctas_per_sm": inf.tuning.ctas_per_sm,
                           "fp64_products": inf.tuning.fp64_products}}

    def close(self):
        if getattr(self, "_h", None):
            _native.check(self._lib.rot_batch_plan_destroy(self._h), "rot_batch_plan_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rot_apply_batched(problems, stream=None):
    """Apply every problem's rotations (list of (A, C, S)) in one launch; waits for it."""
    import ctypes
    lib = _native.load()
    arr = _problem_array(problems)
    _native.check(lib.rot_apply_batched(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                        _stream_handle(stream)), "rot_apply_batched")


def batched_workspace_size(problems):
    """Device bytes rot_apply_batched_ws needs for this list of (A, C, S)."""
    import ctypes
    lib = _native.load()
    arr = _problem_array(problems)
    n = ctypes.c_size_t(0)
    _native.check(lib.rot_batched_workspace_size(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                                 ctypes.byref(n)), "rot_batched_workspace_size")
    return n.value


def rot_apply_batched_ws(problems, workspace, stream=None):
    """One launch over the problems with caller-owned scratch (a CUDA uint8 tensor); no wait."""
    import ctypes
    lib = _native.load()
    arr = _problem_array(problems)
    _native.check(lib.rot_apply_batched_ws(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                           workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                           _stream_handle(stream)), "rot_apply_batched_ws")


def batch_autotune(problems, stream=None):
    """Time the tiling grid on copies of the batch; returns (tuning dict, ms)."""
    import ctypes
    lib = _native.load()
    arr = _problem_array(problems)
    best = _native.Tuning()
    ms = ctypes.c_float(0)
    _native.check(lib.rot_batch_autotune(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                         _stream_handle(stream),
                                         ctypes.cast(ctypes.pointer(best), ctypes.c_void_p),
                                         ctypes.byref(ms)), "rot_batch_autotune")
    return {"K": best.K, "NB": best.NB, "ctas_per_sm": best.ctas_per_sm,
            "fp64_products": best.fp64_products}, ms.value


# ---- serving -----------------------------------------------------------------------

class Server:
    """Continuous-batching server over resident device matrices (rot_server_* in the C ABI).

    ``register(A)`` takes a column-major FP64 CUDA tensor that stays resident;
    ``submit(handle, C, S)`` takes host numpy arrays ((n-1) x k, FP64) and
    returns a ticket; ``wait(ticket, timeout_ms)`` returns when the request is
    done (raises RotError on failure, including a wait that runs out).
    """

    def __init__(self, hbm_budget_bytes=1 << 30, max_inflight=64, streams=4, max_batch=32, max_fused_k=192,
                 wide_rows=0):
        import ctypes
        self._lib = _native.load()
        cfg = _native.ServerConfig(int(hbm_budget_bytes), int(max_inflight), int(streams), int(max_batch),
                                   int(max_fused_k), int(wide_rows))
        h = ctypes.c_void_p()
        _native.check(self._lib.rot_server_create(ctypes.cast(ctypes.pointer(cfg), ctypes.c_void_p),
                                                  ctypes.byref(h)), "rot_server_create")
        self._h = h
        self._mats = []

    def register(self, A):
        import ctypes
        m, n = A.shape
        h = ctypes.c_int(-1)
        _native.check(self._lib.rot_server_register(self._h, m, n, A.data_ptr(), _ld(A, m),
                                                    ctypes.byref(h)), "rot_server_register")
        self._mats.append(A)  # keep the tensor alive while the server may use it
        return h.value

    def submit(self, handle, C, S):
        import ctypes
        import numpy as np
        C = np.asfortranarray(C, dtype=np.float64)
        S = np.asfortranarray(S, dtype=np.float64)
        if C.shape != S.shape or C.ndim != 2:
            raise ValueError("C and S must be (n-1) x k arrays")
        t = ctypes.c_uint64(0)
        _native.check(self._lib.rot_server_submit(self._h, int(handle), C.shape[1], C.ctypes.data,
                                                  max(1, C.shape[0]), S.ctypes.data, max(1, S.shape[0]),
                                                  ctypes.byref(t)), "rot_server_submit")
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        _native.check(self._lib.rot_server_wait(self._h, int(ticket), int(timeout_ms)), "rot_server_wait")

    def wait_latency(self, ticket, timeout_ms=-1):
        """wait(); returns the request's submit-to-completion latency in ms."""
        import ctypes
        ms = ctypes.c_double(0)
        _native.check(self._lib.rot_server_wait_latency(self._h, int(ticket), int(timeout_ms), ctypes.byref(ms)),
                      "rot_server_wait_latency")
        return ms.value

    def try_wait(self, ticket, timeout_ms=0):
        """Status code of the wait (0 = done and ok) instead of raising."""
        return int(self._lib.rot_server_wait(self._h, int(ticket), int(timeout_ms)))

    def stats(self, reset=False):
        import ctypes
        st = _native.ServerStats()
        _native.check(self._lib.rot_server_stats(self._h, ctypes.cast(ctypes.pointer(st), ctypes.c_void_p),
                                                 1 if reset else 0), "rot_server_stats")
        return {f: getattr(st, f) for f, _ in _native.ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _native.check(self._lib.rot_server_destroy(self._h), "rot_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- accumulated blocks (rs_gemm) ----------------------------------------------------

def form_blocks_count(n, k, nb, kb):
    return int(_native.load().rot_form_blocks_count(int(n), int(k), int(nb), int(kb)))


def rot_form_blocks(n, C, S, nb, kb, stream=None):
    """All accumulated blocks (FP64): a (nblk, L, L) tensor whose [b] is Q_b transposed.

    The library writes each L x L block column-major; viewed as a C-ordered
    (L, L) array that is Q_b^T, so ``Q[b].T`` is Q_b.
    """
    lib = _native.load()
    k = C.shape[1]
    nblk = form_blocks_count(n, k, nb, kb)
    L = nb + kb
    Q = torch.empty((max(nblk, 1), L, L), dtype=torch.float64, device=C.device)
    _native.check(lib.rot_form_blocks(int(n), int(k), _ptr(C), _ld(C, n - 1), _ptr(S), _ld(S, n - 1),
                                      int(nb), int(kb), Q.data_ptr(), _stream_handle(stream)),
                  "rot_form_blocks")
    return Q[:nblk]


def rot_form_blocks_f32(n, C, S, nb, kb, stream=None):
    """All accumulated blocks formed in FP32: a (nblk, L, L) float32 tensor whose [b] is Q_b transposed."""
    lib = _native.load()
    k = C.shape[1]
    nblk = form_blocks_count(n, k, nb, kb)
    L = nb + kb
    Q = torch.empty((max(nblk, 1), L, L), dtype=torch.float32, device=C.device)
    _native.check(lib.rot_form_blocks_f32(int(n), int(k), _ptr(C), _ld(C, n - 1), _ptr(S), _ld(S, n - 1),
                                          int(nb), int(kb), Q.data_ptr(), _stream_handle(stream)),
                  "rot_form_blocks_f32")
    return Q[:nblk]


def rot_apply_gemm(A, C, S, nb=256, kb=64, mode="f16", stream=None):
    """Algorithm 2 via accumulated blocks and tensor-core products (mode: dmma, bf16, f16)."""
    lib = _native.load()
    m, n, k, pa, lda, pc, ldc, ps, lds = _args(A, C, S, torch.float64)
    _native.check(lib.rot_apply_gemm(m, n, k, pa, lda, pc, ldc, ps, lds, int(nb), int(kb),
                                     _native.GEMM_MODES[mode], _stream_handle(stream)), "rot_apply_gemm")
    return A


def gemm_workspace_size(m, n, k, nb=256, kb=64, mode="f16"):
    """Device bytes rot_apply_gemm_ws needs (host-only query)."""
    import ctypes
    lib = _native.load()
    out = ctypes.c_size_t(0)
    _native.check(lib.rot_apply_gemm_workspace_size(int(m), int(n), int(k), int(nb), int(kb),
                                                    _native.GEMM_MODES[mode], ctypes.byref(out)),
                  "rot_apply_gemm_workspace_size")
    return out.value


def rot_apply_gemm_ws(A, C, S, workspace, nb=256, kb=64, mode="f16", stream=None):
    """rot_apply_gemm with caller-owned scratch (a CUDA uint8 tensor of gemm_workspace_size bytes)."""
    lib = _native.load()
    m, n, k, pa, lda, pc, ldc, ps, lds = _args(A, C, S, torch.float64)
    _native.check(lib.rot_apply_gemm_ws(m, n, k, pa, lda, pc, ldc, ps, lds, int(nb), int(kb),
                                        _native.GEMM_MODES[mode], workspace.data_ptr(),
                                        workspace.numel() * workspace.element_size(), _stream_handle(stream)),
                  "rot_apply_gemm_ws")
    return A


def rot_apply_tuned(A, C, S, tuning=None, stream=None):
    """rot_apply with an explicit tiling dict {K, NB, ctas_per_sm} (same result for every tiling)."""
    import ctypes
    lib = _native.load()
    t = _tuning(tuning)
    _native.check(lib.rot_apply_tuned(*_args(A, C, S, torch.float64),
                                      ctypes.cast(ctypes.pointer(t), ctypes.c_void_p) if t is not None else None,
                                      _stream_handle(stream)), "rot_apply_tuned")
    return A


def rot_apply_reflectors(A, T, V, stream=None):
    """2x2 reflectors (tau = T, nu = V) in Algorithm 2's order, FP64, in place on A."""
    lib = _native.load()
    _native.check(lib.rot_apply_reflectors(*_args(A, T, V, torch.float64), _stream_handle(stream)),
                  "rot_apply_reflectors")
    return A


def rot_apply_left(A, C, S, stream=None):
    """Rotations on rows j, j+1 of A (column-major m x n); C, S are (m-1) x k device tensors."""
    lib = _native.load()
    for name, t in (("A", A), ("C", C), ("S", S)):
        if t.dtype != torch.float64:
            raise TypeError("%s must be float64" % name)
    m, n = A.shape
    mm1 = max(m - 1, 0)
    if C.shape != S.shape or (m >= 2 and C.shape[0] != mm1):
        raise ValueError("C and S must both be (m-1) x k")
    k = C.shape[1]
    _native.check(lib.rot_apply_left(m, n, k, _ptr(A), _ld(A, m), _ptr(C), _ld(C, mm1), _ptr(S), _ld(S, mm1),
                                     _stream_handle(stream)), "rot_apply_left")
    return A
