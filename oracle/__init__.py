"""CPU oracle for applying sequences of planar rotations (Steel & Langou).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2412_01852_gb300``) and imports nothing from it.

The arithmetic lives in ``rot_oracle.c`` (plain C, FP64, ``-ffp-contract=off``,
C99 ``fma``); this module compiles it with gcc on first use and wraps it for
numpy arrays.  Every function returns a new array and leaves its inputs alone.

Functions and the passages they follow:

* ``rot_sequence``            -- Algorithm 2 (rot_sequence), with Algorithm 1 (rot).
* ``rot_sequence_f32``        -- Algorithm 2 in single precision.
* ``rot_sequence_wavefront``  -- Algorithm 3 (rot_sequence_wavefront), corrected reading.
* ``rot_sequence_inverse``    -- the transposed rotations in reverse order.
* ``rot_sequence_block``      -- Algorithm 4 (rot_sequence_block).
* ``form_block``              -- the accumulated orthogonal block of rs_gemm (Section 8).
* ``form_block_f32``          -- the same block accumulated in single precision.
* ``rot_sequence_gemm``       -- Algorithm 2 regrouped into accumulated blocks applied
                                 by FP64 matrix products (rs_gemm, Section 8).
* ``refl_sequence``           -- 2x2 reflectors (tau, nu) in Algorithm 2's order (Section 6).
* ``rot_sequence_left``       -- the rotations applied to rows (Algorithm 2 on A^T).
* ``refl_sequence_reverse``   -- the same reflectors in reverse order (their inverse).

Beside the oracle, ``rot_sequence_parallel`` runs the multi-core CPU baseline
(``rot_cpu_parallel.c``: row blocks over host threads as in Section 7, wave
order inside each block).  It is the timed CPU leg of ``bench.py``, not a
reference for anything; the tests check it bit for bit against the oracle.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` (closed
forms, exact special cases, invariants, BLAS ``drot`` and exact rational
arithmetic); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rot_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librot_oracle.so")
_PAR_SRC = os.path.join(_HERE, "rot_cpu_parallel.c")
_PAR_SO = os.path.join(_BUILD, "librot_cpu_parallel.so")
_par_lib = None
_par_openmp = None
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile rot_oracle.c into oracle/_build/librot_oracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    build_parallel(force)
    return _SO


def build_parallel(force: bool = False) -> str:
    """Compile rot_cpu_parallel.c with OpenMP (or, if the compiler lacks it, without)."""
    global _par_openmp
    os.makedirs(_BUILD, exist_ok=True)
    flag = _PAR_SO + ".openmp"
    if force or not os.path.exists(_PAR_SO) or os.path.getmtime(_PAR_SO) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_SO + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-o", tmp, _PAR_SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
        openmp = r.returncode == 0
        if not openmp:
            subprocess.run(base, check=True)
        os.replace(tmp, _PAR_SO)
        with open(flag, "w") as f:
            f.write("1" if openmp else "0")
    with open(flag) as f:
        _par_openmp = f.read().strip() == "1"
    return _PAR_SO


def _declare(lib):
    """Attach argument types to a loaded oracle library."""
    seq = [_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
    for name in ("oracle_rot_sequence", "oracle_rot_sequence_wavefront",
                 "oracle_rot_sequence_inverse", "oracle_refl_sequence", "oracle_refl_sequence_reverse",
                 "oracle_rot_sequence_left"):
        getattr(lib, name).argtypes = seq
        getattr(lib, name).restype = None
    lib.oracle_rot_sequence_f32.argtypes = [_i64, _i64, _i64, _fp, _i64, _fp, _i64, _fp, _i64]
    lib.oracle_rot_sequence_f32.restype = None
    lib.oracle_rot_sequence_block.argtypes = seq
    lib.oracle_rot_sequence_block.restype = None
    lib.oracle_rot.argtypes = [_i64, _dp, _dp, ctypes.c_double, ctypes.c_double]
    lib.oracle_rot.restype = None
    lib.oracle_form_block.argtypes = [_i64, _i64, _i64, _i64, _i64, _i64,
                                      _dp, _i64, _dp, _i64, _dp, _i64]
    lib.oracle_form_block.restype = None
    lib.oracle_form_block_f32.argtypes = [_i64, _i64, _i64, _i64, _i64, _i64,
                                          _dp, _i64, _dp, _i64, _fp, _i64]
    lib.oracle_form_block_f32.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def use_library(path):
    """Point this module at another build of rot_oracle.c (returns the previous one).

    Only the mutation test uses this: it plants a mistake in a copy of the C
    source and checks that the pins notice.
    """
    global _lib
    with _lock:
        prev = _lib
        _lib = _declare(ctypes.CDLL(path)) if path is not None else None
    return prev


def restore_library(lib):
    global _lib
    with _lock:
        _lib = lib


def _fortran(a, dtype):
    return np.array(a, dtype=dtype, order="F", copy=True)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(A, C, S):
    m, n = A.shape
    if C.shape != S.shape:
        raise ValueError("C and S must have the same shape")
    if n >= 2 and C.shape[0] != n - 1:
        raise ValueError("C must have n-1 rows")
    return m, n, (C.shape[1] if C.ndim == 2 else 0)


def _run_seq(name, A, C, S):
    lib = _load()
    A = _fortran(A, np.float64)
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    m, n, k = _check(A, C, S)
    if m == 0 or n < 2 or k == 0:
        return A
    getattr(lib, name)(m, n, k, _ptr(A, ctypes.c_double), max(1, m),
                       _ptr(C, ctypes.c_double), max(1, n - 1),
                       _ptr(S, ctypes.c_double), max(1, n - 1))
    return A


def rot(x, y, c, s):
    """Algorithm 1 on two vectors; returns (x', y')."""
    lib = _load()
    x = np.array(x, dtype=np.float64, copy=True)
    y = np.array(y, dtype=np.float64, copy=True)
    lib.oracle_rot(x.size, _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), float(c), float(s))
    return x, y


def rot_sequence(A, C, S):
    """Algorithm 2: A * G(0,0) G(1,0) ... G(n-2,k-1), FP64."""
    return _run_seq("oracle_rot_sequence", A, C, S)


def rot_sequence_left(A, C, S):
    """Rotations on rows j, j+1 of A (C, S are (m-1) x k): Algorithm 2 on A^T, transposed back."""
    lib = _load()
    A = _fortran(A, np.float64)
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    m, n = A.shape
    k = C.shape[1] if C.ndim == 2 else 0
    if n == 0 or m < 2 or k == 0:
        return A
    if C.shape[0] != m - 1 or S.shape != C.shape:
        raise ValueError("C and S must be (m-1) x k")
    lib.oracle_rot_sequence_left(m, n, k, _ptr(A, ctypes.c_double), max(1, m),
                                 _ptr(C, ctypes.c_double), max(1, m - 1),
                                 _ptr(S, ctypes.c_double), max(1, m - 1))
    return A


def refl_sequence(A, T, V):
    """2x2 reflectors H = I - tau*v*v^T, v = (1, nu), in Algorithm 2's order (Section 6)."""
    return _run_seq("oracle_refl_sequence", A, T, V)


def refl_sequence_reverse(A, T, V):
    """The same reflectors applied in reverse order."""
    return _run_seq("oracle_refl_sequence_reverse", A, T, V)


def rot_sequence_wavefront(A, C, S):
    """Algorithm 3 (wavefront order); bit-identical to Algorithm 2."""
    return _run_seq("oracle_rot_sequence_wavefront", A, C, S)


def rot_sequence_inverse(A, C, S):
    """Undo Algorithm 2: rotations (c, -s) in reverse order."""
    return _run_seq("oracle_rot_sequence_inverse", A, C, S)


def rot_sequence_f32(A, C, S):
    """Algorithm 2 in single precision (FP32 inputs, fmaf)."""
    lib = _load()
    A = _fortran(A, np.float32)
    C = _fortran(C, np.float32)
    S = _fortran(S, np.float32)
    m, n, k = _check(A, C, S)
    if m == 0 or n < 2 or k == 0:
        return A
    lib.oracle_rot_sequence_f32(m, n, k, _ptr(A, ctypes.c_float), max(1, m),
                                _ptr(C, ctypes.c_float), max(1, n - 1),
                                _ptr(S, ctypes.c_float), max(1, n - 1))
    return A


def rot_sequence_block(A, C, S):
    """Algorithm 4 with its printed loop bounds; A has nn+1 columns, C/S have nn rows."""
    lib = _load()
    A = _fortran(A, np.float64)
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    m = A.shape[0]
    nn, kk = C.shape
    if A.shape[1] < nn + 1:
        raise ValueError("A needs nn+1 columns")
    lib.oracle_rot_sequence_block(m, nn, kk, _ptr(A, ctypes.c_double), max(1, m),
                                  _ptr(C, ctypes.c_double), max(1, nn),
                                  _ptr(S, ctypes.c_double), max(1, nn))
    return A


def form_block(C, S, n, w0, nb, p0, kb):
    """Accumulated (nb+kb)-square orthogonal block for waves [w0, w0+nb) of sequences [p0, p0+kb)."""
    lib = _load()
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    k = C.shape[1] if C.ndim == 2 else 0
    L = nb + kb
    Q = np.zeros((L, L), dtype=np.float64, order="F")
    lib.oracle_form_block(n, k, w0, nb, p0, kb, _ptr(C, ctypes.c_double), max(1, n - 1),
                          _ptr(S, ctypes.c_double), max(1, n - 1), _ptr(Q, ctypes.c_double), L)
    return Q


def form_block_f32(C, S, n, w0, nb, p0, kb):
    """``form_block`` in single precision: (c,s) rounded to FP32, FP32 rotations on the FP32 identity."""
    lib = _load()
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    k = C.shape[1] if C.ndim == 2 else 0
    L = nb + kb
    Q = np.zeros((L, L), dtype=np.float32, order="F")
    lib.oracle_form_block_f32(n, k, w0, nb, p0, kb, _ptr(C, ctypes.c_double), max(1, n - 1),
                              _ptr(S, ctypes.c_double), max(1, n - 1), _ptr(Q, ctypes.c_float), L)
    return Q


def block_schedule(n, k, nb, kb):
    """The (w0, p0) of every accumulated block, in the order they are applied.

    Sequences are split into p-blocks of kb; within one p-block the waves
    w = j + (p - p0) run from 0 to (n-2) + (kb'-1) and are cut into blocks of
    nb consecutive waves, applied in increasing w0 (the blocked order of
    Section 2: block (j_b, p_b) before (j_b + n_b, p_b)).
    """
    out = []
    for p0 in range(0, k, kb):
        kbe = min(kb, k - p0)
        nw = (n - 1) + (kbe - 1)
        for w0 in range(0, nw, nb):
            out.append((w0, p0))
    return out


def rot_sequence_gemm(A, C, S, nb, kb):
    """Algorithm 2 regrouped as rs_gemm does: form each block, multiply it in FP64."""
    A = _fortran(A, np.float64)
    m, n = A.shape
    k = C.shape[1] if n >= 2 else 0
    if m == 0 or n < 2 or k == 0:
        return A
    L = nb + kb
    for (w0, p0) in block_schedule(n, k, nb, kb):
        Q = form_block(C, S, n, w0, nb, p0, kb)
        c0 = w0 - kb + 1
        lo, hi = max(c0, 0), min(c0 + L, n)
        Qs = Q[lo - c0:hi - c0, lo - c0:hi - c0]
        A[:, lo:hi] = A[:, lo:hi] @ Qs
    return A


def _load_parallel():
    global _par_lib
    with _lock:
        if _par_lib is None:
            build()
            lib = ctypes.CDLL(_PAR_SO)
            lib.cpu_rot_sequence_parallel.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64,
                                                      _i64, _i64, ctypes.c_int]
            lib.cpu_rot_sequence_parallel.restype = ctypes.c_int
            _par_lib = lib
    return _par_lib


def rot_sequence_parallel(A, C, S, mb=32, kb=32, threads=0, inplace=False):
    """Multi-core CPU baseline: Algorithm 2's result from row blocks of mb rows on
    `threads` host threads (0: all), kb sequences per pass in wave order.
    Returns (A', threads used).  With inplace=True a Fortran-ordered float64 A
    is updated in place (for timing without a copy)."""
    lib = _load_parallel()
    if not (inplace and isinstance(A, np.ndarray) and A.dtype == np.float64 and A.flags.f_contiguous):
        A = _fortran(A, np.float64)
    C = _fortran(C, np.float64)
    S = _fortran(S, np.float64)
    m, n, k = _check(A, C, S)
    if m == 0 or n < 2 or k == 0:
        return A, 1
    used = lib.cpu_rot_sequence_parallel(m, n, k, _ptr(A, ctypes.c_double), max(1, m),
                                         _ptr(C, ctypes.c_double), max(1, n - 1),
                                         _ptr(S, ctypes.c_double), max(1, n - 1),
                                         int(mb), int(kb), int(threads))
    return A, int(used)


def parallel_uses_openmp():
    """Whether the CPU baseline was compiled with OpenMP."""
    _load_parallel()
    return bool(_par_openmp)
