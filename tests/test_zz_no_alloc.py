"""rot_apply_noalloc: the FP64 path whose scratch is a static device array.

Some callers cannot let a library allocate device memory: applications that
reserve the GPU's memory up front for their own pool (and plugins running in
them), where a cudaMalloc inside the library fails or fragments that pool and
synchronizes the device.  rot_apply_noalloc serves them with a 32 MiB static
scratch array.  This file is named so that pytest collects it last; it checks
the entry point through the C ABI against rot_apply, bit for bit (the FP64
tolerance of every other GPU test), on two calls in a row, and checks that a
call takes no device memory from the allocator.
"""
import ctypes

import numpy as np
import pytest

from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01852_gb300 import _native, build
    build.build()
    return _native.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def _call(lib, fn, A, C, S):
    m, n = A.shape
    k = C.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    return getattr(lib, fn)(m, n, k, A.data_ptr(), A.stride(1), C.data_ptr(), C.stride(1),
                            S.data_ptr(), S.stride(1), stream or None)


def test_noalloc_matches_rot_apply_twice_in_a_row(lib):
    # Two different problems back to back: the second call finds the first
    # call's data in the shared scratch and must clear what it relies on.
    for (m, n, k, seed) in [(300, 257, 40, 11), (129, 500, 17, 12)]:
        A, C, S = wl.problem(m, n, k, seed)
        A1, A2 = _dev(A), _dev(A)
        Cd, Sd = _dev(C), _dev(S)
        assert _call(lib, "rot_apply", A1, Cd, Sd) == 0
        assert _call(lib, "rot_apply_noalloc", A2, Cd, Sd) == 0
        assert lib.rot_device_status() == 0
        a1 = A1.cpu().numpy()
        a2 = A2.cpu().numpy()
        assert np.array_equal(a1.view(np.uint64), a2.view(np.uint64))


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    # n + k large enough that the repacked (c, s) rows exceed 32 MiB; no
    # pointer is dereferenced because the size check comes first.
    p = ctypes.c_void_p(0x1000)
    n, k = 1 << 20, 64
    assert lib.rot_apply_noalloc(32, n, k, p, 32, p, n - 1, p, n - 1, None) == 1


def _cudart():
    """The CUDA runtime as a plain shared library (for memory-pool queries), or None."""
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_noalloc_prepare_then_calls_take_no_device_memory(lib):
    """After the set-up, a call changes neither the free device memory nor the
    default stream-ordered pool (reserved and used bytes)."""
    assert lib.rot_apply_noalloc_prepare() == 0
    assert lib.rot_apply_noalloc_prepare() == 0
    rt = _cudart()
    if rt is None:
        pytest.skip("CUDA runtime library not found for the memory-pool query")
    dev = torch.cuda.current_device()
    A, C, S = wl.problem(257, 300, 33, 21)
    A1, Cd, Sd = _dev(A), _dev(C), _dev(S)
    assert _call(lib, "rot_apply_noalloc", A1, Cd, Sd) == 0   # warm: first launches of the kernels
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    assert rt.cudaMemPoolTrimTo(pool, ctypes.c_size_t(0)) == 0
    torch.cuda.synchronize()

    def snapshot():
        reserved, used = ctypes.c_uint64(), ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0   # ReservedMemCurrent
        assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0       # UsedMemCurrent
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
        return reserved.value, used.value, free.value

    A2 = _dev(A)
    torch.cuda.synchronize()
    before = snapshot()
    assert _call(lib, "rot_apply_noalloc", A2, Cd, Sd) == 0
    torch.cuda.synchronize()
    after = snapshot()
    assert lib.rot_device_status() == 0
    assert after == before, (before, after)
