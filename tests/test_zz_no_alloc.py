"""rot_apply_noalloc: the FP64 path whose scratch is a static device array.

Some callers cannot let a library allocate device memory: applications that
reserve the GPU's memory up front for their own pool (and plugins running in
them), where a cudaMalloc inside the library fails or fragments that pool and
synchronizes the device.  rot_apply_noalloc serves them with a 32 MiB static
scratch array.  This file is named so that pytest collects it last; it checks
the entry point through the C ABI against rot_apply, bit for bit (the FP64
tolerance of every other GPU test), on two calls in a row.
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
