"""CPU-side checks of the C ABI: the library builds, loads, exports every
declared symbol, and rejects bad arguments before touching the device."""
import ctypes

import pytest

from paper_2412_01852_gb300 import _native, build as _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _native.load()


def test_exports_every_declared_symbol(lib):
    names = _native.header_functions()
    assert "rot_apply" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a binding signature and vice versa
    assert sorted(_native.SIGNATURES) == names


def test_status_strings(lib):
    for code in range(7):
        s = lib.rot_status_string(code).decode()
        assert s.startswith("ROT_")
    assert lib.rot_version() >= 100


P = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails or returns early


@pytest.mark.parametrize("fn", ["rot_apply", "rot_apply_f32"])
@pytest.mark.parametrize("args,code", [
    ((-1, 4, 2, P, 1, P, 3, P, 3), 1),     # m < 0
    ((4, -1, 2, P, 4, P, 1, P, 1), 1),     # n < 0
    ((4, 4, -2, P, 4, P, 3, P, 3), 1),     # k < 0
    ((4, 4, 2, P, 3, P, 3, P, 3), 1),      # lda < m
    ((4, 4, 2, P, 4, P, 2, P, 3), 1),      # ldc < n-1
    ((4, 4, 2, P, 4, P, 3, P, 2), 1),      # lds < n-1
    ((4, 4, 2, None, 4, P, 3, P, 3), 1),   # NULL A with work
    ((4, 4, 2, P, 4, None, 3, P, 3), 1),   # NULL C with work
    ((2**31, 4, 2, P, 2**31, P, 3, P, 3), 1),  # m beyond the limit
    ((0, 4, 2, None, 1, None, 3, None, 3), 0),   # m == 0: quick return
    ((4, 1, 2, None, 4, None, 1, None, 1), 0),   # n == 1: quick return
    ((4, 4, 0, None, 4, None, 3, None, 3), 0),   # k == 0: quick return
])
def test_validation_and_quick_return(lib, fn, args, code):
    assert getattr(lib, fn)(*args, None) == code


def test_batch_plan_rejects_invalid_problems(lib):
    """Invalid problems fail the whole plan before any device work."""
    from paper_2412_01852_gb300 import _native as nat
    arr = (nat.Problem * 3)()
    arr[0] = nat.Problem(4, 4, 2, 0x1000, 4, 0x1000, 3, 0x1000, 3)
    arr[1] = nat.Problem(4, 4, 2, 0x1000, 3, 0x1000, 3, 0x1000, 3)   # lda < m
    arr[2] = nat.Problem(0, 4, 2, 0, 1, 0, 3, 0, 3)                  # quick return
    h = ctypes.c_void_p()
    assert lib.rot_batch_plan_create(3, ctypes.cast(arr, ctypes.c_void_p), None, ctypes.byref(h)) == 1
    assert lib.rot_batch_plan_create(-1, None, None, ctypes.byref(h)) == 1
    assert lib.rot_batch_plan_create(1, None, None, ctypes.byref(h)) == 1
    bad = nat.Tuning(17, 64, 0, 0)
    arr2 = (nat.Problem * 1)()
    arr2[0] = nat.Problem(4, 4, 2, 0x1000, 4, 0x1000, 3, 0x1000, 3)
    assert lib.rot_batch_plan_create(1, ctypes.cast(arr2, ctypes.c_void_p),
                                     ctypes.cast(ctypes.pointer(bad), ctypes.c_void_p),
                                     ctypes.byref(h)) == 1
    assert lib.rot_batch_plan_destroy(None) == 0


def test_server_argument_checks_without_device(lib):
    from paper_2412_01852_gb300 import _native as nat
    h = ctypes.c_void_p()
    cfg = nat.ServerConfig(1000, 4, 2, 4)          # budget below 1 MiB
    assert lib.rot_server_create(ctypes.cast(ctypes.pointer(cfg), ctypes.c_void_p), ctypes.byref(h)) == 1
    cfg = nat.ServerConfig(1 << 30, 0, 2, 4)       # no request slots
    assert lib.rot_server_create(ctypes.cast(ctypes.pointer(cfg), ctypes.c_void_p), ctypes.byref(h)) == 1
    cfg = nat.ServerConfig(1 << 30, 4, 65, 4)      # too many streams
    assert lib.rot_server_create(ctypes.cast(ctypes.pointer(cfg), ctypes.c_void_p), ctypes.byref(h)) == 1
    cfg = nat.ServerConfig(1 << 30, 4, 2, 4, -1)   # negative fusion limit
    assert lib.rot_server_create(ctypes.cast(ctypes.pointer(cfg), ctypes.c_void_p), ctypes.byref(h)) == 1
    assert lib.rot_server_create(None, ctypes.byref(h)) == 1
    t = ctypes.c_uint64()
    assert lib.rot_server_submit(None, 0, 4, None, 1, None, 1, ctypes.byref(t)) == 1
    assert lib.rot_server_wait(None, 1, 0) == 1
    assert lib.rot_server_wait_latency(None, 1, 0, None) == 1
    assert lib.rot_server_destroy(None) == 0


def test_tc_issue_probe_argument_checks_without_device(lib):
    d = ctypes.c_double(0)
    for args in [(32, 160, 2, 100), (64, 8, 1, 100), (64, 168, 1, 100), (128, 272, 1, 100),
                 (64, 160, 4, 100), (64, 160, 0, 100), (64, 160, 2, 0), (64, 160, 2, (1 << 20) + 1)]:
        assert lib.rot_measure_tc_issue(*args, ctypes.byref(d)) == 1, args
    assert lib.rot_measure_tc_issue(64, 160, 2, 100, None) == 1


def test_form_blocks_f32_arguments_checked_on_the_host(lib):
    """Bad arguments of rot_form_blocks_f32 are refused before any device call."""
    assert lib.rot_form_blocks_f32(300, 40, P, 299, P, 299, 64, 16, None, None) == 1             # no Q
    assert lib.rot_form_blocks_f32(300, 40, P, 299, P, 299, 64, 16, ctypes.c_void_p(0x1004), None) == 1
    assert lib.rot_form_blocks_f32(300, 200, P, 299, P, 299, 16, 144, P, None) == 1             # kb > 128
    assert lib.rot_form_blocks_f32(300, 40, P, 299, P, 299, 60, 16, P, None) == 1               # nb % 16
    assert lib.rot_form_blocks_f32(300, 40, P, 10, P, 299, 64, 16, P, None) == 1                # ldc
    assert lib.rot_form_blocks_f32(1, 40, P, 1, P, 1, 64, 16, P, None) == 0                     # no blocks
    assert lib.rot_form_blocks_count(300, 40, 64, 16) == len(
        [(w0, p0) for p0 in range(0, 40, 16) for w0 in range(0, 299 + min(16, 40 - p0) - 1, 64)])


def test_workspace_size_queries_are_host_only(lib):
    """Workspace sizes for the caller-owned-scratch entry points need no device."""
    sz = ctypes.c_size_t(0)
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 1, ctypes.byref(sz)) == 0
    small = sz.value
    assert small > 0
    assert lib.rot_apply_gemm_workspace_size(100, 600, 40, 64, 16, 1, ctypes.byref(sz)) == 0
    assert sz.value > small                                   # more blocks, more scratch
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 0, ctypes.byref(sz)) == 0
    assert 0 < sz.value < small                               # DMMA keeps no split copies
    assert lib.rot_apply_gemm_workspace_size(0, 300, 40, 64, 16, 1, ctypes.byref(sz)) == 0 and sz.value == 0
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 60, 16, 1, ctypes.byref(sz)) == 1   # nb % 16
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 7, ctypes.byref(sz)) == 1   # mode
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 5, ctypes.byref(sz)) == 1   # mode
    # FP32-formed blocks: FP32 blocks plus a (c,s) table instead of the FP64 blocks
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 3, ctypes.byref(sz)) == 0
    assert 0 < sz.value < small
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 4, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.rot_apply_gemm_workspace_size(100, 600, 200, 16, 128, 3, ctypes.byref(sz)) == 0
    assert lib.rot_apply_gemm_workspace_size(100, 600, 200, 16, 144, 3, ctypes.byref(sz)) == 1  # kb > 128
    assert lib.rot_apply_gemm_workspace_size(100, 600, 200, 16, 144, 1, ctypes.byref(sz)) == 0
    assert lib.rot_apply_gemm_workspace_size(100, 300, 40, 64, 16, 1, None) == 1
    # a too-small or misaligned caller workspace is refused before any device call
    assert lib.rot_apply_gemm_ws(100, 300, 40, P, 100, P, 299, P, 299, 64, 16, 1, P, 16, None) == 1
    assert lib.rot_apply_gemm_ws(100, 300, 40, P, 100, P, 299, P, 299, 64, 16, 1,
                                 ctypes.c_void_p(0x1008), small, None) == 1
    arr = (_native.Problem * 2)()
    for i, (m, n, k) in enumerate([(64, 100, 7), (33, 40, 3)]):
        arr[i].m, arr[i].n, arr[i].k = m, n, k
        arr[i].A, arr[i].C, arr[i].S = 0x1000, 0x1000, 0x1000
        arr[i].lda, arr[i].ldc, arr[i].lds = m, n - 1, n - 1
    assert lib.rot_batched_workspace_size(2, ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(sz)) == 0
    assert sz.value > 0
    assert lib.rot_batched_workspace_size(0, None, ctypes.byref(sz)) == 0 and sz.value == 0
    assert lib.rot_apply_batched_ws(2, ctypes.cast(arr, ctypes.c_void_p), P, 16, None) == 1


def test_device_codes_map_to_distinct_statuses(lib):
    """A device status word maps to ROT_ETIMEOUT only for the bounded waits;
    an internal error (a work item decoded outside the problem) is ROT_ECUDA
    and rot_last_error() names it."""
    assert lib.rot_device_code_status(0) == 0
    assert lib.rot_device_code_status(1) == 4
    assert b"wait" in lib.rot_last_error()
    assert lib.rot_device_code_status(2) == 4
    assert lib.rot_device_code_status(3) == 2
    assert b"work item" in lib.rot_last_error()
    assert lib.rot_device_code_status(4) == 2
    assert lib.rot_device_code_status(99) == 2
    assert b"99" in lib.rot_last_error()


def test_fp64_mix_probe_argument_checks_without_device(lib):
    d = ctypes.c_double(0)
    for args in [(-1, 8, 1), (6, 8, 1), (0, 0, 1), (0, 33, 1), (0, 8, 0), (0, 32, 3)]:
        assert lib.rot_measure_fp64_mix(*args, ctypes.byref(d), None) == 1, args
    assert lib.rot_measure_fp64_mix(0, 8, 2, None, None) == 1


def test_packed_layout_arguments_checked_on_the_host(lib):
    """Sizes of the packed layout and argument checks before any device call."""
    assert lib.rot_packed_elems(100, 7) == 128 * 7
    assert lib.rot_packed_elems(32, 5) == 32 * 5
    assert lib.rot_packed_elems(0, 5) == 0
    assert lib.rot_packed_elems(-1, 5) == -1
    assert lib.rot_pack(10, 4, P, 5, P, None) == 1          # lda < m
    assert lib.rot_pack(10, 4, None, 10, P, None) == 1      # no A
    assert lib.rot_unpack(10, 4, P, None, 10, None) == 1    # no A
    assert lib.rot_pack(0, 4, None, 1, None, None) == 0     # nothing to do
    assert lib.rot_apply_packed(10, 4, 2, None, P, 3, P, 3, None) == 1
    assert lib.rot_apply_packed(10, 4, 2, P, P, 2, P, 3, None) == 1   # ldc < n-1
    assert lib.rot_apply_packed(10, 1, 2, None, None, 1, None, 1, None) == 0
    assert lib.rot_apply_packed_f32(-1, 4, 2, P, P, 3, P, 3, None) == 1
    assert lib.rot_apply_packed_f32(10, 4, 0, None, None, 3, None, 3, None) == 0
