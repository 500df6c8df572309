"""The packed resident layout (Section 4's pre-packed A): pack / unpack round
trips, and rotations applied to a packed matrix equal rot_apply on the
column-major one bit for bit (rows are independent, every row sees the same
operations), on both kernels the packed entry points use (the column stream
for few sequences, the wavefront kernel otherwise), ragged shapes included.
"""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01852_gb300 import api, build
    build.build()
    return api


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
    return t if dtype is None else t.to(dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n", [(1, 5), (33, 70), (100, 77), (256, 64)])
def test_pack_unpack_round_trip(api, dtype, m, n):
    A = dev(wl.matrix(m, n, seed=m + n), dtype)
    P = api.pack(A)
    assert P.numel() == api.packed_elems(m, n) == -(-m // 32) * 32 * n
    host = P.cpu().numpy()
    a = A.cpu().numpy()
    for i in {0, m - 1, m // 2}:
        for j in {0, n - 1, n // 3}:
            assert host[(i // 32) * 32 * n + j * 32 + i % 32] == a[i, j]
    pad = [(i // 32) * 32 * n + j * 32 + i % 32 for i in range(m, -(-m // 32) * 32) for j in (0, n - 1)]
    assert not host[pad].any()
    B = torch.zeros_like(A).t().contiguous().t()
    api.unpack(P, B)
    torch.cuda.synchronize()
    assert torch.equal(A, B)


def _bits(t):
    return t.cpu().numpy().view(np.uint64 if t.dtype == torch.float64 else np.uint32)


@pytest.mark.parametrize("k", [1, 2, 5, 8, 9, 16, 17, 40])
@pytest.mark.parametrize("m,n", [(300, 257), (130, 100), (64, 64), (33, 70), (97, 500)])
def test_packed_fp64_equals_column_major(api, m, n, k):
    A, C, S = wl.problem(m, n, k, seed=3 * m + n + k)
    Cd, Sd = dev(C), dev(S)
    ref = dev(A)
    api.rot_apply(ref, Cd, Sd)
    P = api.pack(dev(A))
    api.rot_apply_packed(P, m, n, Cd, Sd)
    out = torch.zeros_like(ref).t().contiguous().t()
    api.unpack(P, out)
    torch.cuda.synchronize()
    api.rot_device_status()
    assert np.array_equal(_bits(out), _bits(ref))


@pytest.mark.parametrize("k", [1, 3, 8, 16, 48, 49, 64])
@pytest.mark.parametrize("m,n", [(300, 257), (64, 1030), (33, 70), (200, 64)])
def test_packed_fp32_equals_column_major(api, m, n, k):
    A, C, S = wl.problem(m, n, k, seed=5 * m + n + k)
    Cd, Sd = dev(C, torch.float32), dev(S, torch.float32)
    ref = dev(A, torch.float32)
    api.rot_apply_f32(ref, Cd, Sd)
    P = api.pack(dev(A, torch.float32))
    api.rot_apply_packed(P, m, n, Cd, Sd)
    out = torch.zeros_like(ref).t().contiguous().t()
    api.unpack(P, out)
    torch.cuda.synchronize()
    api.rot_device_status()
    assert np.array_equal(_bits(out), _bits(ref))


def test_packed_fp64_against_oracle_with_signed_zeros(api):
    """Bit-exact against Algorithm 2 directly, with -0 rows and an Inf."""
    m, n, k = 96, 130, 12
    A, C, S = wl.problem(m, n, k, seed=41)
    A[5, :] = -0.0
    A[7, 3] = np.inf
    ref = oracle.rot_sequence(A, C, S)
    P = api.pack(dev(A))
    api.rot_apply_packed(P, m, n, dev(C), dev(S))
    out = dev(np.zeros((m, n)))
    api.unpack(P, out)
    torch.cuda.synchronize()
    got = np.ascontiguousarray(out.cpu().numpy())
    ref = np.ascontiguousarray(ref)
    # Inf meets zero and opposite infinities: NaN in row 7, whose payload is
    # the device's, not the host's; every other entry bit for bit.
    nan = np.isnan(ref)
    assert nan.any() and np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_packed_large_sampled_rows(api):
    """8192 x 8192 FP32, k = 4 (the column stream at full size): sampled rows
    bit-exact against the FP32 oracle."""
    m = n = 8192
    k = 4
    A, C, S = wl.problem(m, n, k, seed=2)
    rows = np.array([0, 31, 32, 4095, 8191])
    ref = oracle.rot_sequence_f32(A[rows].astype(np.float32), C.astype(np.float32), S.astype(np.float32))
    P = api.pack(dev(A, torch.float32))
    api.rot_apply_packed(P, m, n, dev(C, torch.float32), dev(S, torch.float32))
    out = dev(np.zeros((m, n)), torch.float32)
    api.unpack(P, out)
    torch.cuda.synchronize()
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), np.ascontiguousarray(ref).view(np.uint32))
