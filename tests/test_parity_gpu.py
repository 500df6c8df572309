"""GPU parity of the wavefront kernels against the CPU oracle, through the C ABI.

FP64: bit-exact against ``oracle.rot_sequence`` (same FMA placement).
FP32: bit-exact against ``oracle.rot_sequence_f32``, and within 8*k*2^-24
per-row relative error of the FP64 oracle.
Inputs are seeded synthetic data (``paper_2412_01852_gb300.workloads``).
"""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
NAN_GUARD = np.float64(np.nan)


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import build
    build.build()
    return rs


def to_dev(a, ld=None, fill=np.nan):
    """Column-major device copy of a 2-D numpy array with leading dimension ld.

    Rows ld > rows are padding, filled with `fill` so that a stray write shows.
    Returns (view of the logical matrix, full padded buffer)."""
    rows, cols = a.shape
    ld = max(rows, 1) if ld is None else ld
    buf = np.full((ld, max(cols, 1)), fill, dtype=a.dtype, order="F")
    buf[:rows, :cols] = a
    t = torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()  # (ld, cols) column-major
    return t[:rows, :cols], t


def bits(x):
    x = np.ascontiguousarray(x)
    return x.view(np.uint64 if x.dtype == np.float64 else np.uint32)


SHAPES = [
    (1, 2, 1), (32, 2, 1), (33, 17, 5), (100, 77, 21), (64, 16, 16), (50, 10, 40),
    (31, 3, 33), (5, 200, 3), (257, 130, 17), (64, 300, 48), (96, 64, 1), (7, 1000, 2),
    (40, 66, 64), (130, 129, 100),
]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_f64_bit_exact(rs, m, n, k):
    A, C, S = wl.problem(m, n, k, seed=m * 7 + n * 3 + k)
    A[0, 0] = -0.0
    A[m - 1, n - 1] = -0.0
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = to_dev(A)
    Cd, _ = to_dev(C)
    Sd, _ = to_dev(S)
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(ref))


@pytest.mark.parametrize("m,n,k,lda,ldc", [(10, 40, 7, 13, 41), (33, 21, 30, 64, 23),
                                           (1, 9, 9, 5, 9), (70, 50, 16, 71, 51)])
def test_f64_leading_dimensions_and_guard_rows(rs, m, n, k, lda, ldc):
    """lda > m and odd ldc: the result is bit-exact and padding rows stay untouched."""
    A, C, S = wl.problem(m, n, k, seed=99 + m)
    ref = oracle.rot_sequence(A, C, S)
    Ad, Abuf = to_dev(A, lda)
    Cd, _ = to_dev(C, ldc)
    Sd, _ = to_dev(S, ldc + 2)
    before = Abuf.cpu().numpy().copy()
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    after = Abuf.cpu().numpy()
    assert np.array_equal(bits(after[:m]), bits(ref))
    assert np.array_equal(bits(after[m:]), bits(before[m:]))


def test_f64_plain_512_config(rs):
    """A 512 x 512 N(0,1), C/S 511 x 16 from uniform angles, seed 1."""
    cfg = wl.WORKLOADS["plain-512"]
    A, C, S = wl.problem(cfg["m"], cfg["n"], cfg["k"], seed=cfg["seed"])
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = to_dev(A)
    Cd, _ = to_dev(C)
    Sd, _ = to_dev(S)
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(ref))


def test_f64_special_values(rs):
    """Exact signed swaps, signed zeros, and an Inf that must stay confined to its row."""
    m, n, k = 40, 30, 12
    r = np.random.default_rng(5)
    exact = [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0)]
    idx = r.integers(0, 4, size=(n - 1, k))
    C = np.array([[exact[i][0] for i in row] for row in idx])
    S = np.array([[exact[i][1] for i in row] for row in idx])
    A = r.integers(-5, 6, size=(m, n)).astype(np.float64)
    A[A == 0] = -0.0
    A[3, 4] = np.inf
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = to_dev(A)
    Cd, _ = to_dev(C)
    Sd, _ = to_dev(S)
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    out = Ad.cpu().numpy()
    # 0*Inf makes NaNs; their bit patterns are platform-specific, their places are not.
    nan = np.isnan(ref)
    assert nan.any() and np.array_equal(np.isnan(out), nan)
    assert not np.isnan(np.delete(ref, 3, axis=0)).any()
    assert np.array_equal(bits(out[~nan]), bits(ref[~nan]))


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_f32_bit_exact_and_error_bound(rs, m, n, k):
    A, C, S = wl.problem(m, n, k, seed=m * 5 + n + k)
    A32, C32, S32 = A.astype(np.float32), C.astype(np.float32), S.astype(np.float32)
    ref32 = oracle.rot_sequence_f32(A32, C32, S32)
    ref64 = oracle.rot_sequence(A, C, S)
    Ad, _ = to_dev(A32)
    Cd, _ = to_dev(C32)
    Sd, _ = to_dev(S32)
    rs.rot_apply_f32(Ad, Cd, Sd)
    rs.rot_device_status()
    out = Ad.cpu().numpy()
    assert np.array_equal(bits(out), bits(ref32))
    rel = np.linalg.norm(out.astype(np.float64) - ref64, axis=1) / np.linalg.norm(ref64, axis=1)
    assert rel.max() <= 8 * k * U32


@pytest.mark.parametrize("m,n,k", [(1000, 2000, 40), (4100, 700, 37), (129, 1500, 16)])
def test_f32_many_items_bit_exact(rs, m, n, k):
    """FP32 over many work items per chain: columns handed between items and
    tiles, several p-blocks in flight, a ragged last chain and wave-block."""
    A, C, S = wl.problem(m, n, k, seed=m + n + 11 * k)
    A32, C32, S32 = A.astype(np.float32), C.astype(np.float32), S.astype(np.float32)
    ref32 = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, _ = to_dev(A32)
    Cd, _ = to_dev(C32)
    Sd, _ = to_dev(S32)
    rs.rot_apply_f32(Ad, Cd, Sd)
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(ref32))


@pytest.mark.parametrize("products", [1, 2])
@pytest.mark.parametrize("m,n,k", [(100, 77, 21), (257, 130, 17), (64, 300, 48), (33, 17, 5)])
def test_f64_products_on_either_pipe_bit_exact(rs, m, n, k, products):
    """FP64 products on DMUL (1) or on the integer pipe (2): the same bits as the oracle."""
    from paper_2412_01852_gb300 import api
    A, C, S = wl.problem(m, n, k, seed=m + 3 * n + 7 * k)
    A[2 % m, 3] = 0.0          # zero entries take the DMUL fallback of the integer path
    A[m - 1, 0] = 5e-310       # a subnormal entry as well
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = to_dev(A)
    Cd, _ = to_dev(C)
    Sd, _ = to_dev(S)
    api.rot_apply_tuned(Ad, Cd, Sd, {"fp64_products": products})
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(ref))


def test_f64_paper_shaped_8192_sampled_rows(rs):
    """A 8192 x 8192, k = 192 (the measured workload), checked on sampled rows.

    Rows are independent (the same rotations act on every row), so the oracle
    run on a subset of rows must equal those rows of the full result bit for bit.
    """
    cfg = wl.WORKLOADS["plain-8192"]
    m, n, k = cfg["m"], cfg["n"], cfg["k"]
    A, C, S = wl.problem(m, n, k, seed=cfg["seed"])
    r = np.random.default_rng(77)
    rows = np.unique(np.concatenate([[0, 31, 32, m - 1], r.choice(m, 28, replace=False)]))
    ref = oracle.rot_sequence(A[rows], C, S)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    Cd = torch.from_numpy(np.ascontiguousarray(C.T)).cuda().t()
    Sd = torch.from_numpy(np.ascontiguousarray(S.T)).cuda().t()
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(bits(out), bits(ref))
    # every row keeps its 2-norm (orthogonality), checked on the whole matrix
    n0 = torch.from_numpy(np.linalg.norm(A, axis=1)).cuda()
    n1 = torch.linalg.norm(Ad, dim=1)
    assert float(((n1 - n0).abs() / n0).max()) <= 8 * k * 2.0 ** -53 * 4


def _sample_rows(m, seed):
    r = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, 31, 32, 63, 64, m - 1], r.choice(m, 26, replace=False)]))


def test_f32_precision_8192_sampled_rows(rs):
    """The FP32 workload the bench times (A 8192 x 8192, k = 192, C/S rounded
    to FP32), in its launch configuration: sampled rows bit-exact against the
    FP32 oracle (rows are independent), and every row within 8*k*2^-24 of
    the FP64 oracle's row on the sample."""
    cfg = wl.WORKLOADS["precision-8192"]
    m, n, k = cfg["m"], cfg["n"], cfg["k"]
    A, C, S = wl.problem(m, n, k, seed=cfg["seed"])
    A32, C32, S32 = A.astype(np.float32), C.astype(np.float32), S.astype(np.float32)
    rows = _sample_rows(m, 78)
    ref32 = oracle.rot_sequence_f32(A32[rows], C32, S32)
    ref64 = oracle.rot_sequence(A[rows], C, S)
    Ad = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().t()
    Cd = torch.from_numpy(np.ascontiguousarray(C32.T)).cuda().t()
    Sd = torch.from_numpy(np.ascontiguousarray(S32.T)).cuda().t()
    rs.rot_apply_f32(Ad, Cd, Sd)
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(bits(out), bits(ref32))
    rel = np.linalg.norm(out.astype(np.float64) - ref64, axis=1) / np.linalg.norm(ref64, axis=1)
    assert rel.max() <= 8 * k * U32


def test_reflectors_8192_sampled_rows(rs):
    """The reflector workload the bench times (A 8192 x 8192, k = 192):
    sampled rows bit-exact against the reflector oracle."""
    from paper_2412_01852_gb300 import api
    cfg = wl.WORKLOADS["plain-8192"]
    m, n, k = cfg["m"], cfg["n"], cfg["k"]
    A = wl.matrix(m, n, cfg["seed"])
    T, V = wl.reflectors(n, k, cfg["seed"])
    rows = _sample_rows(m, 79)
    ref = oracle.refl_sequence(A[rows], T, V)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    Td = torch.from_numpy(np.ascontiguousarray(T.T)).cuda().t()
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda().t()
    api.rot_apply_reflectors(Ad, Td, Vd)
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(bits(out), bits(ref))


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_reflectors_bit_exact(rs, m, n, k):
    from paper_2412_01852_gb300 import api
    A = wl.matrix(m, n, seed=m + n + k)
    T, V = wl.reflectors(n, k, seed=m * 3 + k)
    ref = oracle.refl_sequence(A, T, V)
    Ad, _ = to_dev(A)
    Td, _ = to_dev(T)
    Vd, _ = to_dev(V)
    api.rot_apply_reflectors(Ad, Td, Vd)
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(ref))


@pytest.mark.parametrize("m,n,k,lda", [(2, 3, 1, 2), (77, 100, 21, 77), (130, 257, 17, 131),
                                       (300, 64, 48, 301), (17, 1, 5, 17), (64, 2000, 3, 64)])
def test_left_application_bit_exact(rs, m, n, k, lda):
    from paper_2412_01852_gb300 import api
    A = wl.matrix(m, n, seed=m + n)
    C, S = wl.rotations(m, k, seed=k + 5)
    ref = oracle.rot_sequence_left(A, C, S)
    Ad, Abuf = to_dev(A, lda)
    Cd, _ = to_dev(C)
    Sd, _ = to_dev(S)
    before = Abuf.cpu().numpy().copy()
    api.rot_apply_left(Ad, Cd, Sd)
    rs.rot_device_status()
    after = Abuf.cpu().numpy()
    assert np.array_equal(bits(after[:m]), bits(ref))
    assert np.array_equal(bits(after[m:]), bits(before[m:]))


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("m,n,k", [(100, 77, 21), (257, 530, 40), (33, 9, 5), (64, 1000, 3), (300, 2000, 70)])
def test_host_buffers_overlapped_copies_bit_exact(rs, m, n, k, pinned):
    """rot_apply_host: A streamed in by column chunks while the kernel runs and
    copied back as the last p-block finishes each chunk; same bits as the oracle."""
    from paper_2412_01852_gb300 import api
    A, C, S = wl.problem(m, n, k, seed=m + 2 * n + 3 * k)
    ref = oracle.rot_sequence(A, C, S)

    def host(x):
        if not pinned:
            return np.asfortranarray(x.copy())
        t = torch.empty((x.shape[1], x.shape[0]), dtype=torch.float64, pin_memory=True)
        h = t.numpy().T
        h[:] = x
        return h
    Ah, Ch, Sh = host(A), host(C), host(S)
    api.rot_apply_host(Ah, Ch, Sh)
    rs.rot_device_status()
    assert np.array_equal(bits(np.ascontiguousarray(Ah)), bits(np.ascontiguousarray(ref)))
