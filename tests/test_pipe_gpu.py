"""The lane pipeline (rs_pipe.cu).  FP32: rot_apply_f32 takes it for n >= 1024
and k >= 56, and from k = 42 (k = 20 with at most 4096 rows) where the warp
chain does not apply (fewer than 64 rows, a leading dimension TMA cannot
address, or k = 8j + 7 with at most 4096 rows);
FP64: rot_apply (and rot_apply_left) for 3 <= k <= 32 and n >= 256.  FP32 cases: bit-exact against
the FP32 oracle on ragged row counts, padded leading dimensions, every pass
width (32 .. 192 sequences), several passes (k = 224, 384, 448), the k mod 32
sequences left over (on the column stream or the wavefront kernel), signed
zeros and infinities at the two ends of the column stream (where stages pass
values through), and the full 8192 x 8192 matrix at k = 64 on sampled rows.
FP64 cases: every group width (4, 8, 16, 32 lanes), k not a power of two
(stages past k pass values through), the plans that leave up to 4
sequences to the split column stream (at most one strip per SM, and more),
ragged rows, padded leading dimensions, signed zeros and infinities, and
8192 x 8192 at k = 8 and 16 on sampled rows, bit-exact against the FP64
oracle."""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import build
    build.build()
    return rs


def dev(a, ld=None):
    rows, cols = a.shape
    ld = max(rows, 1) if ld is None else ld
    buf = np.full((ld, max(cols, 1)), np.nan, dtype=a.dtype, order="F")
    buf[:rows, :cols] = a
    t = torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()
    return t[:rows, :cols], t


def bits(x):
    return np.ascontiguousarray(x).view(np.uint32)


CASES = [  # m, n, k, lda slack
    (8, 1024, 32, 0), (9, 1024, 32, 3), (33, 1100, 64, 0), (100, 1500, 96, 5), (17, 2000, 192, 0),
    (40, 1057, 160, 1), (31, 4096, 128, 0), (257, 1024, 192, 7), (8, 1024, 224, 0), (64, 1030, 384, 2),
    (1, 1024, 32, 0), (7, 1031, 64, 0), (64, 1030, 448, 0),
    # k not a multiple of 32: the rest on the column stream (m >= 64) or the wavefront kernel
    (70, 1100, 70, 0), (65, 1024, 100, 3), (20, 1024, 45, 0), (100, 1200, 203, 0), (40, 1024, 35, 2),
    # or one more, part-filled lane of sequences (k mod 32 >= 22, or >= 10 after one lane)
    (64, 1024, 42, 0), (80, 1100, 63, 1), (9, 1024, 86, 0), (66, 1030, 95, 0), (30, 1024, 191, 3),
    (70, 1024, 223, 0),
    # 20 <= k < 32 with few rows: a single part-filled pass
    (64, 1024, 20, 0), (100, 1100, 31, 3), (9, 1024, 24, 0),
    # k = 8j + 7 with at most 4096 rows and an aligned A: the warp chain
    # leaves these to the pipeline
    (64, 1024, 31, 0), (100, 1024, 47, 0),
]


@pytest.mark.parametrize("m,n,k,slack", CASES)
def test_pipe_f32_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=m + 7 * n + k)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, buf = dev(A32, m + slack)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))                      # rows past m untouched


CASES64 = [  # m, n, k, lda slack: FP64, 3 <= k <= 32, n >= 256 (groups of 4, 8, 16 or 32 lanes)
    (8, 256, 3, 0), (9, 300, 4, 1), (33, 700, 5, 0), (100, 1024, 8, 3), (17, 257, 9, 0), (64, 1000, 16, 2),
    (5, 400, 17, 0), (71, 600, 31, 0), (40, 1100, 32, 1), (1, 256, 8, 0), (200, 333, 12, 0),
    # k = 4j + 1 with m >= 64 and an even lda: passes, then the rest on the split column stream
    (64, 300, 5, 0), (100, 512, 13, 2), (128, 777, 21, 0), (96, 260, 29, 0),
    # the same k with an odd lda (no column stream): the last pass takes it
    (65, 300, 9, 0),
]


# FP64 just past 32 sequences: the wavefront kernel with p-blocks as long as
# the resident warps allow (short ones for these few rows).
CASES64 += [(64, 300, 33, 0), (70, 256, 34, 2), (40, 400, 40, 0), (100, 260, 61, 0), (33, 512, 64, 1),
            (9, 300, 33, 0)]

# At most one 32-row strip per SM: full passes of 8, 16 and 32 for the
# multiple of 8, the rest (up to 7) on the split column stream; up to 4096
# rows, k >= 29 as one pass of 32 (k = 29, 31 here; 4200 rows: 16 + 8 + 6).
CASES64 += [(100, 300, 10, 0), (64, 257, 11, 2), (70, 400, 12, 0), (96, 300, 18, 0), (128, 256, 20, 2),
            (80, 512, 24, 0), (100, 300, 15, 0), (64, 400, 29, 0), (70, 256, 31, 2), (65, 260, 13, 1),
            (64, 400, 21, 0), (70, 300, 23, 2), (4200, 256, 30, 0)]

# More strips than SMs: passes of powers of two, remainders of 2 (past a
# pass of 8) and of 3 (at most two strips per SM) on the split stream; k = 3
# alone on it; with more than two strips per SM a remainder of 3 stays in a
# pass of 4.
CASES64 += [(4900, 256, 10, 0), (4900, 300, 11, 0), (5000, 256, 19, 0), (4900, 260, 26, 2), (5000, 256, 3, 0),
            (9800, 256, 3, 0), (9800, 256, 11, 0)]


@pytest.mark.parametrize("m,n,k,slack", CASES64)
def test_pipe_f64_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=m + 5 * n + k)
    ref = oracle.rot_sequence(A, C, S)
    Ad, buf = dev(A, m + slack)
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    assert np.array_equal(out[:m, :n].view(np.uint64), ref.view(np.uint64))
    assert np.all(np.isnan(out[m:, :n]))


def test_pipe_f64_signed_zeros_and_infinities(rs):
    m, n, k = 24, 500, 8
    A, C, S = wl.problem(m, n, k, seed=92)
    A[0, 0] = -0.0
    A[1, n - 1] = -0.0
    A[2, 3] = np.inf
    A[9, n - 1] = -np.inf
    A[11, :] = 0.0
    A[12, :] = -0.0
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = dev(A)
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    out = Ad.cpu().numpy()
    nan = np.isnan(ref)
    assert nan.any() and np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.uint64), ref[~nan].view(np.uint64))


@pytest.mark.parametrize("k", [8, 16])
def test_pipe_f64_full_8192_sampled_rows(rs, k):
    m = n = 8192
    A, C, S = wl.problem(m, n, k, seed=6 + k)
    rows = np.unique(np.concatenate([[0, 1, 7, 8, m - 1], np.random.default_rng(k).choice(m, 12, replace=False)]))
    ref = oracle.rot_sequence(A[rows], C, S)
    Ad, _ = dev(A)
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


def test_pipe_f32_signed_zeros_and_infinities(rs):
    """Zeros and infinities in the first and last columns, where some stages
    pass values through: signs of zeros and the places of NaNs (0*Inf) match
    the oracle; NaN bit patterns are platform-specific."""
    m, n, k = 24, 1200, 192
    A, C, S = wl.problem(m, n, k, seed=91)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    A32[0, 0] = -0.0
    A32[1, n - 1] = -0.0
    A32[5, 0] = 0.0
    A32[2, 3] = np.inf
    A32[9, n - 1] = -np.inf
    A32[11, :] = 0.0
    A32[12, :] = -0.0
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, _ = dev(A32)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = Ad.cpu().numpy()
    nan = np.isnan(ref)
    assert nan.any() and np.array_equal(np.isnan(out), nan)
    assert np.array_equal(bits(out[~nan]), bits(ref[~nan]))
    assert np.array_equal(bits(out[11:13]), bits(ref[11:13]))   # zero rows keep their zeros' signs


def test_pipe_f32_full_8192_sampled_rows(rs):
    """A 8192 x 8192 FP32 at k = 64 (one pass of 64 stages) in the launch
    configuration of the library: sampled rows bit-exact."""
    m = n = 8192
    k = 64
    A, C, S = wl.problem(m, n, k, seed=5)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    rows = np.unique(np.concatenate([[0, 7, 8, m - 1], np.random.default_rng(3).choice(m, 12, replace=False)]))
    ref = oracle.rot_sequence_f32(A32[rows], C32, S32)
    Ad, _ = dev(A32)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(bits(out), bits(ref))
