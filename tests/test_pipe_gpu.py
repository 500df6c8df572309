"""The FP32 lane pipeline (rs_pipe_f32.cu) that rot_apply_f32 takes for
k >= 32 and n >= 1024 (where the column stream does not): bit-exact against
the FP32 oracle on ragged row counts, padded leading dimensions, every pass
width (32 .. 192 sequences), several passes (k = 224, 384, 448), the k mod 32
sequences left over (on the column stream or the wavefront kernel), signed
zeros and infinities at the two ends of the column stream (where stages pass
values through), and the full 8192 x 8192 matrix at k = 64 on sampled rows."""
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
    (70, 1100, 70, 0), (65, 1024, 100, 3), (20, 1024, 45, 0), (100, 1200, 203, 0),
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
