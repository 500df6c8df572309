"""The FP32 warp chain (rs_chain.cu): rot_apply_f32 with 16 <= k <= 55 on a
TMA-addressable A runs one pass of 16, 24, 32, 40 or 48 sequences as eight
chained warps per 32-row strip, and k mod 8 on the column stream after it.
Bit-exact against the FP32 oracle on ragged row counts, padded leading
dimensions, n around each configuration's tile width and below a tile,
every pass size with and without a remainder, signed zeros and infinities
(NaN places compared, NaN bit patterns being platform-specific), and the
full 8192 x 8192 matrix on sampled rows.  A leading dimension the chain
cannot address falls back to another kernel, with the same bits."""
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


CASES = [  # m, n, k, lda slack (a multiple of 4 keeps the column pitch a 16-byte multiple)
    (64, 64, 16, 0), (65, 100, 16, 4), (97, 301, 24, 0), (130, 257, 32, 8), (200, 500, 40, 0), (1000, 700, 48, 4),
    (64, 64, 48, 0), (96, 65, 40, 0), (33 * 32, 90, 32, 0),
    # k mod 8 left to the column stream
    (70, 300, 17, 0), (100, 256, 23, 4), (130, 129, 31, 0), (64, 400, 37, 0), (99, 333, 47, 0),
    (128, 200, 49, 0), (160, 1000, 55, 4),
    # n below or around one tile (15, 16, 15, 12, 14 columns for 16 .. 48 sequences)
    (64, 70, 16, 0), (64, 76, 24, 0), (65, 79, 32, 0), (64, 70, 40, 0), (64, 75, 48, 0),
]


@pytest.mark.parametrize("m,n,k,slack", CASES)
def test_chain_f32_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=3 * m + n + k)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, buf = dev(A32, m + slack)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))                      # rows past m untouched


@pytest.mark.parametrize("k", [16, 32, 48, 37])
def test_chain_signed_zeros_and_infinities(rs, k):
    m, n = 100, 400
    A, C, S = wl.problem(m, n, k, seed=11 + k)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    A32[0, 0] = -0.0
    A32[1, n - 1] = -0.0
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


@pytest.mark.parametrize("ld_extra", [1, 2, 3])
def test_chain_unaligned_leading_dimension_falls_back(rs, ld_extra):
    m, n, k = 64, 300, 32
    A, C, S = wl.problem(m, n, k, seed=17)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, buf = dev(A32, m + ld_extra)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    assert np.array_equal(bits(buf.cpu().numpy()[:m, :n]), bits(ref))


@pytest.mark.parametrize("k", [48, 37])
def test_chain_full_8192_sampled_rows(rs, k):
    """8192 x 8192 in the launch configuration of the library (256 strips of
    eight chained warps and a producer warp): sampled rows bit-exact."""
    m = n = 8192
    A = wl.matrix(m, n, 4)
    C, S = wl.rotations(n, k, 4)
    A32, C32, S32 = (X.astype(np.float32) for X in (A, C, S))
    rows = np.unique(np.concatenate([[0, 31, 32, m - 1], np.random.default_rng(k).choice(m, 16, replace=False)]))
    ref = oracle.rot_sequence_f32(A32[rows], C32, S32)
    Ad = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().t()
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(bits(out), bits(ref))
