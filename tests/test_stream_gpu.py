"""The column stream (passes of up to 8 sequences; FP64 passes of up to 4 on
the split stream) that rot_apply (k <= 16 where the lane pipeline does not
apply, small k and the pipeline's remainders where it does) and
rot_apply_f32 (k <= 41, or k <= 48 where the lane pipeline does not apply)
take when A is TMA-addressable: bit-exact against the
oracles on ragged shapes, padded leading dimensions, every k from 1 to 8 (so
every window size and the k < window case), several passes (k = 9, 16, 23,
48), and the full 8192 x 8192 matrix at k = 1.  Leading dimensions the stream
cannot address fall back to the wavefront kernel, with the same bits."""
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
    x = np.ascontiguousarray(x)
    return x.view(np.uint64 if x.dtype == np.float64 else np.uint32)


CASES = [  # m, n, k, lda slack (m < 64 or n < 32: the wavefront kernel)
    (32, 32, 1, 0), (33, 40, 2, 4), (64, 32, 1, 0), (65, 40, 2, 4), (127, 41, 3, 0), (100, 77, 4, 8),
    (95, 200, 5, 0), (128, 33, 6, 4), (257, 130, 7, 0), (64, 300, 8, 12), (1000, 3000, 1, 0),
    (50, 1001, 8, 2), (300, 31, 2, 0), (96, 100, 9, 0), (130, 257, 16, 4), (70, 90, 23, 0), (64, 200, 48, 8),
    # at the thresholds: no tile of all-complete waves (n = 64, k = 8), a single tile, one row past a strip
    (64, 64, 8, 0), (64, 64, 1, 0), (65, 65, 3, 0), (64, 127, 5, 4), (97, 64, 2, 0),
]


@pytest.mark.parametrize("m,n,k,slack", CASES)
def test_stream_f64_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=m + 3 * n + k)
    ref = oracle.rot_sequence(A, C, S)
    Ad, buf = dev(A, (m + slack + 1) // 2 * 2)      # FP64: an even lda keeps the pitch a 16-byte multiple
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))


@pytest.mark.parametrize("m,n,k,slack", CASES)
def test_stream_f32_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=2 * m + n + k)
    A32, C32, S32 = (x.astype(np.float32) for x in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    ld = (m + slack + 3) // 4 * 4                   # FP32: a multiple of 4
    Ad, buf = dev(A32, ld)
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))


@pytest.mark.parametrize("ld_extra", [1, 3])
def test_unaligned_leading_dimension_falls_back(rs, ld_extra):
    m, n, k = 64, 100, 3
    A, C, S = wl.problem(m, n, k, seed=5)
    A32, C32, S32 = (x.astype(np.float32) for x in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, buf = dev(A32, m + ld_extra)                # pitch not a 16-byte multiple
    rs.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    rs.rot_device_status()
    assert np.array_equal(bits(buf.cpu().numpy()[:m, :n]), bits(ref))


def test_stream_8192_k1_sampled_rows(rs):
    m = n = 8192
    A = wl.matrix(m, n, 2)
    C, S = wl.rotations(n, 1, 2)
    r = np.random.default_rng(80)
    rows = np.unique(np.concatenate([[0, 31, 32, m - 1], r.choice(m, 28, replace=False)]))
    ref = oracle.rot_sequence(A[rows], C, S)
    ref32 = oracle.rot_sequence_f32(A[rows].astype(np.float32), C.astype(np.float32), S.astype(np.float32))
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    A32 = torch.from_numpy(np.ascontiguousarray(A.astype(np.float32).T)).cuda().t()
    rs.rot_apply_f32(A32, dev(C.astype(np.float32))[0], dev(S.astype(np.float32))[0])
    rs.rot_device_status()
    idx = torch.from_numpy(rows).cuda()
    assert np.array_equal(bits(Ad[idx].cpu().numpy()), bits(ref))
    assert np.array_equal(bits(A32[idx].cpu().numpy()), bits(ref32))


# FP64 passes of one to four sequences on column-major A run as two warps a
# sequence per 32-row strip (one carrying the sequence's chain, the other
# its finished columns, which feed the next sequence's pair), handing values
# over through rings of shared-memory tiles.  Ragged strips, padded leading
# dimensions, n around the 20-, 21- and 16-column tiles and the rings' wrap
# (more than four tiles), k = 5..7 as a pass of four and the rest, ±0 and
# infinities, bit-exact against the oracle.
SPLIT_CASES = [(64, 64, 1, 0), (64, 64, 2, 0), (65, 81, 1, 2), (95, 80, 2, 4), (128, 126, 2, 0),
               (200, 300, 1, 6), (333, 301, 2, 2), (1000, 1001, 2, 0), (97, 127, 1, 0), (160, 64, 2, 8),
               (64, 64, 3, 0), (64, 64, 4, 0), (65, 81, 3, 2), (95, 200, 4, 4), (128, 126, 3, 0),
               (333, 250, 4, 2), (97, 127, 3, 0), (160, 64, 4, 8), (1000, 255, 3, 0), (96, 100, 7, 0),
               (200, 150, 6, 2), (130, 255, 5, 0), (64, 65, 4, 0), (64, 79, 3, 0)]


@pytest.mark.parametrize("m,n,k,slack", SPLIT_CASES)
def test_stream_split_f64_bit_exact(rs, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=7 * m + n + k)
    A[::7, ::5] = -0.0
    A[3, 2] = np.inf
    A[5, n - 1] = -np.inf
    ref = oracle.rot_sequence(A, C, S)
    Ad, buf = dev(A, (m + slack + 1) // 2 * 2)
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    out = buf.cpu().numpy()
    # Two infinities meeting in one rotation make NaNs (Inf - Inf); their bit
    # patterns are platform-specific, their places are not.
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(out[:m, :n]), nan)
    assert np.array_equal(bits(out[:m, :n][~nan]), bits(ref[~nan]))
    assert np.all(np.isnan(out[m:, :n]))


@pytest.mark.parametrize("m,n,k", [(8192, 8192, 2), (8192, 8192, 3), (4096, 4096, 4), (4096, 4096, 7)])
def test_stream_split_full_size_sampled_rows(rs, m, n, k):
    """Full-size matrices in the launch configuration of the library: two
    strips per SM at k = 2 and 3, one at k = 4 and 7 (passes of 4 and 3)."""
    A = wl.matrix(m, n, 2)
    C, S = wl.rotations(n, k, 2)
    r = np.random.default_rng(81)
    rows = np.unique(np.concatenate([[0, 31, 32, m - 1], r.choice(m, 28, replace=False)]))
    ref = oracle.rot_sequence(A[rows], C, S)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    rs.rot_apply(Ad, dev(C)[0], dev(S)[0])
    rs.rot_device_status()
    idx = torch.from_numpy(rows).cuda()
    assert np.array_equal(bits(Ad[idx].cpu().numpy()), bits(ref))
