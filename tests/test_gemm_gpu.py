"""Accumulated blocks (rs_gemm, Section 8) against the oracle.

Block formation is FP64 and follows the same per-element operation order as
the oracle's form_block, so every non-zero entry is bit-identical (zeros may
differ in sign: rotations on two zeros are skipped).  The block apply uses
tensor-core products; each mode is held to an error bound against the FP64
oracle, per row, with P = ceil(k/kb) p-blocks.  Every element passes through
about two block products per p-block and the errors of the p-blocks add up
like a random walk or linearly:
  DMMA        32*sqrt(P)*2^-53    (FP64 products, FP64 accumulation)
  split FP16  P*2^-20             (x = hi + 2^-11 lo: operands exact to ~2^-22)
  split BF16  1.5*P*2^-17         (x = hi + lo: operands exact to ~2^-17)
The constants were set from the errors measured on GB300 for these shapes
(each bound is 1.8x to 4x the largest measured error; at the 8192 x 8192,
k = 192, nb = 256, kb = 64 precision workload the measured errors are
1.8e-15, 6.2e-7 and 9.1e-6, against bounds of 6.2e-15, 2.9e-6 and 3.4e-5), so
that an accuracy regression of a few times fails.
The *-q32 modes form the blocks in FP32 (rot_form_blocks_f32), which equal
the oracle's FP32 blocks entry for entry; their products are held to the
same bounds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01852_gb300 import api, build
    build.build()
    return api


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def row_rel(out, ref):
    return np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)


def bound(mode, k, nb, kb):
    mode = mode.split("-")[0]
    P = math.ceil(k / kb)
    if mode == "dmma":
        return 32 * math.sqrt(P) * U64
    if mode == "f16":
        return P * 2.0 ** -20
    return 1.5 * P * 2.0 ** -17


@pytest.mark.parametrize("n,k,nb,kb", [(40, 9, 16, 16), (100, 40, 32, 16), (300, 64, 64, 32),
                                       (70, 100, 48, 16), (600, 130, 256, 64)])
def test_form_blocks_match_oracle(api, n, k, nb, kb):
    C, S = wl.rotations(n, k, seed=n + k)
    Q = api.rot_form_blocks(n, dev(C), dev(S), nb, kb)
    torch.cuda.synchronize()
    api.rot_device_status()
    sched = oracle.block_schedule(n, k, nb, kb)
    assert Q.shape[0] == len(sched) == api.form_blocks_count(n, k, nb, kb)
    Qh = Q.cpu().numpy()
    for b, (w0, p0) in enumerate(sched):
        ref = oracle.form_block(C, S, n, w0, nb, p0, kb)
        got = Qh[b].T
        assert np.array_equal(got, ref), b                   # equal values (+0 == -0)
        nz = ref != 0
        assert np.array_equal(got[nz].view(np.uint64), ref[nz].view(np.uint64)), b


@pytest.mark.parametrize("n,k,nb,kb", [(40, 9, 16, 16), (100, 40, 32, 16), (300, 64, 64, 32),
                                       (70, 100, 48, 16), (600, 130, 256, 64), (200, 50, 16, 48),
                                       (300, 70, 64, 96), (150, 40, 32, 128), (2, 3, 16, 64)])
def test_form_blocks_f32_match_oracle(api, n, k, nb, kb):
    """FP32 blocks from the lane pipeline equal the oracle's sequential FP32
    blocks entry for entry (non-zero entries bit for bit)."""
    C, S = wl.rotations(n, k, seed=n + k + 5)
    Q = api.rot_form_blocks_f32(n, dev(C), dev(S), nb, kb)
    torch.cuda.synchronize()
    api.rot_device_status()
    sched = oracle.block_schedule(n, k, nb, kb)
    assert Q.shape[0] == len(sched) and Q.dtype == torch.float32
    Qh = Q.cpu().numpy()
    for b, (w0, p0) in enumerate(sched):
        ref = oracle.form_block_f32(C, S, n, w0, nb, p0, kb)
        got = Qh[b].T
        assert np.array_equal(got, ref), b
        nz = ref != 0
        assert np.array_equal(got[nz].view(np.uint32), ref[nz].view(np.uint32)), b


def test_form_blocks_f32_rejects_kb_over_128(api):
    C, S = wl.rotations(300, 200, seed=1)
    with pytest.raises(Exception):
        api.rot_form_blocks_f32(300, dev(C), dev(S), 16, 144)


@pytest.mark.parametrize("mode", ["dmma", "f16", "bf16", "f16-q32", "bf16-q32"])
@pytest.mark.parametrize("m,n,k,nb,kb", [(100, 300, 40, 64, 16), (33, 130, 70, 32, 32),
                                         (257, 500, 64, 256, 64), (64, 40, 100, 16, 16),
                                         (90, 200, 50, 16, 48),
                                         # 320-wide windows with few carried columns (two
                                         # tensor-memory windows do not fit beside four Q
                                         # stages, so the split modes take mma.sync)
                                         (200, 700, 40, 288, 32), (150, 900, 30, 304, 16)])
def test_apply_gemm_within_bound(api, mode, m, n, k, nb, kb):
    A, C, S = wl.problem(m, n, k, seed=m + n + k)
    ref = oracle.rot_sequence(A, C, S)
    Ad = dev(A)
    api.rot_apply_gemm(Ad, dev(C), dev(S), nb=nb, kb=kb, mode=mode)
    torch.cuda.synchronize()
    api.rot_device_status()
    out = Ad.cpu().numpy()
    rel = row_rel(out, ref)
    assert rel.max() <= bound(mode, k, nb, kb), rel.max()
    if mode == "dmma":
        viaq = oracle.rot_sequence_gemm(A, C, S, nb, kb)
        assert np.max(np.abs(out - viaq)) <= 16 * (nb + kb) * U64 * np.abs(A).max() * 4


@pytest.mark.parametrize("mode", ["f16", "bf16", "f16-q32", "bf16-q32"])
def test_wide_window_split_modes(api, mode):
    """Windows wider than the tensor-memory kernel takes (nb + kb = 384) run
    on the mma.sync kernel; same bound."""
    m, n, k, nb, kb = 100, 700, 40, 352, 32
    A, C, S = wl.problem(m, n, k, seed=m + n + k + 1)
    ref = oracle.rot_sequence(A, C, S)
    Ad = dev(A)
    api.rot_apply_gemm(Ad, dev(C), dev(S), nb=nb, kb=kb, mode=mode)
    torch.cuda.synchronize()
    api.rot_device_status()
    rel = row_rel(Ad.cpu().numpy(), ref)
    assert rel.max() <= bound(mode, k, nb, kb), rel.max()


@pytest.mark.parametrize("mode", ["dmma", "f16", "bf16", "f16-q32", "bf16-q32"])
def test_orthogonality_drift_on_identity(api, mode):
    n, k, nb, kb = 256, 48, 64, 16
    C, S = wl.rotations(n, k, seed=3)
    Ad = dev(np.eye(n))
    api.rot_apply_gemm(Ad, dev(C), dev(S), nb=nb, kb=kb, mode=mode)
    torch.cuda.synchronize()
    Q = Ad.cpu().numpy()
    drift = np.abs(Q.T @ Q - np.eye(n)).max()
    tol = bound(mode, k, nb, kb)
    assert drift <= tol, drift


@pytest.mark.parametrize("mode", ["f16", "bf16", "dmma", "f16-q32", "bf16-q32"])
def test_precision_config_8192_sampled_rows(api, mode):
    """A 8192 x 8192, k = 192, nb = 256, kb = 64: rows sampled against the FP64 oracle."""
    cfg = wl.WORKLOADS["precision-8192"]
    m, n, k, nb, kb = cfg["m"], cfg["n"], cfg["k"], cfg["nb"], cfg["kb"]
    A, C, S = wl.problem(m, n, k, seed=cfg["seed"])
    g = np.random.default_rng(8)
    rows = np.unique(np.concatenate([[0, m - 1], g.choice(m, 10, replace=False)]))
    ref = oracle.rot_sequence(A[rows], C, S)
    Ad = dev(A)
    api.rot_apply_gemm(Ad, dev(C), dev(S), nb=nb, kb=kb, mode=mode)
    torch.cuda.synchronize()
    api.rot_device_status()
    out = Ad[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert row_rel(out, ref).max() <= bound(mode, k, nb, kb)


@pytest.mark.parametrize("mode", ["bf16", "f16", "dmma", "bf16-q32", "f16-q32"])
def test_caller_workspace_gives_the_same_bits(api, mode):
    """rot_apply_gemm_ws with caller-owned scratch equals rot_apply_gemm bit for bit."""
    m, n, k, nb, kb = 100, 300, 40, 64, 16
    A, C, S = wl.problem(m, n, k, seed=77)
    Cd, Sd = dev(C), dev(S)
    a1, a2 = dev(A), dev(A)
    api.rot_apply_gemm(a1, Cd, Sd, nb=nb, kb=kb, mode=mode)
    nbytes = api.gemm_workspace_size(m, n, k, nb=nb, kb=kb, mode=mode)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    api.rot_apply_gemm_ws(a2, Cd, Sd, ws, nb=nb, kb=kb, mode=mode)
    torch.cuda.synchronize()
    api.rot_device_status()
    assert torch.equal(a1.view(torch.int64), a2.view(torch.int64))


def test_tc_issue_probe(api):
    """The issue-rate probe runs and is consistent: more independent
    accumulators never make a product slower, and one product costs between
    1 ns and 10 us."""
    one = api.measure_tc_issue(64, 160, 1, 2000)
    three = api.measure_tc_issue(64, 160, 3, 2000)
    big = api.measure_tc_issue(128, 256, 2, 2000)
    for v in (one, three, big):
        assert 1.0 < v < 10000.0, v
    assert three <= one * 1.05, (one, three)
