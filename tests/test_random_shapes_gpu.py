"""Seeded random shapes through every GPU path, against the CPU oracle.

The hand-picked shapes of the other parity tests cover the edge cases by
name; this sweep draws further (m, n, k), leading-dimension slack and block
sizes from a fixed seed, so each run checks the same 68 cases:
  FP64 wavefront        bit-exact vs oracle.rot_sequence
  FP32 wavefront        bit-exact vs oracle.rot_sequence_f32
  left application      bit-exact vs oracle.rot_sequence_left
  2x2 reflectors        bit-exact vs oracle.refl_sequence
  block apply           per-row error within each mode's bound
  batch of problems     every problem bit-exact
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


def dev(a, ld=None):
    """Column-major device copy with leading dimension ld (padding rows NaN)."""
    rows, cols = a.shape
    ld = max(rows, 1) if ld is None else ld
    buf = np.full((ld, max(cols, 1)), np.nan, dtype=a.dtype, order="F")
    buf[:rows, :cols] = a
    t = torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()
    return t[:rows, :cols], t


def bits(x):
    x = np.ascontiguousarray(x)
    return x.view(np.uint64 if x.dtype == np.float64 else np.uint32)


def draw(seed, count, m_hi=300, n_hi=600, k_hi=80):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(g.integers(1, m_hi + 1))
        n = int(g.integers(2, n_hi + 1))
        k = int(g.integers(1, k_hi + 1))
        slack = int(g.integers(0, 5))
        out.append((m, n, k, slack))
    return out


@pytest.mark.parametrize("m,n,k,slack", draw(101, 16))
def test_random_f64_bit_exact(api, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=m * 7 + n * 3 + k)
    ref = oracle.rot_sequence(A, C, S)
    Ad, Abuf = dev(A, m + slack)
    api.rot_apply(Ad, dev(C)[0], dev(S)[0])
    api.rot_device_status()
    out = Abuf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))            # padding rows untouched


@pytest.mark.parametrize("m,n,k,slack", draw(202, 16))
def test_random_f32_bit_exact(api, m, n, k, slack):
    A, C, S = wl.problem(m, n, k, seed=m * 5 + n + k)
    A32, C32, S32 = (x.astype(np.float32) for x in (A, C, S))
    ref = oracle.rot_sequence_f32(A32, C32, S32)
    Ad, Abuf = dev(A32, m + slack)
    api.rot_apply_f32(Ad, dev(C32)[0], dev(S32)[0])
    api.rot_device_status()
    out = Abuf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))


@pytest.mark.parametrize("m,n,k,slack", draw(505, 8, m_hi=400, n_hi=200))
def test_random_left_bit_exact(api, m, n, k, slack):
    A = wl.matrix(m, n, seed=m + 2 * n + k)
    C, S = wl.rotations(m, k, seed=k + 7)                # rotations mix the m rows
    ref = oracle.rot_sequence_left(A, C, S)
    Ad, Abuf = dev(A, m + slack)
    api.rot_apply_left(Ad, dev(C)[0], dev(S)[0])
    api.rot_device_status()
    out = Abuf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))


@pytest.mark.parametrize("m,n,k,slack", draw(606, 8))
def test_random_reflectors_bit_exact(api, m, n, k, slack):
    A = wl.matrix(m, n, seed=3 * m + n + k)
    T, V = wl.reflectors(n, k, seed=m + k)
    ref = oracle.refl_sequence(A, T, V)
    Ad, Abuf = dev(A, m + slack)
    api.rot_apply_reflectors(Ad, dev(T)[0], dev(V)[0])
    api.rot_device_status()
    out = Abuf.cpu().numpy()
    assert np.array_equal(bits(out[:m, :n]), bits(ref))
    assert np.all(np.isnan(out[m:, :n]))


def gemm_cases(seed, count):
    g = np.random.default_rng(seed)
    out = []
    for (m, n, k, _) in draw(seed, count, m_hi=200, n_hi=500, k_hi=70):
        kb = 16 * int(g.integers(1, 5))
        nb = 16 * int(g.integers(1, 21 - kb // 16))       # nb + kb <= 320
        out.append((m, n, k, nb, kb))
    return out


@pytest.mark.parametrize("mode", ["bf16", "f16", "dmma"])
@pytest.mark.parametrize("m,n,k,nb,kb", gemm_cases(303, 6))
def test_random_block_apply_within_bound(api, mode, m, n, k, nb, kb):
    A, C, S = wl.problem(m, n, k, seed=m + 11 * n + k)
    ref = oracle.rot_sequence(A, C, S)
    Ad, _ = dev(A)
    api.rot_apply_gemm(Ad, dev(C)[0], dev(S)[0], nb=nb, kb=kb, mode=mode)
    api.rot_device_status()
    out = Ad.cpu().numpy()
    rel = np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)
    if mode == "dmma":
        lim = 16 * (k + nb + kb) * U64
    elif mode == "f16":
        lim = 8 * k * U32
    else:
        lim = 4 * math.ceil(k / kb) * 2.0 ** -16
    assert rel.max() <= lim, (rel.max(), lim)


@pytest.mark.parametrize("seed", [404, 405])
def test_random_batch_bit_exact(api, seed):
    cases = draw(seed, 12, m_hi=400, n_hi=300, k_hi=60)
    probs, refs, bufs = [], [], []
    for i, (m, n, k, slack) in enumerate(cases):
        A, C, S = wl.problem(m, n, k, seed=seed * 100 + i)
        refs.append(oracle.rot_sequence(A, C, S))
        Ad, Abuf = dev(A, m + slack)
        bufs.append(Abuf)
        probs.append((Ad, dev(C)[0], dev(S)[0]))
    api.rot_apply_batched(probs)
    api.rot_device_status()
    for (m, n, k, _), Abuf, ref in zip(cases, bufs, refs):
        out = Abuf.cpu().numpy()
        assert np.array_equal(bits(out[:m, :n]), bits(ref)), (m, n, k)
        assert np.all(np.isnan(out[m:, :n]))
