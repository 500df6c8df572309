"""The multi-core CPU baseline (row blocks on host threads, wave order inside a
block; Section 7 and Algorithm 3) equals the oracle's Algorithm 2 bit for bit.

Row independence (each row is updated as a_i <- a_i * G) lets threads take
any blocks of rows; the wave order keeps every element's operations in
Algorithm 2's order.  So the baseline's result must match the oracle exactly
on every shape and blocking, including ragged row blocks, k > n-1 and a last
p-block shorter than the rest.
"""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

SHAPES = [(1, 2, 1), (37, 5, 9), (100, 77, 21), (65, 300, 40), (33, 17, 50), (129, 64, 65)]
BLOCKINGS = [(32, 32), (7, 5), (1, 1), (64, 100), (16, 3)]


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_parallel_baseline_bit_exact(m, n, k):
    A, C, S = wl.problem(m, n, k, seed=11)
    ref = oracle.rot_sequence(A, C, S)
    for mb, kb in BLOCKINGS:
        for threads in (1, 3, 0):
            out, used = oracle.rot_sequence_parallel(A, C, S, mb=mb, kb=kb, threads=threads)
            assert used >= 1
            assert np.array_equal(_bits(out), _bits(ref)), (m, n, k, mb, kb, threads)


def test_parallel_baseline_signed_zeros_and_inf():
    """IEEE special values propagate exactly as in the oracle (no padding rotations)."""
    A, C, S = wl.problem(40, 23, 7, seed=5)
    A[3, :] = -0.0
    A[5, 4] = np.inf
    A[9, 0] = -np.inf
    ref = oracle.rot_sequence(A, C, S)
    out, _ = oracle.rot_sequence_parallel(A, C, S, mb=16, kb=4)
    assert np.array_equal(_bits(out), _bits(ref))


def test_parallel_baseline_quick_return_and_inplace():
    A, C, S = wl.problem(8, 1, 0, seed=1)
    out, used = oracle.rot_sequence_parallel(A, C, S)
    assert used == 1 and np.array_equal(out, A)
    A, C, S = wl.problem(50, 30, 6, seed=3)
    ref = oracle.rot_sequence(A, C, S)
    B = np.asfortranarray(A.copy())
    out, _ = oracle.rot_sequence_parallel(B, C, S, inplace=True)
    assert out is B
    assert np.array_equal(_bits(B), _bits(ref))


def test_parallel_baseline_uses_several_threads():
    """With OpenMP available the baseline runs on more than one host thread."""
    import os
    if not oracle.parallel_uses_openmp() or (os.cpu_count() or 1) < 2:
        pytest.skip("compiler without OpenMP or a single-core host")
    A, C, S = wl.problem(256, 40, 8, seed=2)
    _, used = oracle.rot_sequence_parallel(A, C, S, threads=2)
    assert used == 2
