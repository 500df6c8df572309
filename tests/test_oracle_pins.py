"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with a retyped copy of itself.  Each check is
a closed form, an exact special case, an invariant of orthogonal matrices, a
library routine (BLAS drot), exact rational arithmetic on tiny inputs, or an
equivalence between two different algorithms of the paper.  A dropped term, a
sign error, a wrong C/S index or a transposed operand in the oracle fails at
least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl
from conftest import read_golden

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- P1 closed form
def test_p1_closed_form_single_rotation_golden():
    """Algorithm 1 on (3, 4) with (c, s) = (3/5, 4/5) gives (5, 0)."""
    g = read_golden("closed_form_n2.txt")
    c, s = g["c"][0][0], g["s"][0][0]
    x, y = g["x"][0][0], g["y"][0][0]
    A = np.array([[x, y]])
    out = oracle.rot_sequence(A, np.array([[c]]), np.array([[s]]))
    assert abs(out[0, 0] - g["x_out"][0][0]) <= g["tol"][0][0]
    assert abs(out[0, 1] - g["y_out"][0][0]) <= g["tol"][0][0]


def test_p1_single_rotation_exact_rational_bound():
    """x' = c x + s y, y' = -s x + c y to within two roundings, random values."""
    r = _rng(11)
    for _ in range(200):
        x, y = r.standard_normal(2) * 10.0 ** r.integers(-5, 5)
        th = r.uniform(0, 2 * math.pi)
        c, s = math.cos(th), math.sin(th)
        xo, yo = oracle.rot([x], [y], c, s)
        fx, fy, fc, fs = map(Fraction, (x, y, c, s))
        ex = fc * fx + fs * fy
        ey = -fs * fx + fc * fy
        bx = 2 * U64 * (abs(c * x) + abs(s * y))
        by = 2 * U64 * (abs(s * x) + abs(c * y))
        assert abs(Fraction(float(xo[0])) - ex) <= Fraction(bx)
        assert abs(Fraction(float(yo[0])) - ey) <= Fraction(by)


def test_p1_n2_composition_equals_sum_of_angles():
    """n = 2: k plane rotations compose to one rotation by the summed angle."""
    r = _rng(12)
    for k in (1, 2, 5, 17, 64):
        th = r.uniform(0, 2 * math.pi, size=k)
        C = np.cos(th).reshape(1, k)
        S = np.sin(th).reshape(1, k)
        A = r.standard_normal((7, 2))
        out = oracle.rot_sequence(A, C, S)
        T = th.sum()
        ct, st = math.cos(T), math.sin(T)
        exp = np.stack([A[:, 0] * ct + A[:, 1] * st, -A[:, 0] * st + A[:, 1] * ct], axis=1)
        tol = 8 * (k + 1) * U64 * np.linalg.norm(A, axis=1, keepdims=True)
        assert np.all(np.abs(out - exp) <= tol)


# ---------------------------------------------------------- P2 exact special case
_EXACT = [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0)]


def test_p2_golden_signed_permutation():
    g = read_golden("signed_permutation_2x4.txt")
    A = np.array(g["A"])
    C = np.array(g["C"])
    S = np.array(g["S"])
    R = np.array(g["R"])
    out = oracle.rot_sequence(A, C, S)
    assert np.array_equal(out, R)


def _track_signed_permutation(n, k, Cc, Ss):
    """Follow where each original column goes, as (source column, sign)."""
    cols = [(j, 1) for j in range(n)]
    for p in range(k):
        for j in range(n - 1):
            c, s = Cc[j, p], Ss[j, p]
            x, y = cols[j], cols[j + 1]
            if (c, s) == (1.0, 0.0):
                continue
            if (c, s) == (-1.0, 0.0):
                cols[j], cols[j + 1] = (x[0], -x[1]), (y[0], -y[1])
            elif (c, s) == (0.0, 1.0):
                cols[j], cols[j + 1] = y, (x[0], -x[1])
            elif (c, s) == (0.0, -1.0):
                cols[j], cols[j + 1] = (y[0], -y[1]), x
            else:
                raise AssertionError
    return cols


@pytest.mark.parametrize("n,k", [(2, 1), (3, 4), (9, 5), (16, 16), (5, 23)])
def test_p2_random_signed_permutations_bit_exact(n, k):
    r = _rng(100 + n * 31 + k)
    m = 6
    A = r.integers(1, 1000, size=(m, n)).astype(np.float64) * r.choice([-1.0, 1.0], size=(m, n))
    idx = r.integers(0, 4, size=(n - 1, k))
    C = np.array([[_EXACT[i][0] for i in row] for row in idx]).reshape(n - 1, k)
    S = np.array([[_EXACT[i][1] for i in row] for row in idx]).reshape(n - 1, k)
    out = oracle.rot_sequence(A, C, S)
    cols = _track_signed_permutation(n, k, C, S)
    exp = np.stack([A[:, src] * sg for (src, sg) in cols], axis=1)
    assert np.array_equal(out, exp)


# ------------------------------------------------------------- P3/P4 invariants
@pytest.mark.parametrize("n,k", [(2, 1), (8, 3), (33, 17), (64, 64), (40, 90)])
def test_p3_identity_gives_orthogonal_q(n, k):
    C, S = wl.rotations(n, k, seed=n + k)
    Q = oracle.rot_sequence(np.eye(n), C, S)
    I = np.eye(n)
    assert np.linalg.norm(Q.T @ Q - I) <= 10 * n * U64 * max(1, k) ** 0.5 * 4
    assert np.linalg.norm(Q @ Q.T - I) <= 10 * n * U64 * max(1, k) ** 0.5 * 4


@pytest.mark.parametrize("n,k", [(8, 3), (33, 17), (40, 90)])
def test_p3_q_from_identity_reproduces_direct_application(n, k):
    """A * Q(identity) equals applying the rotations to A (associativity)."""
    A = wl.matrix(13, n, seed=5)
    C, S = wl.rotations(n, k, seed=6)
    Q = oracle.rot_sequence(np.eye(n), C, S)
    direct = oracle.rot_sequence(A, C, S)
    tol = 4 * (n + 2 * k) * U64 * np.linalg.norm(A, axis=1, keepdims=True)
    assert np.all(np.abs(A @ Q - direct) <= tol)


def test_p4_row_norms_preserved():
    A = wl.matrix(64, 100, seed=7)
    C, S = wl.rotations(100, 48, seed=7)
    out = oracle.rot_sequence(A, C, S)
    n0 = np.linalg.norm(A, axis=1)
    n1 = np.linalg.norm(out, axis=1)
    assert np.all(np.abs(n1 - n0) <= 4 * 48 * U64 * n0 * 2)


# ---------------------------------------------------------------- P5 inverse
def test_p5_inverse_recovers_a():
    A = wl.matrix(20, 50, seed=8)
    C, S = wl.rotations(50, 30, seed=8)
    rec = oracle.rot_sequence_inverse(oracle.rot_sequence(A, C, S), C, S)
    assert np.linalg.norm(rec - A) <= 8 * 30 * U64 * np.linalg.norm(A) * 4


def test_p5_reversed_transposed_sequence_through_forward_only():
    """Flip columns, reverse both axes of C, S, apply forward, flip back: recovers A."""
    A = wl.matrix(20, 37, seed=9)
    C, S = wl.rotations(37, 11, seed=9)
    B = oracle.rot_sequence(A, C, S)
    Cr = C[::-1, ::-1].copy()
    Sr = S[::-1, ::-1].copy()
    rec = oracle.rot_sequence(B[:, ::-1], Cr, Sr)[:, ::-1]
    assert np.linalg.norm(rec - A) <= 8 * 11 * U64 * np.linalg.norm(A) * 8


# ---------------------------------------------------- P6 wavefront == standard
@pytest.mark.parametrize("m,n,k", [(1, 2, 1), (3, 5, 4), (17, 33, 8), (5, 40, 39),
                                   (4, 40, 40), (9, 12, 50), (7, 3, 9), (2, 64, 1)])
def test_p6_wavefront_order_bit_identical(m, n, k):
    A, C, S = wl.problem(m, n, k, seed=m * 1000 + n * 10 + k)
    A[0, 0] = -0.0
    std = oracle.rot_sequence(A, C, S)
    wav = oracle.rot_sequence_wavefront(A, C, S)
    assert np.array_equal(std.view(np.uint64), wav.view(np.uint64))


# ---------------------------------------------------------- P7 row independence
def test_p7_row_subset_bit_identical():
    A, C, S = wl.problem(40, 30, 12, seed=10)
    full = oracle.rot_sequence(A, C, S)
    rows = [0, 3, 4, 17, 39]
    sub = oracle.rot_sequence(A[rows], C, S)
    assert np.array_equal(full[rows].view(np.uint64), sub.view(np.uint64))


# ------------------------------------------------------------- P8 BLAS drot
def test_p8_matches_blas_drot_k1():
    from scipy.linalg.blas import drot
    A, C, S = wl.problem(25, 9, 1, seed=12)
    out = oracle.rot_sequence(A, C, S)
    B = np.array(A, order="F", copy=True)
    for j in range(8):
        x, y = drot(B[:, j].copy(), B[:, j + 1].copy(), C[j, 0], S[j, 0])
        B[:, j], B[:, j + 1] = x, y
    scale = np.abs(A).max()
    assert np.max(np.abs(out - B)) <= 8 * 2 * U64 * scale * 4


# --------------------------------------------------------- P9 exact rationals
@pytest.mark.parametrize("m,n,k", [(2, 3, 2), (3, 4, 3), (1, 6, 4), (4, 5, 5)])
def test_p9_exact_rational_product_bound(m, n, k):
    A, C, S = wl.problem(m, n, k, seed=20 + m + n + k)
    out = oracle.rot_sequence(A, C, S)
    # Exact product A * G(0,0) ... G(n-2,k-1) with the given double c, s.
    E = [[Fraction(float(v)) for v in row] for row in A]
    for p in range(k):
        for j in range(n - 1):
            c, s = Fraction(float(C[j, p])), Fraction(float(S[j, p]))
            for row in E:
                x, y = row[j], row[j + 1]
                row[j], row[j + 1] = c * x + s * y, -s * x + c * y
    for i in range(m):
        nrm = float(np.linalg.norm(A[i]))
        bound = 4 * (n - 1) * k * U64 * nrm
        for j in range(n):
            assert abs(Fraction(float(out[i, j])) - E[i][j]) <= Fraction(bound)


# ----------------------------------------------------- Algorithm 4 and rs_gemm
def test_alg4_block_equals_alg2_with_identity_outside():
    """Algorithm 4 applies exactly the rotations of its parallelogram, in order."""
    r = _rng(30)
    nn, kk, m = 11, 4, 5
    A = r.standard_normal((m, nn + 1)) + 3.0  # no zeros in the data
    C, S = wl.rotations(nn + 1, kk, seed=31)
    blk = oracle.rot_sequence_block(A, C, S)
    Cm, Sm = C.copy(), S.copy()
    for p in range(kk):
        for j in range(nn):
            if not (kk - 1 - p <= j < nn - p):
                Cm[j, p], Sm[j, p] = 1.0, 0.0
    ref = oracle.rot_sequence(A, Cm, Sm)
    assert np.array_equal(blk, ref)


@pytest.mark.parametrize("n,k,nb,kb,w0,p0", [(40, 9, 8, 4, 0, 0), (40, 9, 8, 4, 16, 4),
                                             (40, 9, 8, 4, 40, 8), (300, 64, 256, 64, 256, 0)])
def test_form_block_orthogonal_and_structured(n, k, nb, kb, w0, p0):
    C, S = wl.rotations(n, k, seed=40)
    Q = oracle.form_block(C, S, n, w0, nb, p0, kb)
    L = nb + kb
    assert np.linalg.norm(Q.T @ Q - np.eye(L)) <= 10 * L * U64 * 8
    # Row i can only reach columns >= i - kb: the lower-left triangle stays zero.
    ii, jj = np.nonzero(Q)
    assert np.all(jj >= ii - kb)


@pytest.mark.parametrize("n,k,nb,kb", [(600, 130, 256, 64), (300, 40, 64, 16), (130, 70, 32, 32),
                                       (200, 50, 16, 48)])
def test_every_block_of_a_schedule_has_the_zero_triangle(n, k, nb, kb):
    """Every block of the apply order, edge blocks and short p-blocks
    included, is zero at (i, j) for j < i - kb; the tensor-core apply skips
    the products that only meet these zeros."""
    C, S = wl.rotations(n, k, seed=41)
    for w0, p0 in oracle.block_schedule(n, k, nb, kb):
        ii, jj = np.nonzero(oracle.form_block(C, S, n, w0, nb, p0, kb))
        assert np.all(jj >= ii - kb), (w0, p0)


@pytest.mark.parametrize("n,k,nb,kb,w0,p0", [(40, 9, 8, 4, 16, 4), (40, 9, 8, 4, 32, 8),
                                             (300, 64, 256, 64, 256, 0), (600, 130, 256, 64, 0, 128)])
def test_form_block_f32_within_rotation_error_of_f64(n, k, nb, kb, w0, p0):
    """The FP32 block against the FP64 one.  A block's rotations fall into
    about L + 2kb sets of disjoint pairs (one per anti-diagonal j + 2p), and
    each set perturbs a row by a few units of FP32 rounding (the rounded
    (c,s) and the four operations), so every row stays within
    6 (L + 2kb) u32 of the FP64 row; it is also orthogonal to that order and
    keeps the zero triangle."""
    C, S = wl.rotations(n, k, seed=42)
    Q64 = oracle.form_block(C, S, n, w0, nb, p0, kb)
    Q32 = oracle.form_block_f32(C, S, n, w0, nb, p0, kb)
    L = nb + kb
    assert Q32.dtype == np.float32 and Q32.shape == (L, L)
    err = np.linalg.norm(Q32.astype(np.float64) - Q64, axis=1)
    assert err.max() <= 6 * (L + 2 * kb) * U32
    assert err.max() > 0                      # it did round
    Qd = Q32.astype(np.float64)
    assert np.abs(Qd.T @ Qd - np.eye(L)).max() <= 12 * (L + 2 * kb) * U32
    ii, jj = np.nonzero(Q32)
    assert np.all(jj >= ii - kb)


def test_form_block_f32_exact_for_signed_permutations():
    """With c, s in {0, +-1} every operation is exact in any precision, so the
    FP32 block equals the FP64 one entry for entry."""
    n, k, nb, kb = 70, 12, 16, 8
    rng = _rng(43)
    pick = rng.integers(0, 4, size=(n - 1, k))
    C = np.choose(pick, [1.0, 0.0, 0.0, -1.0])
    S = np.choose(pick, [0.0, 1.0, -1.0, 0.0])
    for w0, p0 in oracle.block_schedule(n, k, nb, kb):
        Q64 = oracle.form_block(C, S, n, w0, nb, p0, kb)
        Q32 = oracle.form_block_f32(C, S, n, w0, nb, p0, kb)
        assert np.array_equal(Q32.astype(np.float64), Q64), (w0, p0)


@pytest.mark.parametrize("m,n,k,nb,kb", [(9, 40, 9, 8, 4), (5, 70, 20, 16, 8), (3, 12, 30, 4, 4),
                                         (16, 300, 64, 64, 16)])
def test_gemm_regrouping_equals_rotations(m, n, k, nb, kb):
    A, C, S = wl.problem(m, n, k, seed=50 + n)
    direct = oracle.rot_sequence(A, C, S)
    viaq = oracle.rot_sequence_gemm(A, C, S, nb, kb)
    tol = 16 * (k + nb + kb) * U64 * np.linalg.norm(A, axis=1, keepdims=True)
    assert np.all(np.abs(viaq - direct) <= tol)


# ----------------------------------------------------------------- FP32 oracle
def test_f32_within_stated_error_of_f64():
    A, C, S = wl.problem(32, 200, 40, seed=60)
    ref = oracle.rot_sequence(A, C, S)
    out = oracle.rot_sequence_f32(A.astype(np.float32), C.astype(np.float32), S.astype(np.float32))
    rel = np.linalg.norm(out.astype(np.float64) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 8 * 40 * U32


def test_f32_exact_special_case():
    g = read_golden("signed_permutation_2x4.txt")
    out = oracle.rot_sequence_f32(np.array(g["A"]), np.array(g["C"]), np.array(g["S"]))
    assert np.array_equal(out, np.array(g["R"], dtype=np.float32))


# ------------------------------------------------------------ degenerate sizes
@pytest.mark.parametrize("m,n,k", [(0, 5, 3), (4, 1, 3), (4, 5, 0), (4, 0, 0)])
def test_degenerate_sizes_are_noops(m, n, k):
    A = np.arange(m * n, dtype=np.float64).reshape(m, n)
    C = np.ones((max(n - 1, 0), k))
    S = np.zeros((max(n - 1, 0), k))
    out = oracle.rot_sequence(A, C, S)
    assert np.array_equal(out, A)


# ------------------------------------------------------------ 2x2 reflectors
def test_reflector_closed_form_exact_rational_bound():
    """x' = x - tau(x + nu y), y' = y - nu tau (x + nu y), to within a few roundings."""
    r = _rng(70)
    for _ in range(200):
        x, y = r.standard_normal(2)
        nu = math.tan(r.uniform(-math.pi / 4, math.pi / 4))
        tau = 2.0 / (1.0 + nu * nu)
        out = oracle.refl_sequence(np.array([[x, y]]), np.array([[tau]]), np.array([[nu]]))
        fx, fy, ft, fn = map(Fraction, (x, y, tau, nu))
        t = fx + fn * fy
        ex, ey = fx - ft * t, fy - fn * ft * t
        b = Fraction(8 * U64 * (abs(x) + abs(y) + 1.0))
        assert abs(Fraction(float(out[0, 0])) - ex) <= b
        assert abs(Fraction(float(out[0, 1])) - ey) <= b


def test_reflector_is_an_involution_and_reverse_undoes_a_sequence():
    A = wl.matrix(10, 30, seed=71)
    T, V = wl.reflectors(30, 9, seed=71)
    one = oracle.refl_sequence(A, T[:, :1], V[:, :1])
    # H H = I for one sequence applied twice in reverse order
    back = oracle.refl_sequence_reverse(oracle.refl_sequence(A, T, V), T, V)
    assert np.linalg.norm(back - A) <= 64 * 9 * 30 * U64 * np.linalg.norm(A)
    assert not np.allclose(one, A)


def test_reflectors_orthogonal_and_norm_preserving():
    n, k = 40, 17
    T, V = wl.reflectors(n, k, seed=72)
    Q = oracle.refl_sequence(np.eye(n), T, V)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 16 * n * k * U64
    # det = (-1)^(number of reflectors)
    assert np.sign(np.linalg.det(Q)) == (-1) ** ((n - 1) * k)
    A = wl.matrix(25, n, seed=73)
    out = oracle.refl_sequence(A, T, V)
    n0, n1 = np.linalg.norm(A, axis=1), np.linalg.norm(out, axis=1)
    assert np.all(np.abs(n1 - n0) <= 16 * k * U64 * n0 * 4)


def test_reflector_matches_matrix_definition():
    """Each step equals multiplying by the 2x2 matrix I - tau v v^T (k = 1, n = 2, many rows)."""
    A = wl.matrix(50, 2, seed=74)
    T, V = wl.reflectors(2, 1, seed=74)
    tau, nu = T[0, 0], V[0, 0]
    H = np.eye(2) - tau * np.outer([1.0, nu], [1.0, nu])
    out = oracle.refl_sequence(A, T, V)
    assert np.max(np.abs(out - A @ H)) <= 16 * U64 * np.abs(A).max()


# ------------------------------------------------------- rotations from the left
@pytest.mark.parametrize("m,n,k", [(2, 3, 1), (9, 5, 4), (33, 17, 12), (40, 1, 3)])
def test_left_application_is_the_transpose_of_right_application(m, n, k):
    """Rotating rows of A equals Algorithm 2 on A^T, bit for bit (same operations per element)."""
    A = wl.matrix(m, n, seed=80 + m)
    C, S = wl.rotations(m, k, seed=81 + k)
    left = oracle.rot_sequence_left(A, C, S)
    right = oracle.rot_sequence(np.asfortranarray(A.T), C, S).T
    assert np.array_equal(left.view(np.uint64), np.ascontiguousarray(right).view(np.uint64))


def test_left_application_orthogonal_and_golden():
    # rows of the golden signed permutation example become columns of A^T
    g = read_golden("signed_permutation_2x4.txt")
    A = np.array(g["A"]).T            # 4 x 2: rotations now act on rows
    out = oracle.rot_sequence_left(A, np.array(g["C"]), np.array(g["S"]))
    assert np.array_equal(out, np.array(g["R"]).T)
    C, S = wl.rotations(30, 9, seed=82)
    Q = oracle.rot_sequence_left(np.eye(30), C, S)
    assert np.linalg.norm(Q @ Q.T - np.eye(30)) <= 16 * 30 * 9 * U64
