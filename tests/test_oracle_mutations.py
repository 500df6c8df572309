"""Plant plausible mistakes in a copy of the oracle's C source and check that the pins catch each.

Every mutant is compiled with the same flags into a temporary directory and
swapped in through ``oracle.use_library``; the pins of ``test_oracle_pins`` are
then run against it and at least one must fail.  Nothing here touches a GPU.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rot_oracle.c")

PINS = [
    pins.test_p1_closed_form_single_rotation_golden,
    pins.test_p1_single_rotation_exact_rational_bound,
    pins.test_p1_n2_composition_equals_sum_of_angles,
    pins.test_p2_golden_signed_permutation,
    lambda: pins.test_p2_random_signed_permutations_bit_exact(9, 5),
    lambda: pins.test_p3_identity_gives_orthogonal_q(33, 17),
    lambda: pins.test_p3_q_from_identity_reproduces_direct_application(33, 17),
    pins.test_p4_row_norms_preserved,
    pins.test_p5_inverse_recovers_a,
    pins.test_p5_reversed_transposed_sequence_through_forward_only,
    lambda: pins.test_p6_wavefront_order_bit_identical(17, 33, 8),
    pins.test_p7_row_subset_bit_identical,
    pins.test_p8_matches_blas_drot_k1,
    lambda: pins.test_p9_exact_rational_product_bound(3, 4, 3),
    pins.test_alg4_block_equals_alg2_with_identity_outside,
    lambda: pins.test_form_block_orthogonal_and_structured(40, 9, 8, 4, 16, 4),
    lambda: pins.test_form_block_f32_within_rotation_error_of_f64(40, 9, 8, 4, 16, 4),
    pins.test_form_block_f32_exact_for_signed_permutations,
    lambda: pins.test_gemm_regrouping_equals_rotations(5, 70, 20, 16, 8),
    pins.test_f32_within_stated_error_of_f64,
    pins.test_f32_exact_special_case,
    pins.test_reflector_closed_form_exact_rational_bound,
    pins.test_reflector_is_an_involution_and_reverse_undoes_a_sequence,
    pins.test_reflectors_orthogonal_and_norm_preserving,
    pins.test_reflector_matches_matrix_definition,
    lambda: pins.test_left_application_is_the_transpose_of_right_application(33, 17, 12),
    pins.test_left_application_orthogonal_and_golden,
]

# (name, text to find, replacement, occurrence index among matches)
MUTANTS = [
    ("y_sign", "y[i] = fma(c, yi, -sx);", "y[i] = fma(c, yi, sx);", 0),
    ("x_sign", "double t = fma(c, xi, sy);", "double t = fma(c, xi, -sy);", 0),
    ("wrong_factor", "double sy = s * yi;", "double sy = c * yi;", 0),
    ("dropped_term", "double sx = s * xi;", "double sx = 0.0 * xi;", 0),
    ("s_from_c", "C[j + p * ldc], S[j + p * lds]);", "C[j + p * ldc], C[j + p * ldc]);", 0),
    ("swapped_columns", "rot_f64(m, A + j * lda, A + (j + 1) * lda, C[j + p * ldc]",
     "rot_f64(m, A + (j + 1) * lda, A + j * lda, C[j + p * ldc]", 0),
    ("reversed_sequences", "C[j + p * ldc], S[j + p * lds]);",
     "C[j + (k - 1 - p) * ldc], S[j + (k - 1 - p) * lds]);", 0),
    ("loop_order", "    for (int64_t p = 0; p < k; ++p)\n        for (int64_t j = 0; j + 1 < n; ++j)\n"
                   "            rot_f64(",
     "    for (int64_t j = 0; j + 1 < n; ++j)\n        for (int64_t p = 0; p < k; ++p)\n"
     "            rot_f64(", 0),
    ("wave_order", "for (int64_t l = lo; l <= hi; ++l)", "for (int64_t l = hi; l >= lo; --l)", 0),
    ("inverse_sign", "-S[j + p * lds]);", "S[j + p * lds]);", 0),
    ("block_bounds", "for (int64_t j = kk - 1 - p; j < nn - p; ++j)",
     "for (int64_t j = kk - 1 - p; j < nn - p - 1; ++j)", 0),
    ("form_block_cs", "C[j + p * ldc], S[j + p * lds]);\n        }\n    }\n}",
     "S[j + p * lds], C[j + p * ldc]);\n        }\n    }\n}", 0),
    ("form_block_f32_cs", "(float)C[j + p * ldc], (float)S[j + p * lds]",
     "(float)S[j + p * lds], (float)C[j + p * ldc]", 0),
    ("form_block_f32_window", "if (w < w0 || w >= w0 + nb) continue;",
     "if (w < w0 || w >= w0 + nb - 1) continue;", 1),
    ("form_block_f32_identity", "Q[ii + jj * ldq] = (ii == jj) ? 1.0f : 0.0f;",
     "Q[ii + jj * ldq] = (ii + 1 == jj) ? 1.0f : 0.0f;", 0),
    ("f32_sign", "y[i] = fmaf(c, yi, -sx);", "y[i] = fmaf(c, yi, sx);", 0),
    ("refl_sign", "y[i] = fma(-nu, w, yi);", "y[i] = fma(nu, w, yi);", 0),
    ("refl_dropped", "double t = fma(nu, yi, xi);", "double t = xi;", 0),
    ("refl_tau", "double w = tau * t;", "double w = nu * t;", 0),
    ("left_rows", "double xi = A[j + i * lda], yi = A[j + 1 + i * lda];",
     "double xi = A[j + i * lda], yi = A[j + (i + 1) % n * lda];", 0),
    ("left_sign", "A[j + 1 + i * lda] = fma(c, yi, -sx);", "A[j + 1 + i * lda] = fma(c, yi, sx);", 0),
]


def _mutate(text, find, repl, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = text.index(find, pos + 1)
    return text[:pos] + repl + text[pos + len(find):]


@pytest.mark.parametrize("name,find,repl,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, find, repl, occ):
    src = open(SRC).read()
    mutated = _mutate(src, find, repl, occ)
    assert mutated != src
    c = tmp_path / ("m_%s.c" % name)
    so = tmp_path / ("m_%s.so" % name)
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), "-lm"], check=True)
    prev = oracle.use_library(str(so))
    failed = []
    try:
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failed.append(getattr(pin, "__name__", "lambda"))
    finally:
        oracle.restore_library(prev)
    assert failed, "mutant %s passed every pin" % name
