/*
 * rot_oracle.c -- plain, slow, obviously correct CPU reference for applying a
 * sequence of planar (Givens) rotations to the columns of a matrix
 * (Steel & Langou, "Communication efficient application of sequences of
 * planar rotations to a matrix").
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke() entry of
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load this file.
 * It shares no code, header or table with the CUDA library and includes none
 * of it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared rot_oracle.c -lm
 * -ffp-contract=off is required: every product below is a separately rounded
 * IEEE multiply, every fma() is one fused multiply-add (C99 fma, round to
 * nearest even).
 *
 * Storage conventions (all column-major, as the paper's A is, Section 4 fig.):
 *   A(i,j) = A[i + j*lda],   0 <= i < m, 0 <= j < n
 *   C(j,p) = C[j + p*ldc],   S(j,p) = S[j + p*lds],   0 <= j < n-1, 0 <= p < k
 * Rotation (j,p) acts on columns j and j+1 of A with (c,s) = (C(j,p),S(j,p)).
 *
 * Fused-multiply-add placement (the paper does not fix one; this is the
 * reading used everywhere in this project):
 *     x' = fma(c, x,  RN(s*y))
 *     y' = fma(c, y, -RN(s*x))
 * i.e. Algorithm 1's  t = c*x + s*y ;  y = -s*x + c*y ;  x = t  with the
 * s-products rounded first.  Parity of the GPU FP64 path is bit-exact
 * against these functions.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* Algorithm 1 (rot): apply one rotation to two length-m vectors x, y. */
static void rot_f64(int64_t m, double *x, double *y, double c, double s)
{
    for (int64_t i = 0; i < m; ++i) {
        double xi = x[i], yi = y[i];
        double sy = s * yi;           /* rounded product */
        double sx = s * xi;           /* rounded product */
        double t = fma(c, xi, sy);    /* t = c*x + s*y   */
        y[i] = fma(c, yi, -sx);       /* y = -s*x + c*y  */
        x[i] = t;
    }
}

static void rot_f32(int64_t m, float *x, float *y, float c, float s)
{
    for (int64_t i = 0; i < m; ++i) {
        float xi = x[i], yi = y[i];
        float sy = s * yi;
        float sx = s * xi;
        float t = fmaf(c, xi, sy);
        y[i] = fmaf(c, yi, -sx);
        x[i] = t;
    }
}

/* Algorithm 1 exported on its own, for the closed-form pins. */
void oracle_rot(int64_t m, double *x, double *y, double c, double s)
{
    rot_f64(m, x, y, c, s);
}

/*
 * Algorithm 2 (rot_sequence): for p = 0..k-1, for j = 0..n-2, apply rotation
 * (j,p) to columns j, j+1.  This is the definition of the result.
 */
void oracle_rot_sequence(int64_t m, int64_t n, int64_t k,
                         double *A, int64_t lda,
                         const double *C, int64_t ldc,
                         const double *S, int64_t lds)
{
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j + 1 < n; ++j)
            rot_f64(m, A + j * lda, A + (j + 1) * lda, C[j + p * ldc], S[j + p * lds]);
}

/* Algorithm 2 in single precision (FP32 data, FP32 rotations, fmaf). */
void oracle_rot_sequence_f32(int64_t m, int64_t n, int64_t k,
                             float *A, int64_t lda,
                             const float *C, int64_t ldc,
                             const float *S, int64_t lds)
{
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j + 1 < n; ++j)
            rot_f32(m, A + j * lda, A + (j + 1) * lda, C[j + p * ldc], S[j + p * lds]);
}

/*
 * Algorithm 3 (rot_sequence_wavefront), read as: for wave w = 0 .. (n-2)+(k-1),
 * apply rotations (j = w-l, p = l) for l = max(0, w-(n-2)) .. min(k-1, w) in
 * increasing l, i.e. (w,0), (w-1,1), (w-2,2), ... as Section 1.1 describes.
 * The printed startup/pipeline/shutdown loop bounds are garbled (their inner
 * condition and the sequence index of C/S do not match that description);
 * this single loop covers all three phases and any k, including k > n-1.
 */
void oracle_rot_sequence_wavefront(int64_t m, int64_t n, int64_t k,
                                   double *A, int64_t lda,
                                   const double *C, int64_t ldc,
                                   const double *S, int64_t lds)
{
    if (n < 2 || k < 1) return;
    int64_t nwaves = (n - 1) + (k - 1);
    for (int64_t w = 0; w < nwaves; ++w) {
        int64_t lo = w - (n - 2);
        if (lo < 0) lo = 0;
        int64_t hi = w < k - 1 ? w : k - 1;
        for (int64_t l = lo; l <= hi; ++l) {
            int64_t j = w - l;
            rot_f64(m, A + j * lda, A + (j + 1) * lda, C[j + l * ldc], S[j + l * lds]);
        }
    }
}

/*
 * Inverse of Algorithm 2: the transpose of G(j,p) is the rotation with
 * (c, -s); apply them in reverse order (p = k-1..0, j = n-2..0).
 */
void oracle_rot_sequence_inverse(int64_t m, int64_t n, int64_t k,
                                 double *A, int64_t lda,
                                 const double *C, int64_t ldc,
                                 const double *S, int64_t lds)
{
    for (int64_t p = k - 1; p >= 0; --p)
        for (int64_t j = n - 2; j >= 0; --j)
            rot_f64(m, A + j * lda, A + (j + 1) * lda, C[j + p * ldc], -S[j + p * lds]);
}

/*
 * Algorithm 4 (rot_sequence_block) with its printed loop bounds:
 * for p = 0..kk-1, for j = kk-1-p .. nn-p-1, rotation (j,p) on columns j, j+1.
 * It touches columns 0..nn of A (nn+1 columns) and rows 0..nn-1 of C, S:
 * nn-kk+1 waves of kk rotations with no startup or shutdown triangle.
 */
void oracle_rot_sequence_block(int64_t m, int64_t nn, int64_t kk,
                               double *A, int64_t lda,
                               const double *C, int64_t ldc,
                               const double *S, int64_t lds)
{
    for (int64_t p = 0; p < kk; ++p)
        for (int64_t j = kk - 1 - p; j < nn - p; ++j)
            rot_f64(m, A + j * lda, A + (j + 1) * lda, C[j + p * ldc], S[j + p * lds]);
}

/*
 * Accumulated block of the "rs_gemm" method (Section 8, rs_gemm): the
 * orthogonal matrix that one parallelogram block of rotations applies.
 * The block holds the rotations (j,p) of sequences p in [p0, p0+kb) whose
 * wave index relative to the block, w = j + (p - p0), lies in [w0, w0+nb),
 * restricted to 0 <= j <= n-2 and p < k.  They touch columns
 * [c0, c0+L) with c0 = w0 - kb + 1 and L = nb + kb; Q (L x L, leading
 * dimension ldq) starts as the identity and receives those rotations on its
 * columns (j - c0, j - c0 + 1) in Algorithm 2 order (p outer, j inner).
 * Then A(:, c0:c0+L) * Q equals applying the block to A (columns of the
 * window outside [0, n) are never touched and stay identity).
 */
void oracle_form_block(int64_t n, int64_t k,
                       int64_t w0, int64_t nb, int64_t p0, int64_t kb,
                       const double *C, int64_t ldc,
                       const double *S, int64_t lds,
                       double *Q, int64_t ldq)
{
    int64_t L = nb + kb;
    int64_t c0 = w0 - kb + 1;
    for (int64_t jj = 0; jj < L; ++jj)
        for (int64_t ii = 0; ii < L; ++ii)
            Q[ii + jj * ldq] = (ii == jj) ? 1.0 : 0.0;
    for (int64_t p = p0; p < p0 + kb && p < k; ++p) {
        for (int64_t j = 0; j + 1 < n; ++j) {
            int64_t w = j + (p - p0);
            if (w < w0 || w >= w0 + nb) continue;
            int64_t col = j - c0;
            rot_f64(L, Q + col * ldq, Q + (col + 1) * ldq, C[j + p * ldc], S[j + p * lds]);
        }
    }
}

/*
 * The same accumulated block in single precision: each (c,s) is rounded to
 * the nearest FP32 value and the block's rotations are applied to the FP32
 * identity with rot_f32, in the order of oracle_form_block.
 */
void oracle_form_block_f32(int64_t n, int64_t k,
                           int64_t w0, int64_t nb, int64_t p0, int64_t kb,
                           const double *C, int64_t ldc,
                           const double *S, int64_t lds,
                           float *Q, int64_t ldq)
{
    int64_t L = nb + kb;
    int64_t c0 = w0 - kb + 1;
    for (int64_t jj = 0; jj < L; ++jj)
        for (int64_t ii = 0; ii < L; ++ii)
            Q[ii + jj * ldq] = (ii == jj) ? 1.0f : 0.0f;
    for (int64_t p = p0; p < p0 + kb && p < k; ++p) {
        for (int64_t j = 0; j + 1 < n; ++j) {
            int64_t w = j + (p - p0);
            if (w < w0 || w >= w0 + nb) continue;
            int64_t col = j - c0;
            rot_f32(L, Q + col * ldq, Q + (col + 1) * ldq, (float)C[j + p * ldc], (float)S[j + p * lds]);
        }
    }
}

/*
 * 2x2 reflectors in place of rotations (Section 6): the reflector (tau, nu)
 * is H = I - tau * v v^T with v = (1, nu)^T; applied to a row [x, y] it gives
 *     x' = x - tau*(x + nu*y),   y' = y - nu*tau*(x + nu*y),
 * three multiplications and three additions.  Placement of the fused
 * operations (the paper fixes none; this is the reading used here):
 *     t = fma(nu, y, x),  w = RN(tau*t),  x' = RN(x - w),  y' = fma(-nu, w, y).
 * T(j,p) = T[j + p*ldt] holds tau, V(j,p) = V[j + p*ldv] holds nu; the
 * reflectors are applied in Algorithm 2's order.
 */
static void refl_f64(int64_t m, double *x, double *y, double tau, double nu)
{
    for (int64_t i = 0; i < m; ++i) {
        double xi = x[i], yi = y[i];
        double t = fma(nu, yi, xi);
        double w = tau * t;
        x[i] = xi - w;
        y[i] = fma(-nu, w, yi);
    }
}

void oracle_refl_sequence(int64_t m, int64_t n, int64_t k,
                          double *A, int64_t lda,
                          const double *T, int64_t ldt,
                          const double *V, int64_t ldv)
{
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j + 1 < n; ++j)
            refl_f64(m, A + j * lda, A + (j + 1) * lda, T[j + p * ldt], V[j + p * ldv]);
}

/* The same reflectors in reverse order (each 2x2 reflector is its own inverse). */
void oracle_refl_sequence_reverse(int64_t m, int64_t n, int64_t k,
                                  double *A, int64_t lda,
                                  const double *T, int64_t ldt,
                                  const double *V, int64_t ldv)
{
    for (int64_t p = k - 1; p >= 0; --p)
        for (int64_t j = n - 2; j >= 0; --j)
            refl_f64(m, A + j * lda, A + (j + 1) * lda, T[j + p * ldt], V[j + p * ldv]);
}

/*
 * Rotations applied from the left, to rows: for p = 0..k-1, j = 0..m-2,
 * Algorithm 1 on the row vectors x = A(j,:), y = A(j+1,:) with
 * (c, s) = (C(j,p), S(j,p)); C and S are (m-1) x k.  This is Algorithm 2 on
 * A^T, written directly on the rows of the column-major A.
 */
void oracle_rot_sequence_left(int64_t m, int64_t n, int64_t k,
                              double *A, int64_t lda,
                              const double *C, int64_t ldc,
                              const double *S, int64_t lds)
{
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j + 1 < m; ++j) {
            double c = C[j + p * ldc], s = S[j + p * lds];
            for (int64_t i = 0; i < n; ++i) {
                double xi = A[j + i * lda], yi = A[j + 1 + i * lda];
                double sy = s * yi;
                double sx = s * xi;
                A[j + i * lda] = fma(c, xi, sy);
                A[j + 1 + i * lda] = fma(c, yi, -sx);
            }
        }
}
