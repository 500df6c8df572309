/*
 * rot_cpu_parallel.c -- multi-core CPU baseline for applying a sequence of
 * planar rotations to the columns of a matrix (Steel & Langou, Section 7:
 * threads apply the same rotations to different row blocks of A; Algorithm 3's
 * wave order inside each block).
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE, NOT PRODUCT CODE.  This is the timed
 * CPU baseline that bench.py reports beside the GPU; the tests check it bit for
 * bit against the oracle in rot_oracle.c.  It shares no code, header or table
 * with the CUDA library and includes none of it, and it shares no code with
 * the oracle either (it restates Algorithm 1 itself).
 *
 * Build: gcc -O3 -fopenmp -ffp-contract=off -fPIC -shared rot_cpu_parallel.c -lm
 * (without -fopenmp it runs on one thread).  -ffp-contract=off keeps every
 * product a separately rounded multiply, so the result is bit-identical to the
 * oracle: the same fused multiply-add placement,
 *     x' = fma(c, x, RN(s*y)),   y' = fma(c, y, -RN(s*x)),
 * and every element sees the same operations in the same order.  Why the order
 * is the same:
 *   - rows are independent (each row a_i is updated as a_i <- a_i * G), so a
 *     thread may take any block of rows;
 *   - inside a block, sequences are taken kb at a time (p-blocks, Section 2)
 *     and inside a p-block wave w = j + (p - p0) runs its rotations in
 *     increasing p (Algorithm 3's reading of Section 1.1).  Rotations that
 *     share a column keep Algorithm 2's relative order, and rotations on
 *     disjoint column pairs commute exactly.
 *
 * Layout as in rot_oracle.c: A(i,j) = A[i + j*lda], C(j,p) = C[j + p*ldc],
 * S(j,p) = S[j + p*lds], all column-major.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One rotation (Algorithm 1) on mr consecutive rows of columns x and y. */
static inline void rot_rows(int64_t mr, double *restrict x, double *restrict y, double c, double s)
{
    for (int64_t i = 0; i < mr; ++i) {
        const double xi = x[i], yi = y[i];
        const double sy = s * yi;
        const double sx = s * xi;
        x[i] = fma(c, xi, sy);
        y[i] = fma(c, yi, -sx);
    }
}

/* Rows [i0, i0+mr) of A, every rotation, p-block by p-block in wave order. */
static void apply_row_block(int64_t i0, int64_t mr, int64_t n, int64_t k, double *A, int64_t lda,
                            const double *C, int64_t ldc, const double *S, int64_t lds, int64_t kb)
{
    for (int64_t p0 = 0; p0 < k; p0 += kb) {
        const int64_t kr = (k - p0 < kb) ? k - p0 : kb;
        const int64_t nwaves = (n - 1) + kr - 1;
        for (int64_t w = 0; w < nwaves; ++w) {
            const int64_t lo = (w - (n - 2) > 0) ? w - (n - 2) : 0;
            const int64_t hi = (w < kr - 1) ? w : kr - 1;
            for (int64_t l = lo; l <= hi; ++l) {
                const int64_t j = w - l, p = p0 + l;
                rot_rows(mr, A + i0 + j * lda, A + i0 + (j + 1) * lda, C[j + p * ldc], S[j + p * lds]);
            }
        }
    }
}

/*
 * Algorithm 2's result on `threads` host threads (0: all that OpenMP offers).
 * Row blocks of mb rows are handed out dynamically; kb sequences are fused per
 * pass over a block.  Returns the number of threads that ran (1 without
 * OpenMP).  m, n, k >= 0; quick return when m == 0, n <= 1 or k == 0.
 */
int cpu_rot_sequence_parallel(int64_t m, int64_t n, int64_t k, double *A, int64_t lda,
                              const double *C, int64_t ldc, const double *S, int64_t lds,
                              int64_t mb, int64_t kb, int threads)
{
    int used = 1;
    if (m <= 0 || n <= 1 || k <= 0) return used;
    if (mb < 1) mb = 32;
    if (kb < 1) kb = 32;
    const int64_t nblk = (m + mb - 1) / mb;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel num_threads(threads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nblk; ++b) {
            const int64_t i0 = b * mb;
            const int64_t mr = (m - i0 < mb) ? m - i0 : mb;
            apply_row_block(i0, mr, n, k, A, lda, C, ldc, S, lds, kb);
        }
    }
#else
    (void)threads;
    for (int64_t b = 0; b < nblk; ++b) {
        const int64_t i0 = b * mb;
        const int64_t mr = (m - i0 < mb) ? m - i0 : mb;
        apply_row_block(i0, mr, n, k, A, lda, C, ldc, S, lds, kb);
    }
#endif
    return used;
}
