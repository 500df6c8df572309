// rs_left.cu -- rotations applied from the left (to rows j, j+1 of A).
//
// Rotating rows of a column-major A is Algorithm 2 on A^T.  The wave kernel
// streams columns with one row per lane, so the GB300 path transposes A into
// a scratch matrix (32 x 32 tiles through shared memory, coalesced on both
// sides), runs the column kernel on it and transposes back.  The kernel is
// bound by the FP64 pipe with DRAM about 1 % busy, so the two extra passes
// over A cost well under 1 % of the run.
#include <algorithm>
#include <cuda_runtime.h>
#include "rs_internal.h"

namespace rs {
namespace {

// dst = src^T: src is rows x cols (leading dimension lds), dst is cols x rows
// (leading dimension ldd), both column-major.
__global__ void transpose_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                                 int64_t ldd, int rows, int cols) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r0 = blockIdx.x * 32;
  for (int c0 = blockIdx.y * 32; c0 < cols; c0 += gridDim.y * 32) {
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
      const int r = r0 + tx, c = c0 + ty + i;
      if (r < rows && c < cols) tile[ty + i][tx] = src[(int64_t)r + (int64_t)c * lds];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
      const int c = c0 + tx, r = r0 + ty + i;
      if (r < rows && c < cols) dst[(int64_t)c + (int64_t)r * ldd] = tile[tx][ty + i];
    }
    __syncthreads();
  }
}

cudaError_t transpose(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                      cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd((unsigned)((rows + 31) / 32), (unsigned)std::min<int64_t>((cols + 31) / 32, 65535));
  transpose_kernel<<<grd, blk, 0, s>>>(src, lds, dst, ldd, (int)rows, (int)cols);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace rs

extern "C" rot_status rot_apply_left(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                                     int64_t ldc, const double* S, int64_t lds, void* stream) {
  const int64_t lim = (int64_t(1) << 31) - 1;
  if (m < 0 || n < 0 || k < 0) return ROT_EINVAL;
  if (m > lim || n > lim || k > lim || m + k > lim) return ROT_EINVAL;
  if (lda < std::max<int64_t>(1, m)) return ROT_EINVAL;
  const int64_t mm1 = std::max<int64_t>(1, m - 1);
  if (ldc < mm1 || lds < mm1) return ROT_EINVAL;
  if (n == 0 || m <= 1 || k == 0) return ROT_OK;
  if (!A || !C || !S) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* B = nullptr;                                  // A^T, n x m, leading dimension n
  cudaError_t e = cudaMallocAsync((void**)&B, (size_t)n * (size_t)m * sizeof(double), s);
  if (e != cudaSuccess) { cudaGetLastError(); return ROT_ENOMEM; }
  rot_status st = ROT_OK;
  do {
    e = rs::transpose(A, lda, B, n, m, n, s);
    if (e != cudaSuccess) { st = rs::cuda_failed(e, "rot_apply_left: transpose"); break; }
    st = rs::apply_f64(n, m, k, B, n, C, ldc, S, lds, s);     // the same dispatch as rot_apply
    if (st != ROT_OK) break;
    e = rs::transpose(B, n, A, lda, n, m, s);
    if (e != cudaSuccess) { st = rs::cuda_failed(e, "rot_apply_left: transpose back"); break; }
  } while (0);
  cudaFreeAsync(B, s);
  return st;
}
