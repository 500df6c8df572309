// rs_packed.cu -- the packed resident layout (the paper's pre-packed A of
// rs_kernel_v2, Section 4: A copied once into the order the kernel walks it)
// and the rotation entry points that work on it.
//
// Layout: A (m x n) as ceil(m/32) strips of 32 rows, strip s holding rows
// 32s .. 32s+31 as a 32 x n column-major panel (leading dimension 32), the
// strips one after the other:
//     P[(i / 32) * 32 * n + j * 32 + i % 32] = A(i, j),
// rows past m in the last strip are zero padding.  A warp streaming its 32
// rows through the columns then reads and writes one contiguous run of memory
// (128 bytes per column in FP32, 256 in FP64) instead of one run per column
// lda elements apart.
//
// The kernels take the layout through two numbers: the leading dimension
// (32) and the distance between the strips' first rows (32 n).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_internal.h"

namespace rs {
namespace {

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Block (32, 8): lane = row within the strip, y = column; strips on
// blockIdx.x, columns strided over blockIdx.y.  Both sides move 32
// consecutive elements per warp access.
template <typename T>
__global__ void pack_kernel(const T* __restrict__ A, int64_t lda, int m, int n, T* __restrict__ P) {
  const int strip = blockIdx.x;
  const int row = strip * 32 + threadIdx.x;
  T* dst = P + (int64_t)strip * 32 * n + threadIdx.x;
  for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < n; j += gridDim.y * blockDim.y)
    dst[(int64_t)j * 32] = row < m ? A[row + (int64_t)j * lda] : T(0);
}

template <typename T>
__global__ void unpack_kernel(const T* __restrict__ P, int m, int n, T* __restrict__ A, int64_t lda) {
  const int strip = blockIdx.x;
  const int row = strip * 32 + threadIdx.x;
  if (row >= m) return;
  const T* src = P + (int64_t)strip * 32 * n + threadIdx.x;
  for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < n; j += gridDim.y * blockDim.y)
    A[row + (int64_t)j * lda] = src[(int64_t)j * 32];
}

constexpr int64_t kLimit = (int64_t(1) << 31) - 1;

bool sizes_ok(int64_t m, int64_t n) { return m >= 0 && n >= 0 && m <= kLimit && n <= kLimit; }

template <typename T>
rot_status pack_impl(int64_t m, int64_t n, const T* A, int64_t lda, T* P, void* stream, bool to_packed) {
  if (!sizes_ok(m, n) || lda < (m > 1 ? m : 1)) return ROT_EINVAL;
  if (m == 0 || n == 0) return ROT_OK;
  if (!A || !P) return ROT_EINVAL;
  if (ceil_div(m, 32) > kLimit) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 b(32, 8);
  dim3 g((unsigned)ceil_div(m, 32), (unsigned)std::min<int64_t>(ceil_div(n, 8), 1024));
  if (to_packed) pack_kernel<T><<<g, b, 0, s>>>(A, lda, (int)m, (int)n, P);
  else unpack_kernel<T><<<g, b, 0, s>>>(P, (int)m, (int)n, const_cast<T*>(A), lda);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_failed(e, to_packed ? "rot_pack: launch" : "rot_unpack: launch");
  count_launches(1);
  return ROT_OK;
}

template <typename T>
rot_status apply_packed_impl(int64_t m, int64_t n, int64_t k, T* P, const T* C, int64_t ldc, const T* S,
                             int64_t lds, void* stream) {
  if (m < 0 || n < 0 || k < 0 || m > kLimit || n > kLimit || k > kLimit || n + k > kLimit) return ROT_EINVAL;
  const int64_t nm1 = n - 1 > 1 ? n - 1 : 1;
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) return ROT_OK;
  if (!P || !C || !S) return ROT_EINVAL;
  if (ceil_div(m, 32) * 32 * n > (int64_t(1) << 62) / (int64_t)sizeof(T)) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Few sequences: the column stream over the strips (it needs a 16-byte
  // aligned panel, as TMA does, and at least 64 rows and columns).
  const int64_t kmax = sizeof(T) == 4 ? 48 : 16;
  if (k <= kmax && m >= 64 && n >= 64 && reinterpret_cast<uintptr_t>(P) % 16 == 0)
    return stream_apply<T>(m, n, k, P, 32, C, ldc, S, lds, s, true);
  WaveOptions o{};
  o.chain_stride = 32 * n;
  if constexpr (sizeof(T) == 8) return wave_apply<double>(m, n, k, P, 32, C, ldc, S, lds, s, o);
  else return wave_apply_f32(m, n, k, P, 32, C, ldc, S, lds, s, o);
}

}  // namespace
}  // namespace rs

extern "C" {

int64_t rot_packed_elems(int64_t m, int64_t n) {
  if (m < 0 || n < 0 || m > rs::kLimit || n > rs::kLimit) return -1;
  return rs::ceil_div(m, 32) * 32 * n;
}

rot_status rot_pack(int64_t m, int64_t n, const double* A, int64_t lda, double* P, void* stream) {
  return rs::pack_impl<double>(m, n, A, lda, P, stream, true);
}
rot_status rot_unpack(int64_t m, int64_t n, const double* P, double* A, int64_t lda, void* stream) {
  return rs::pack_impl<double>(m, n, A, lda, const_cast<double*>(P), stream, false);
}
rot_status rot_pack_f32(int64_t m, int64_t n, const float* A, int64_t lda, float* P, void* stream) {
  return rs::pack_impl<float>(m, n, A, lda, P, stream, true);
}
rot_status rot_unpack_f32(int64_t m, int64_t n, const float* P, float* A, int64_t lda, void* stream) {
  return rs::pack_impl<float>(m, n, A, lda, const_cast<float*>(P), stream, false);
}

rot_status rot_apply_packed(int64_t m, int64_t n, int64_t k, double* P, const double* C, int64_t ldc,
                            const double* S, int64_t lds, void* stream) {
  return rs::apply_packed_impl<double>(m, n, k, P, C, ldc, S, lds, stream);
}
rot_status rot_apply_packed_f32(int64_t m, int64_t n, int64_t k, float* P, const float* C, int64_t ldc,
                                const float* S, int64_t lds, void* stream) {
  return rs::apply_packed_impl<float>(m, n, k, P, C, ldc, S, lds, stream);
}

}  // extern "C"
