// rs_stream.cu -- host side of the single-p-block column stream
// (rs_stream.cuh).  rot_apply_f32 takes it for k <= 41 (k <= 48 where the
// lane pipeline does not apply), as passes of at most 8 sequences in
// sequence order (Algorithm 2 applies sequence p entirely before p+1, so the
// passes compute the same thing); a pass of 8 takes 0.30 ms at 8192 x 8192,
// where the wavefront kernel takes 2.0-2.3 ms (k = 16..64).  rot_apply
// (FP64) takes it for k = 1, 2, for k <= 8 while its 32-row strips fit one
// per SM, for k = 3 with up to two per SM, for what the lane pipeline's
// passes leave over, and for k <= 16 where the pipeline does not apply
// (n < 256): on column-major A as passes of at most 4 sequences, each on
// the split stream (stream_split_kernel, two warps a sequence).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_internal.h"
#include "rs_stream.cuh"

namespace rs {
namespace {

inline int64_t round_up256(int64_t x) { return (x + 255) / 256 * 256; }

template <typename T, int KR>
rot_status stream_launch(int64_t m, int64_t n, int64_t k, T* A, int64_t lda, const T* C, int64_t ldc, const T* S,
                         int64_t lds, cudaStream_t s, bool packed) {
  constexpr int R = stream_rows<T, KR>();
  static_assert(R == 1, "the packed layout's strips are 32 rows");
  using SS = StreamShape<T, KR, R>;
  constexpr bool kF64 = sizeof(T) == 8;
  const int64_t W2 = 2 * SS::KP;                   // elements per (c,s) row
  const int64_t cs_rows = n + k;                   // row j + p <= n + k - 3, plus the TMA's reach
  const int64_t cs_bytes = cs_rows * W2 * (int64_t)sizeof(T);
  const int64_t st_off = round_up256(cs_bytes);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, (size_t)(st_off + 256), s) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  T* cs = reinterpret_cast<T*>(base);
  int* status = reinterpret_cast<int*>(base + st_off);
  rot_status st = ROT_OK;
  do {
    // Pairs the repack does not write are only read by rotations that do not exist.
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) { st = cuda_failed(e, "stream: memset"); break; }
    dim3 rb(32, 8);
    dim3 rg((unsigned)((n - 1 + 31) / 32), (unsigned)((k + 7) / 8));
    repack_cs_kernel<T><<<rg, rb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
    // One to four FP64 sequences on column-major A: each column's
    // instructions split over two warps a sequence, two FP64 instructions a
    // column each (stream_split_kernel, with tiles of its own width).
    constexpr bool kCanSplit = kF64 && KR <= 4;
    const bool split = kCanSplit && !packed && k == KR;
    if (kF64 && KR == 3 && !split) { st = ROT_EINVAL; break; }   // three sequences: split passes only
    int cb = SS::CB;
    if constexpr (kCanSplit) cb = split ? SplitShape<KR>::CB : SS::CB;
    CUtensorMap amap, csmap;
    // Packed: a tensor 32 elements wide with one row per (strip, column).
    const uint64_t a_inner = packed ? 32 : (uint64_t)m;
    const uint64_t a_outer = packed ? (uint64_t)((m + 31) / 32) * (uint64_t)n : (uint64_t)n;
    const uint64_t a_pitch = packed ? 32 * sizeof(T) : (uint64_t)lda * sizeof(T);
    if (!encode_tile_map_2d(&amap, A, kF64, a_inner, a_outer, a_pitch, 32 * R, (uint32_t)cb) ||
        !encode_tile_map_2d(&csmap, cs, kF64, (uint64_t)W2, (uint64_t)cs_rows, (uint64_t)W2 * sizeof(T),
                            (uint32_t)W2, (uint32_t)cb)) {
      note_error("stream: cuTensorMapEncodeTiled failed");
      st = ROT_ECUDA;
      break;
    }
    const int tr = trace_begin(kF64 ? ROT_KERNEL_WAVE_F64 : ROT_KERNEL_WAVE_F32, m * (n - 1) * k, s);
    if constexpr (kCanSplit) {
      if (split) {
        auto kfn = stream_split_kernel<KR>;
        e = smem_opt_in(reinterpret_cast<const void*>(kfn), SplitShape<KR>::kSmem);
        if (e != cudaSuccess) { st = cuda_failed(e, "stream: shared-memory opt-in"); break; }
        kfn<<<(unsigned)((m + 31) / 32), 64 * KR + 32, SplitShape<KR>::kSmem, s>>>(amap, csmap, A, lda, (int)m, (int)n,
                                                                              status);
        trace_end(tr, s);
        e = cudaGetLastError();
        if (e != cudaSuccess) { st = cuda_failed(e, "stream: kernel launch"); break; }
        record_status_async(status, s);
        count_launches(3);
        break;
      }
    }
    if constexpr (!(kF64 && KR == 3)) {
      auto kfn = stream_kernel<T, KR, R>;
      e = smem_opt_in(reinterpret_cast<const void*>(kfn), SS::kSmem);
      if (e != cudaSuccess) { st = cuda_failed(e, "stream: shared-memory opt-in"); break; }
      kfn<<<(unsigned)((m + 32 * R - 1) / (32 * R)), 32, SS::kSmem, s>>>(amap, csmap, A, packed ? 32 : lda, (int)m,
                                                                         (int)n, (int)k, status,
                                                                         packed ? (int)n : 0);
      trace_end(tr, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) { st = cuda_failed(e, "stream: kernel launch"); break; }
      record_status_async(status, s);
      count_launches(3);
    }
  } while (0);
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace

template <typename T>
bool stream_fits(int64_t m, int64_t n, int64_t k, const T* A, int64_t lda) {
  // At most 48 (FP32) or 16 (FP64) sequences; TMA needs a 16-byte aligned
  // base and column pitch, and the boxes (up to 64 rows, up to 63 columns)
  // inside the matrix.
  const int64_t kmax = sizeof(T) == 4 ? 48 : 16;
  return k >= 1 && k <= kmax && m >= 64 && n >= 64 && (reinterpret_cast<uintptr_t>(A) % 16) == 0 &&
         ((uint64_t)lda * sizeof(T)) % 16 == 0;
}

template <typename T>
rot_status stream_apply(int64_t m, int64_t n, int64_t k, T* A, int64_t lda, const T* C, int64_t ldc, const T* S,
                        int64_t lds, cudaStream_t s, bool packed) {
  // Passes of 8, 4, 2 or 1 sequences (8 while they last, then the binary
  // digits of the rest), so that every pass fills its window: a window
  // wider than its sequences runs every wave with predicates (FP32 at
  // 8192 x 8192: k = 5 in one window of 8 took 1.41 ms, as 4 + 1 it takes
  // about 0.28 ms; k = 3 in a window of 4 0.38 ms, as 2 + 1 about 0.23).
  // FP64 on column-major A takes passes of at most 4 sequences, each on
  // the split stream.
  const bool split64 = sizeof(T) == 8 && !packed;
  for (int64_t p0 = 0; p0 < k;) {
    const int64_t left = k - p0;
    const int64_t kk = split64 ? std::min<int64_t>(left, 4) : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    const T* Cp = C + p0 * ldc;
    const T* Sp = S + p0 * lds;
    rot_status st;
    if (kk == 1) st = stream_launch<T, 1>(m, n, kk, A, lda, Cp, ldc, Sp, lds, s, packed);
    else if (kk == 2) st = stream_launch<T, 2>(m, n, kk, A, lda, Cp, ldc, Sp, lds, s, packed);
    else if (kk == 3) {
      if constexpr (sizeof(T) == 8) st = stream_launch<T, 3>(m, n, kk, A, lda, Cp, ldc, Sp, lds, s, packed);
      else st = ROT_EINVAL;
    } else if (kk == 4) st = stream_launch<T, 4>(m, n, kk, A, lda, Cp, ldc, Sp, lds, s, packed);
    else st = stream_launch<T, 8>(m, n, kk, A, lda, Cp, ldc, Sp, lds, s, packed);
    if (st != ROT_OK) return st;
    p0 += kk;
  }
  return ROT_OK;
}

template bool stream_fits<double>(int64_t, int64_t, int64_t, const double*, int64_t);
template bool stream_fits<float>(int64_t, int64_t, int64_t, const float*, int64_t);
template rot_status stream_apply<double>(int64_t, int64_t, int64_t, double*, int64_t, const double*, int64_t,
                                         const double*, int64_t, cudaStream_t, bool);
template rot_status stream_apply<float>(int64_t, int64_t, int64_t, float*, int64_t, const float*, int64_t,
                                        const float*, int64_t, cudaStream_t, bool);

}  // namespace rs
