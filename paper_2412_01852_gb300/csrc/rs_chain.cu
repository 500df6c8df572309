// rs_chain.cu -- host side of the FP32 warp-chain column stream
// (rs_chain.cuh).  rot_apply_f32 takes it for 16 <= k <= 55 sequences on a
// TMA-addressable A (but not k = 8j + 7 with at most 4096 rows): one pass
// of 8*floor(k/8) (16, 24, 32, 40 or 48) sequences on eight chained warps
// per 32-row strip, the other k mod 8 on the column stream (rs_stream.cu)
// after it.  Algorithm 2 applies sequence p
// entirely before p+1, so the passes compute the same thing.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_chain.cuh"
#include "rs_internal.h"

namespace rs {
namespace {

inline int64_t round_up256(int64_t x) { return (x + 255) / 256 * 256; }

constexpr int kChainWarps = 8;

// One pass of KW*8 sequences (exactly: the kernel's interior tiles assume
// every warp's sequences exist).
template <int KW>
rot_status chain_launch(int64_t m, int64_t n, float* A, int64_t lda, const float* C, int64_t ldc, const float* S,
                        int64_t lds, cudaStream_t s) {
  using CS = ChainShape<KW, kChainWarps>;
  const int64_t k = CS::KR;
  const int64_t W2 = 2 * CS::KP;                   // elements per (c,s) row
  const int64_t cs_rows = n + CS::KR;              // row j + p <= n + k - 3, plus the TMA's reach
  const int64_t cs_bytes = cs_rows * W2 * (int64_t)sizeof(float);
  const int64_t st_off = round_up256(cs_bytes);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, (size_t)(st_off + 256), s) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  float* cs = reinterpret_cast<float*>(base);
  int* status = reinterpret_cast<int*>(base + st_off);
  rot_status st = ROT_OK;
  do {
    // Pairs the repack does not write are only read by rotations that do not exist.
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) { st = cuda_failed(e, "chain: memset"); break; }
    dim3 rb(32, 8);
    dim3 rg((unsigned)((n - 1 + 31) / 32), (unsigned)((k + 7) / 8));
    repack_cs_kernel<float><<<rg, rb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
    CUtensorMap amap, csmap;
    if (!encode_tile_map_2d(&amap, A, false, (uint64_t)m, (uint64_t)n, (uint64_t)lda * sizeof(float), 32,
                            CS::CB) ||
        !encode_tile_map_2d(&csmap, cs, false, (uint64_t)W2, (uint64_t)cs_rows, (uint64_t)W2 * sizeof(float),
                            (uint32_t)W2, CS::CB)) {
      note_error("chain: cuTensorMapEncodeTiled failed");
      st = ROT_ECUDA;
      break;
    }
    auto kfn = chain_kernel<KW, kChainWarps>;
    e = smem_opt_in(reinterpret_cast<const void*>(kfn), CS::kSmem);
    if (e != cudaSuccess) { st = cuda_failed(e, "chain: shared-memory opt-in"); break; }
    const int tr = trace_begin(ROT_KERNEL_WAVE_F32, m * (n - 1) * k, s);
    kfn<<<(unsigned)((m + 31) / 32), 32 * (kChainWarps + 1), CS::kSmem, s>>>(amap, csmap, A, lda, (int)m, (int)n,
                                                                             (int)k, status);
    trace_end(tr, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_failed(e, "chain: kernel launch"); break; }
    record_status_async(status, s);
    count_launches(3);
  } while (0);
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace

bool chain_f32_fits(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda) {
  // With at most 4096 rows a remainder of 7 (three stream passes: 4, 2, 1)
  // costs more than the lane pipeline saves (2048 x 2048, k = 31: 0.37 ms
  // against 0.32; 4096 x 4096: 0.56 against 0.52).
  if (m <= 4096 && k % 8 == 7) return false;
  return k >= 16 && k <= 55 && stream_fits<float>(m, n, 1, A, lda) && m < (int64_t(1) << 31) &&
         n < (int64_t(1) << 30);
}

rot_status chain_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C, int64_t ldc,
                           const float* S, int64_t lds, cudaStream_t s) {
  const int64_t kr = std::min<int64_t>(k / 8 * 8, 48);
  rot_status st;
  switch (kr) {
    case 16: st = chain_launch<2>(m, n, A, lda, C, ldc, S, lds, s); break;
    case 24: st = chain_launch<3>(m, n, A, lda, C, ldc, S, lds, s); break;
    case 32: st = chain_launch<4>(m, n, A, lda, C, ldc, S, lds, s); break;
    case 40: st = chain_launch<5>(m, n, A, lda, C, ldc, S, lds, s); break;
    case 48: st = chain_launch<6>(m, n, A, lda, C, ldc, S, lds, s); break;
    default: return ROT_EINVAL;
  }
  if (st != ROT_OK || kr == k) return st;
  return stream_apply<float>(m, n, k - kr, A, lda, C + kr * ldc, ldc, S + kr * lds, lds, s);
}

}  // namespace rs
