// rs_gemm_tc.h -- the tcgen05 (TMEM-accumulator) block apply of the
// accumulated-block variant, split BF16 and split FP16 (rs_gemm_tc.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

struct TcApplyParams {
  double* A;
  int64_t lda;
  int m, n;
  int L;                  // nb + kb: window width
  int Lp;                 // L rounded up to a multiple of 32 (Q's padded size)
  int nb;                 // columns a window advances within a p-block
  int nblk;
  const int* c0;          // first window column of each block, in apply order
  const uint16_t* Qhi;    // nblk x Lp x Lp BF16 in the staging order of split_chunked
  const uint16_t* Qlo;
  uint32_t tmem_cols;     // power of two >= Lp (the accumulator's columns)
  int* status;            // first device error (timeouts), 0 if none
};

// Whether the tensor-core apply supports this block shape.
bool apply_tc_supported(int L, int Lp, int nb, int mode);
size_t apply_tc_smem_bytes(int Lp, int kb);
// mode: ROT_GEMM_SPLIT_BF16 or ROT_GEMM_SPLIT_F16.
cudaError_t launch_apply_tc(const TcApplyParams& P, int mode, cudaStream_t s);

// Split Q (nblk blocks of Lp x Lp FP64, column-major) into the BF16 hi/lo
// operands of launch_apply_tc, in its staging order.
void split_chunked(const double* Q, uint16_t* hi, uint16_t* lo, int Lp, long long nblk, int mode, cudaStream_t s);
// The same from FP32 blocks.
void split_chunked(const float* Q, uint16_t* hi, uint16_t* lo, int Lp, long long nblk, int mode, cudaStream_t s);

}  // namespace rs
