// rs_form_f32.h -- accumulated blocks of rs_gemm (Section 8) formed in FP32
// (rs_form_f32.cu), for the split tensor-core modes whose products carry
// less precision than FP32.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_internal.h"

namespace rs {

// Largest kb the FP32 formation takes (sequences are spread over the 32
// lanes, at most 4 per lane).
constexpr int kForm32MaxKb = 128;

// Block b of the apply order (p-blocks of kb sequences in order, within one
// of them runs of nb waves): its first window column c0 = w0 - kb + 1, its
// first sequence p0 and its sequence count kbe.  Every p-block but the last
// has ceil((n + kb - 2) / nb) blocks, the last one no more.
__host__ __device__ inline void block_at(int64_t b, int64_t n, int64_t k, int nb, int kb, int* c0, int* p0,
                                         int* kbe) {
  const int64_t B0 = (n + kb - 2 + nb - 1) / nb;
  const int64_t G = (k + kb - 1) / kb;
  int64_t g = b / B0;
  if (g > G - 1) g = G - 1;
  *p0 = (int)(g * kb);
  *kbe = (int)((k - g * kb) < kb ? (k - g * kb) : kb);
  *c0 = (int)((b - g * B0) * nb) - kb + 1;
}

struct Form32Layout {
  int64_t nblk = 0;
  int L = 0, Lq = 0;      // block size and the size it is stored at (Lq >= L, zero padded)
  int spl = 0, KS = 0;    // sequences per lane, lanes * spl
  int NT = 0;             // pipeline steps: Lq + 2 KS - 1
  size_t o_c0 = 0, o_tab = 0, total = 0;   // workspace: c0 per block, the (c,s) step table
};

// Layout of an FP32 formation of every block for (n, k, nb, kb), stored
// Lq x Lq apart.  kb <= kForm32MaxKb.
void form32_layout(int64_t n, int64_t k, int nb, int kb, int Lq, Form32Layout* F);

// Queue the formation into Q (nblk blocks of Lq x Lq FP32, column-major, the
// padding zero) using the workspace at `ws` (F.total bytes, 256-byte
// aligned); the workspace's c0 array (F.o_c0) then holds each block's first
// window column.  Two launches, no host synchronisation.
rot_status form32_enqueue(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S, int64_t lds,
                          int nb, int kb, const Form32Layout& F, unsigned char* ws, float* Q, cudaStream_t s);

}  // namespace rs
