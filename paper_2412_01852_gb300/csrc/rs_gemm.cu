// rs_gemm.cu -- the accumulated-block variant ("rs_gemm", Section 8):
// the rotations of each parallelogram block (nb waves x kb sequences,
// Section 2) are first accumulated in FP64 into an orthogonal
// (nb+kb)-square matrix Q_b, and A is then updated block after block by the
// matrix product A(:, window_b) <- A(:, window_b) * Q_b on tensor cores.
//
// Block formation: Q_b = the block's rotations applied to the identity, i.e.
// Algorithm 4 on I.  Every block is one instance of the batched wavefront
// kernel whose rotations are restricted to the block (a window of waves and a
// range of j), so forming all blocks is one persistent FP64 launch.  Rows of
// the identity start as unit vectors, which lets whole waves on zero columns
// be skipped (values are unchanged; only the sign of zeros can differ).
//
// The split modes also come with blocks formed in FP32 (rs_form_f32.cu):
// their products keep about 16 (BF16) or 22 (FP16) bits, so FP32 blocks,
// formed on the FP32 pipe at 64 times GB300's FP64 rate, lose little.
//
// Block apply: the split modes run on the 5th-generation tensor cores
// (tcgen05, TMEM accumulators; rs_gemm_tc.cu) for windows up to 320 columns.
// FP64 DMMA, and wider windows, use mma.sync: one CTA per 32-row tile of A
// walks the blocks in order.  Modes:
//   ROT_GEMM_F64_DMMA   FP64 tensor MMA (m8n8k4), FP64 accumulation;
//   ROT_GEMM_SPLIT_BF16 x = hi + lo in BF16; hi*hi + hi*lo + lo*hi in FP32;
//   ROT_GEMM_SPLIT_F16  x = hi + lo*2^-11 in FP16; hi*hi in one FP32
//                       accumulator, hi*lo + lo*hi in another, combined as
//                       acc0 + 2^-11*acc1.
#include <algorithm>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "rs_batch.h"
#include "rs_form_f32.h"
#include "rs_gemm_tc.h"

namespace rs {
namespace {

constexpr int kKMAX = 16;
constexpr int kNBT = 16;
constexpr int kWarps = 8;
constexpr int kTM = 32;        // rows of A per CTA in the apply kernel
constexpr int kKC = 32;        // k rows of Q per staged chunk (split modes)
constexpr int kKC64 = 16;      // k rows of Q per staged chunk (DMMA)
constexpr int kLMax = 512;     // largest supported nb + kb

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

struct BlockPos {
  int w0, p0;   // first wave (relative to its p-block) and first sequence
};

// Blocks in the order they are applied: p-blocks of kb sequences in order,
// within one p-block the waves 0 .. (n-2)+(kb'-1) cut into runs of nb.
std::vector<BlockPos> block_schedule(int64_t n, int64_t k, int nb, int kb) {
  std::vector<BlockPos> out;
  for (int64_t p0 = 0; p0 < k; p0 += kb) {
    const int64_t kbe = std::min<int64_t>(kb, k - p0);
    const int64_t nw = (n - 1) + (kbe - 1);
    for (int64_t w0 = 0; w0 < nw; w0 += nb) out.push_back(BlockPos{(int)w0, (int)p0});
  }
  return out;
}

// Q holds nblk blocks of Lp x Lp (column-major); each becomes the L x L
// identity padded with zeros.
__global__ void identity_kernel(double* Q, int L, int Lp, long long nblk) {
  const long long total = nblk * (long long)Lp * Lp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long within = e % ((long long)Lp * Lp);
    const int r = (int)(within % Lp), c = (int)(within / Lp);
    Q[e] = (r == c && r < L) ? 1.0 : 0.0;
  }
}

// Split Q (FP64 or FP32 blocks) into hi/lo halves of the mode's 16-bit type
// (same column-major layout).  From an FP32 block, q - hi is exact in FP32,
// so both give the halves of the same value the same way.
template <int MODE, typename TQ>
__global__ void split_kernel(const TQ* __restrict__ Q, uint16_t* __restrict__ hi,
                             uint16_t* __restrict__ lo, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const TQ q = Q[e];
    if (MODE == ROT_GEMM_SPLIT_BF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)q);
      const __nv_bfloat16 l = __float2bfloat16_rn((float)(q - (TQ)__bfloat162float(h)));
      hi[e] = __bfloat16_as_ushort(h);
      lo[e] = __bfloat16_as_ushort(l);
    } else {
      const __half h = __float2half_rn((float)q);
      const __half l = __float2half_rn((float)((q - (TQ)__half2float(h)) * (TQ)2048));
      hi[e] = __half_as_ushort(h);
      lo[e] = __half_as_ushort(l);
    }
  }
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) {
  return (uint32_t)a | ((uint32_t)b << 16);
}

template <int MODE>
__device__ __forceinline__ void split_pair(double x0, double x1, uint32_t& h, uint32_t& l) {
  if (MODE == ROT_GEMM_SPLIT_BF16) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn((float)x0), h1 = __float2bfloat16_rn((float)x1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn((float)(x0 - (double)__bfloat162float(h0)));
    const __nv_bfloat16 l1 = __float2bfloat16_rn((float)(x1 - (double)__bfloat162float(h1)));
    h = pack2(__bfloat16_as_ushort(h0), __bfloat16_as_ushort(h1));
    l = pack2(__bfloat16_as_ushort(l0), __bfloat16_as_ushort(l1));
  } else {
    const __half h0 = __float2half_rn((float)x0), h1 = __float2half_rn((float)x1);
    const __half l0 = __float2half_rn((float)((x0 - (double)__half2float(h0)) * 2048.0));
    const __half l1 = __float2half_rn((float)((x1 - (double)__half2float(h1)) * 2048.0));
    h = pack2(__half_as_ushort(h0), __half_as_ushort(h1));
    l = pack2(__half_as_ushort(l0), __half_as_ushort(l1));
  }
}

template <int MODE>
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  if (MODE == ROT_GEMM_SPLIT_BF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

__device__ __forceinline__ void dmma884(double* d, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct ApplyParams {
  double* A;
  int64_t lda;
  int m, n;
  int L;                    // nb + kb
  int Lp;                   // L rounded up to a multiple of 32 (the tiling's width)
  int nblk;
  const int* c0;            // first window column of each block (may be negative)
  const double* Q;          // nblk x Lp x Lp, column-major, zero beyond L (DMMA)
  const uint16_t* Qhi;      // split modes
  const uint16_t* Qlo;
};

// sA: the block's window of this CTA's 32 rows, FP64, column-major with a
// 33-double column pitch.  Split modes stage Q in chunks of kKC k-rows as
// [n][kKC + 8] halves (hi and lo); DMMA stages [n][kKC64 + 2] doubles.
constexpr int kApitch = kTM + 1;

template <int MODE, int NT>
__global__ void __launch_bounds__(256, 1) apply_kernel(const ApplyParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  double* sA = reinterpret_cast<double*>(smem);
  unsigned char* sQ = smem + (size_t)kLMax * kApitch * sizeof(double);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int group = lane >> 2, tig = lane & 3;
  const int rh = warp & 1;            // rows [16 rh, 16 rh + 16)
  const int cg = warp >> 1;           // cols [cg * L/4, (cg+1) * L/4)
  const int L = P.L;
  const int Lp = P.Lp;
  const int r0 = blockIdx.x * kTM;
  const int ncol0 = cg * (NT * 8);

  for (int b = 0; b < P.nblk; ++b) {
    const int c0 = P.c0[b];
    // ---- stage the window of A (columns outside [0, n) and rows >= m read as 0)
    {
      const int row = tid & 31;
      const int grow = r0 + row;
      for (int col = tid >> 5; col < Lp; col += 8) {
        const int gcol = c0 + col;
        double v = 0.0;
        if (col < L && grow < P.m && gcol >= 0 && gcol < P.n) v = P.A[(int64_t)gcol * P.lda + grow];
        sA[col * kApitch + row] = v;
      }
    }
    __syncthreads();

    if (MODE == ROT_GEMM_F64_DMMA) {
      double acc[2][NT][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[mt][t][0] = acc[mt][t][1] = 0.0;
      double* sQd = reinterpret_cast<double*>(sQ);
      constexpr int QP = kKC64 + 2;     // k pitch (doubles) per n row
      const double* Qb = P.Q + (int64_t)b * Lp * Lp;
      for (int kc = 0; kc < Lp; kc += kKC64) {
        // stage Q(kc .. kc+16, 0 .. Lp) as [n][k]
        for (int e = tid; e < Lp * (kKC64 / 2); e += 256) {
          const int nn = e / (kKC64 / 2), kk = (e % (kKC64 / 2)) * 2;
          cp_async16(&sQd[nn * QP + kk], &Qb[(int64_t)nn * Lp + kc + kk]);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int k4 = 0; k4 < kKC64; k4 += 4) {
          double a[2];
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) a[mt] = sA[(kc + k4 + tig) * kApitch + rh * 16 + mt * 8 + group];
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const double bq = sQd[(ncol0 + t * 8 + group) * QP + k4 + tig];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) dmma884(acc[mt][t], a[mt], bq);
          }
        }
        __syncthreads();
      }
      // results back into sA (this CTA's rows of the window), then to A
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int rr = rh * 16 + mt * 8 + group;
          const int cc = ncol0 + t * 8 + 2 * tig;
          sA[cc * kApitch + rr] = acc[mt][t][0];
          sA[(cc + 1) * kApitch + rr] = acc[mt][t][1];
        }
    } else {
      float acc0[NT][4], acc1[NT][4];
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc0[t][i] = acc1[t][i] = 0.f;
      uint16_t* sQh = reinterpret_cast<uint16_t*>(sQ);
      constexpr int QP = kKC + 8;       // k pitch (halves) per n row
      uint16_t* sQl = sQh + (size_t)kLMax * QP;
      const uint16_t* Qh = P.Qhi + (int64_t)b * Lp * Lp;
      const uint16_t* Ql = P.Qlo + (int64_t)b * Lp * Lp;
      for (int kc = 0; kc < Lp; kc += kKC) {
        for (int e = tid; e < Lp * (kKC / 8); e += 256) {
          const int nn = e / (kKC / 8), kk = (e % (kKC / 8)) * 8;
          cp_async16(&sQh[nn * QP + kk], &Qh[(int64_t)nn * Lp + kc + kk]);
          cp_async16(&sQl[nn * QP + kk], &Ql[(int64_t)nn * Lp + kc + kk]);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kKC; ks += 16) {
          // A fragment (16 x 16, row-major): rows rh*16 + group (+8), cols kc+ks+2tig (+1, +8, +9)
          uint32_t ah[4], al[4];
          const int ra = rh * 16 + group;
          const int ka = kc + ks + 2 * tig;
          split_pair<MODE>(sA[ka * kApitch + ra], sA[(ka + 1) * kApitch + ra], ah[0], al[0]);
          split_pair<MODE>(sA[ka * kApitch + ra + 8], sA[(ka + 1) * kApitch + ra + 8], ah[1], al[1]);
          split_pair<MODE>(sA[(ka + 8) * kApitch + ra], sA[(ka + 9) * kApitch + ra], ah[2], al[2]);
          split_pair<MODE>(sA[(ka + 8) * kApitch + ra + 8], sA[(ka + 9) * kApitch + ra + 8], ah[3], al[3]);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const int nb_ = ncol0 + t * 8 + group;
            uint32_t bh[2], bl[2];
            bh[0] = *reinterpret_cast<const uint32_t*>(&sQh[nb_ * QP + ks + 2 * tig]);
            bh[1] = *reinterpret_cast<const uint32_t*>(&sQh[nb_ * QP + ks + 8 + 2 * tig]);
            bl[0] = *reinterpret_cast<const uint32_t*>(&sQl[nb_ * QP + ks + 2 * tig]);
            bl[1] = *reinterpret_cast<const uint32_t*>(&sQl[nb_ * QP + ks + 8 + 2 * tig]);
            mma16816<MODE>(acc0[t], ah, bh);
            if (MODE == ROT_GEMM_SPLIT_BF16) {
              mma16816<MODE>(acc0[t], ah, bl);
              mma16816<MODE>(acc0[t], al, bh);
            } else {
              mma16816<MODE>(acc1[t], ah, bl);
              mma16816<MODE>(acc1[t], al, bh);
            }
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int rr = rh * 16 + group;
        const int cc = ncol0 + t * 8 + 2 * tig;
        const double s1 = (MODE == ROT_GEMM_SPLIT_F16) ? (1.0 / 2048.0) : 0.0;
        sA[cc * kApitch + rr] = (double)acc0[t][0] + s1 * (double)acc1[t][0];
        sA[(cc + 1) * kApitch + rr] = (double)acc0[t][1] + s1 * (double)acc1[t][1];
        sA[cc * kApitch + rr + 8] = (double)acc0[t][2] + s1 * (double)acc1[t][2];
        sA[(cc + 1) * kApitch + rr + 8] = (double)acc0[t][3] + s1 * (double)acc1[t][3];
      }
    }
    __syncthreads();
    // ---- write the window back (coalesced over rows)
    {
      const int row = tid & 31;
      const int grow = r0 + row;
      for (int col = tid >> 5; col < L; col += 8) {
        const int gcol = c0 + col;
        if (grow < P.m && gcol >= 0 && gcol < P.n) P.A[(int64_t)gcol * P.lda + grow] = sA[col * kApitch + row];
      }  // columns L .. Lp-1 are padding and are never stored
    }
    __syncthreads();
  }
}

// Split modes, second design: the block's window of A is converted once into
// hi/lo halves in shared memory ([row][k], pitch Lp+8 halves), Q_b arrives in
// double-buffered chunks of 16 k-rows by cp.async ([n][k], pitch 24 halves),
// and shared memory is sized for the block width so that two CTAs share an
// SM and all 32-row tiles are resident at once.  Both pitches make the
// fragment loads bank-conflict free: row g / tig t of a warp read banks
// 4g + t (A, for Lp = 320) and 12g + t (Q) modulo 32.
constexpr int kQP = 24;         // halves per n row of a staged Q chunk
constexpr int kQK = 16;         // k rows per Q chunk

template <int MODE, int NT>
__global__ void __launch_bounds__(256, 2) apply_split_kernel(const ApplyParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int Lp = P.Lp, L = P.L;
  const int AP = Lp + 8;                                   // A pitch (halves)
  uint16_t* sAh = reinterpret_cast<uint16_t*>(smem);
  uint16_t* sAl = sAh + kTM * AP;
  uint16_t* sQ = sAl + kTM * AP;                           // [2 buffers][hi, lo][Lp][kQP]
  const int qbuf = 2 * Lp * kQP;                           // halves per buffer (hi + lo)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int group = lane >> 2, tig = lane & 3;
  const int rh = warp & 1, cg = warp >> 1;
  const int r0 = blockIdx.x * kTM;
  const int ncol0 = cg * (NT * 8);
  const int nk = Lp / kQK;

  for (int b = 0; b < P.nblk; ++b) {
    const int c0 = P.c0[b];
    const uint16_t* Qh = P.Qhi + (int64_t)b * Lp * Lp;
    const uint16_t* Ql = P.Qlo + (int64_t)b * Lp * Lp;
    auto stage_q = [&](int kc, int buf) {
      uint16_t* dh = sQ + buf * qbuf;
      uint16_t* dl = dh + Lp * kQP;
      for (int e = tid; e < Lp * 2; e += 256) {            // two 16-byte pieces per n row
        const int nn = e >> 1, kk = (e & 1) * 8;
        cp_async16(&dh[nn * kQP + kk], &Qh[(int64_t)nn * Lp + kc + kk]);
        cp_async16(&dl[nn * kQP + kk], &Ql[(int64_t)nn * Lp + kc + kk]);
      }
      cp_async_commit();
    };
    stage_q(0, 0);
    // ---- the window of A, split into halves (8 loads in flight per thread)
    {
      const int row = tid & 31;
      const int grow = r0 + row;
      const bool rok = grow < P.m;
      for (int col0 = tid >> 5; col0 < Lp; col0 += 64) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int col = col0 + 8 * u;
          const int gcol = c0 + col;
          v[u] = (col < L && rok && gcol >= 0 && gcol < P.n) ? P.A[(int64_t)gcol * P.lda + grow] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int col = col0 + 8 * u;
          if (col < Lp) {
            uint32_t h, l;
            split_pair<MODE>(v[u], 0.0, h, l);
            sAh[row * AP + col] = (uint16_t)(h & 0xffffu);
            sAl[row * AP + col] = (uint16_t)(l & 0xffffu);
          }
        }
      }
    }
    float acc0[NT][4], acc1[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc0[t][i] = acc1[t][i] = 0.f;
    for (int kc = 0; kc < nk; ++kc) {
      if (kc + 1 < nk) stage_q((kc + 1) * kQK, (kc + 1) & 1);
      if (kc + 1 < nk) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      else cp_async_wait_all();
      __syncthreads();
      const uint16_t* qh = sQ + (kc & 1) * qbuf;
      const uint16_t* ql = qh + Lp * kQP;
      const int ka = kc * kQK + 2 * tig;
      const int ra = rh * 16 + group;
      uint32_t ah[4], al[4];
      ah[0] = *reinterpret_cast<const uint32_t*>(&sAh[ra * AP + ka]);
      ah[1] = *reinterpret_cast<const uint32_t*>(&sAh[(ra + 8) * AP + ka]);
      ah[2] = *reinterpret_cast<const uint32_t*>(&sAh[ra * AP + ka + 8]);
      ah[3] = *reinterpret_cast<const uint32_t*>(&sAh[(ra + 8) * AP + ka + 8]);
      al[0] = *reinterpret_cast<const uint32_t*>(&sAl[ra * AP + ka]);
      al[1] = *reinterpret_cast<const uint32_t*>(&sAl[(ra + 8) * AP + ka]);
      al[2] = *reinterpret_cast<const uint32_t*>(&sAl[ra * AP + ka + 8]);
      al[3] = *reinterpret_cast<const uint32_t*>(&sAl[(ra + 8) * AP + ka + 8]);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int nb_ = ncol0 + t * 8 + group;
        uint32_t bh[2], bl[2];
        bh[0] = *reinterpret_cast<const uint32_t*>(&qh[nb_ * kQP + 2 * tig]);
        bh[1] = *reinterpret_cast<const uint32_t*>(&qh[nb_ * kQP + 8 + 2 * tig]);
        bl[0] = *reinterpret_cast<const uint32_t*>(&ql[nb_ * kQP + 2 * tig]);
        bl[1] = *reinterpret_cast<const uint32_t*>(&ql[nb_ * kQP + 8 + 2 * tig]);
        mma16816<MODE>(acc0[t], ah, bh);
        if (MODE == ROT_GEMM_SPLIT_BF16) {
          mma16816<MODE>(acc0[t], ah, bl);
          mma16816<MODE>(acc0[t], al, bh);
        } else {
          mma16816<MODE>(acc1[t], ah, bl);
          mma16816<MODE>(acc1[t], al, bh);
        }
      }
      __syncthreads();   // the buffer read now is refilled two chunks later
    }
    // ---- results straight to A (columns past L are padding and are not stored)
    const double s1 = (MODE == ROT_GEMM_SPLIT_F16) ? (1.0 / 2048.0) : 0.0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int cc = ncol0 + t * 8 + 2 * tig;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = rh * 16 + group + (i >> 1) * 8;
        const int col = cc + (i & 1);
        const int grow = r0 + rr, gcol = c0 + col;
        if (col < L && grow < P.m && gcol >= 0 && gcol < P.n)
          P.A[(int64_t)gcol * P.lda + grow] = (double)acc0[t][i] + s1 * (double)acc1[t][i];
      }
    }
    __syncthreads();   // the next block reads columns this block just wrote
  }
}

size_t apply_split_smem_bytes(int Lp) {
  return (size_t)2 * kTM * (Lp + 8) * sizeof(uint16_t) + (size_t)2 * 2 * Lp * kQP * sizeof(uint16_t);
}

size_t apply_smem_bytes(int mode) {
  const size_t a = (size_t)kLMax * kApitch * sizeof(double);
  if (mode == ROT_GEMM_F64_DMMA) return a + (size_t)kLMax * (kKC64 + 2) * sizeof(double);
  return a + 2 * (size_t)kLMax * (kKC + 8) * sizeof(uint16_t);
}

template <int MODE, int NT>
cudaError_t launch_apply_nt(const ApplyParams& P, cudaStream_t s) {
  if constexpr (MODE != ROT_GEMM_F64_DMMA) {
    const size_t smem = apply_split_smem_bytes(P.Lp);
    cudaError_t e = cudaFuncSetAttribute(apply_split_kernel<MODE, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    apply_split_kernel<MODE, NT><<<(unsigned)ceil_div(P.m, kTM), 256, smem, s>>>(P);
    return cudaGetLastError();
  } else {
  const size_t smem = apply_smem_bytes(MODE);
  cudaError_t e = cudaFuncSetAttribute(apply_kernel<MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  apply_kernel<MODE, NT><<<(unsigned)ceil_div(P.m, kTM), 256, smem, s>>>(P);
  return cudaGetLastError();
  }
}

template <int MODE>
cudaError_t launch_apply(const ApplyParams& P, cudaStream_t s) {
  switch (P.Lp / 32) {
    case 1: return launch_apply_nt<MODE, 1>(P, s);
    case 2: return launch_apply_nt<MODE, 2>(P, s);
    case 3: return launch_apply_nt<MODE, 3>(P, s);
    case 4: return launch_apply_nt<MODE, 4>(P, s);
    case 5: return launch_apply_nt<MODE, 5>(P, s);
    case 6: return launch_apply_nt<MODE, 6>(P, s);
    case 7: return launch_apply_nt<MODE, 7>(P, s);
    case 8: return launch_apply_nt<MODE, 8>(P, s);
    case 9: return launch_apply_nt<MODE, 9>(P, s);
    case 10: return launch_apply_nt<MODE, 10>(P, s);
    case 11: return launch_apply_nt<MODE, 11>(P, s);
    case 12: return launch_apply_nt<MODE, 12>(P, s);
    case 13: return launch_apply_nt<MODE, 13>(P, s);
    case 14: return launch_apply_nt<MODE, 14>(P, s);
    case 15: return launch_apply_nt<MODE, 15>(P, s);
    case 16: return launch_apply_nt<MODE, 16>(P, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// ---- block formation: one batched wave launch over all blocks ---------------------
struct FormLayout {
  std::vector<BlockPos> blocks;
  std::vector<WaveInstance> inst;
  std::vector<WavePlan> wp;
  std::vector<WaveSegment> seg;
  size_t done_ints = 0;
  long long tickets = 0;
  long long executed_rows = 0;   // rotation-row updates the formation kernel executes
  // workspace offsets
  size_t o_cs = 0, o_tmap = 0, o_inst = 0, o_seg = 0, o_cnt = 0, cnt_bytes = 0, o_c0 = 0, total = 0;
  int64_t W2 = 0;
  int cs_rows = 0;
};

// Rotation-row updates that run_item executes for one formation instance
// (rows < m only): the same wave and rotation bounds as the kernel, including
// the waves it skips because a chain's rows are still zero there.  Per
// p-block the rotations of every wave are summed once (a prefix sum over the
// waves); each chain then takes the sum over its waves.
static long long executed_rotation_rows(const WaveInstance& I) {
  long long total = 0;
  std::vector<long long> prefix;
  for (int g = 0; g < I.G; ++g) {
    const int p0 = g * I.K;
    const int kr = std::min(I.K, I.k - p0);
    const int nw = I.n + kr - 2;
    const int wr_hi = std::min(nw, I.W_hi - p0);
    const int w_lo = std::max(0, I.W_lo - p0);
    // prefix[w] = rotations in waves [w_lo, w) of this p-block
    prefix.assign((size_t)std::max(0, wr_hi - w_lo) + 1, 0);
    for (int w = w_lo; w < wr_hi; ++w) {
      const int l_lo = std::max(0, w - I.j_hi);
      const int l_hi = std::min(kr - 1, w - I.j_lo);
      prefix[(size_t)(w - w_lo) + 1] = prefix[(size_t)(w - w_lo)] + (l_hi >= l_lo ? l_hi - l_lo + 1 : 0);
    }
    for (int c = 0; c < I.nchains; ++c) {
      const int rows = std::min(32, I.m - 32 * c);
      int lo = w_lo;
      if (I.unit_rows) lo = std::max(lo, c * 32 - p0 - 2);
      if (lo >= wr_hi) continue;
      total += (prefix[(size_t)(wr_hi - w_lo)] - prefix[(size_t)(lo - w_lo)]) * rows;
    }
  }
  return total;
}

static void form_layout(int64_t n, int64_t k, int nb, int kb, FormLayout* F) {
  F->blocks = block_schedule(n, k, nb, kb);
  const int L = nb + kb;
  const WavePlan gpl = plan_wave(1, n, k, kKMAX, kNBT, 0, 0, 8);
  F->W2 = 2 * (int64_t)gpl.kpad;
  F->cs_rows = gpl.cs_rows;
  int max_key = 0;
  for (const BlockPos& bp : F->blocks) {
    const int kbe = (int)std::min<int64_t>(kb, k - bp.p0);
    const int c0 = bp.w0 - kb + 1;
    WavePlan pl = plan_wave(L, L, kbe, kKMAX, kNBT, 0, 0, 8);
    WaveInstance I{};
    I.m = L; I.n = L; I.k = kbe; I.lda = L;
    I.K = pl.K; I.NB = pl.NB; I.delta = pl.delta; I.nchains = pl.nchains; I.G = pl.G; I.B = pl.B;
    I.cs_row0 = c0 + bp.p0;
    I.p_base = bp.p0;
    I.j_lo = std::max(0, -c0);
    I.j_hi = (int)std::min<int64_t>(L - 2, n - 2 - c0);
    I.W_lo = kb - 1;
    I.W_hi = kb - 1 + nb;
    I.unit_rows = 1;
    F->executed_rows += executed_rotation_rows(I);
    F->inst.push_back(I);
    F->wp.push_back(pl);
    max_key = std::max(max_key, (pl.B - 1) + pl.delta * (pl.G - 1));
  }
  const int ni = (int)F->inst.size();
  std::vector<size_t> done_off(ni);
  for (int t = 0; t < ni; ++t) {
    done_off[t] = F->done_ints;
    F->done_ints += (size_t)F->wp[t].nchains * F->wp[t].G;
  }
  for (int kappa = 0; kappa <= max_key; ++kappa)
    for (int t = 0; t < ni; ++t) {
      const WavePlan& pl = F->wp[t];
      int hi = kappa / pl.delta;
      if (hi > pl.G - 1) hi = pl.G - 1;
      int lo = kappa - (pl.B - 1);
      lo = lo <= 0 ? 0 : (lo + pl.delta - 1) / pl.delta;
      if (hi < lo) continue;
      F->seg.push_back(WaveSegment{F->tickets, t, kappa});
      F->tickets += (long long)(hi - lo + 1) * pl.nchains;
    }
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (size_t)round_up((int64_t)off, (int64_t)align);
    const size_t o = off;
    off += bytes;
    return o;
  };
  F->o_tmap = take(sizeof(CUtensorMap), 128);
  F->o_inst = take(sizeof(WaveInstance) * std::max(ni, 1), 256);
  F->o_seg = take(sizeof(WaveSegment) * std::max<size_t>(F->seg.size(), 1), 256);
  F->o_c0 = take(sizeof(int) * std::max(ni, 1), 256);
  F->cnt_bytes = (size_t)round_up((int64_t)(F->done_ints * sizeof(int)), 256) + 256;
  F->o_cnt = take(F->cnt_bytes, 256);
  F->o_cs = take((size_t)F->cs_rows * F->W2 * sizeof(double), 1024);
  F->total = off;
  // done pointers are set once the base address is known
  for (int t = 0; t < ni; ++t) F->inst[t].done = reinterpret_cast<int*>(done_off[t] * sizeof(int));
}

// Form every block's Q (FP64) into Q (nblk x L x L) using workspace `ws`.
// Blocks are written Lq x Lq apart with leading dimension Lq (Lq >= L; the
// padding beyond L is zero).
static rot_status form_blocks_enqueue(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S,
                                      int64_t lds, int nb, int kb, const FormLayout& F, unsigned char* ws,
                                      double* Q, int Lq, cudaStream_t s) {
  const int L = nb + kb;
  const int ni = (int)F.inst.size();
  std::vector<unsigned char> img(F.o_cs, 0);
  CUtensorMap* ht = reinterpret_cast<CUtensorMap*>(img.data() + F.o_tmap);
  double* cs = reinterpret_cast<double*>(ws + F.o_cs);
  if (!encode_tile_map_2d(ht, cs, true, (uint64_t)F.W2, (uint64_t)F.cs_rows, (uint64_t)F.W2 * sizeof(double),
                          2 * kKMAX, kNBT)) {
    note_error("form_blocks: cuTensorMapEncodeTiled failed");
    return ROT_ECUDA;
  }
  WaveInstance* hi = reinterpret_cast<WaveInstance*>(img.data() + F.o_inst);
  int* hc0 = reinterpret_cast<int*>(img.data() + F.o_c0);
  int* d_done = reinterpret_cast<int*>(ws + F.o_cnt);
  for (int t = 0; t < ni; ++t) {
    WaveInstance I = F.inst[t];
    I.A = Q + (int64_t)t * Lq * Lq;
    I.lda = Lq;
    I.done = d_done + reinterpret_cast<size_t>(F.inst[t].done) / sizeof(int);
    I.tmap = reinterpret_cast<const CUtensorMap*>(ws + F.o_tmap);
    hi[t] = I;
    hc0[t] = F.blocks[t].w0 - kb + 1;
  }
  std::memcpy(img.data() + F.o_seg, F.seg.data(), F.seg.size() * sizeof(WaveSegment));
  // The image is uploaded synchronously (it is small); the rest is queued.
  cudaError_t e = cudaMemcpyAsync(ws, img.data(), img.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks: upload");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks: synchronize");
  e = cudaMemsetAsync(ws + F.o_cnt, 0, F.cnt_bytes, s);
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks: memset");
  dim3 rb(32, 8);
  dim3 rg((unsigned)ceil_div(n - 1, 32), (unsigned)ceil_div(k, 8));
  repack_cs_kernel<double><<<rg, rb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, cs, F.W2, 0);
  identity_kernel<<<1024, 256, 0, s>>>(Q, L, Lq, (long long)ni);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks: repack/identity launch");
  BatchLaunch B;
  B.count = ni;
  B.d_inst = reinterpret_cast<WaveInstance*>(ws + F.o_inst);
  B.d_seg = reinterpret_cast<WaveSegment*>(ws + F.o_seg);
  B.launch.ticket = reinterpret_cast<unsigned long long*>(ws + F.o_cnt +
                                                          round_up((int64_t)(F.done_ints * sizeof(int)), 256));
  B.launch.status = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(B.launch.ticket) + 64);
  B.launch.total = F.tickets;
  B.nseg = (int)F.seg.size();
  B.total = F.tickets;
  B.tuning.fp64_products = 1;  // identity rows are mostly zeros: keep the products on DMUL
  rot_status st = batch_prepare(&B);
  if (st != ROT_OK) return st;
  st = batch_launch_kernel(B, s, ROT_KERNEL_FORM_BLOCKS, F.executed_rows);
  if (st != ROT_OK) return st;
  count_launches(2);
  return ROT_OK;
}

static rot_status validate_gemm(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* C,
                                int64_t ldc, const void* S, int64_t lds, int nb, int kb, bool* quick) {
  *quick = false;
  if (m < 0 || n < 0 || k < 0) return ROT_EINVAL;
  const int64_t lim = (int64_t(1) << 31) - 1;
  if (m > lim || n > lim || k > lim || n + k > lim) return ROT_EINVAL;
  if (nb < 16 || kb < 16 || nb % 16 || kb % 16 || nb + kb > kLMax) return ROT_EINVAL;
  if (lda < std::max<int64_t>(1, m)) return ROT_EINVAL;
  const int64_t nm1 = std::max<int64_t>(1, n - 1);
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) { *quick = true; return ROT_OK; }
  if (!A || !C || !S) return ROT_EINVAL;
  return ROT_OK;
}

}  // namespace rs

namespace rs {

// The modes: their product arithmetic, and whether the blocks are formed in FP32.
static bool mode_known(int mode) { return mode >= ROT_GEMM_F64_DMMA && mode <= ROT_GEMM_SPLIT_F16_Q32; }
static bool mode_q32(int mode) { return mode == ROT_GEMM_SPLIT_BF16_Q32 || mode == ROT_GEMM_SPLIT_F16_Q32; }
static int mode_split(int mode) {
  if (mode == ROT_GEMM_SPLIT_BF16_Q32) return ROT_GEMM_SPLIT_BF16;
  if (mode == ROT_GEMM_SPLIT_F16_Q32) return ROT_GEMM_SPLIT_F16;
  return mode;
}
static bool mode_ok(int mode, int kb) { return mode_known(mode) && (!mode_q32(mode) || kb <= kForm32MaxKb); }

// Workspace of one rs_gemm call: the formation layout, the blocks (FP64, or
// FP32 for the *_Q32 modes), their split copies and a status word, at fixed
// offsets from a 256-byte aligned base.
struct GemmLayout {
  FormLayout F;           // FP64 formation
  Form32Layout F32;       // FP32 formation
  bool q32 = false;
  int L = 0, Lp = 0;
  int64_t nblk = 0;
  size_t o_q = 0, o_hi = 0, o_lo = 0, o_status = 0, total = 0;
};

static void gemm_layout(int64_t n, int64_t k, int nb, int kb, rot_gemm_mode mode, GemmLayout* G) {
  G->L = nb + kb;
  G->Lp = (int)round_up(G->L, 32);
  G->q32 = mode_q32(mode);
  size_t head, q_elem;
  if (G->q32) {
    form32_layout(n, k, nb, kb, G->Lp, &G->F32);
    G->nblk = G->F32.nblk;
    head = G->F32.total;
    q_elem = sizeof(float);
  } else {
    form_layout(n, k, nb, kb, &G->F);
    G->nblk = (int64_t)G->F.blocks.size();
    head = G->F.total;
    q_elem = sizeof(double);
  }
  const size_t q_bytes = (size_t)G->nblk * G->Lp * G->Lp * q_elem;
  const size_t split_bytes = mode == ROT_GEMM_F64_DMMA ? 0 : (size_t)G->nblk * G->Lp * G->Lp * sizeof(uint16_t);
  G->o_q = round_up((int64_t)head, 1024);
  G->o_hi = round_up((int64_t)(G->o_q + q_bytes), 1024);
  G->o_lo = round_up((int64_t)(G->o_hi + split_bytes), 1024);
  G->o_status = round_up((int64_t)(G->o_lo + split_bytes), 256);
  G->total = G->o_status + 256;
}

// Form the blocks and apply them, all in the workspace at `base`.
static rot_status gemm_enqueue(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                               int64_t ldc, const double* S, int64_t lds, int nb, int kb, rot_gemm_mode mode,
                               const GemmLayout& G, unsigned char* base, cudaStream_t s) {
  const int L = G.L, Lp = G.Lp;
  const int64_t nblk = G.nblk;
  const size_t o_hi = G.o_hi, o_lo = G.o_lo, o_status = G.o_status;
  const int smode = mode_split(mode);
  double* Q = nullptr;
  float* Q32 = nullptr;
  const int* c0 = nullptr;
  rot_status st;
  if (G.q32) {
    Q32 = reinterpret_cast<float*>(base + G.o_q);
    st = form32_enqueue(n, k, C, ldc, S, lds, nb, kb, G.F32, base, Q32, s);
    c0 = reinterpret_cast<const int*>(base + G.F32.o_c0);
  } else {
    Q = reinterpret_cast<double*>(base + G.o_q);
    st = form_blocks_enqueue(n, k, C, ldc, S, lds, nb, kb, G.F, base, Q, Lp, s);
    c0 = reinterpret_cast<const int*>(base + G.F.o_c0);
  }
  if (st == ROT_OK) {
    ApplyParams P{};
    P.A = A; P.lda = lda; P.m = (int)m; P.n = (int)n; P.L = L; P.Lp = Lp; P.nblk = (int)nblk;
    P.c0 = c0;
    P.Q = Q;
    P.Qhi = reinterpret_cast<const uint16_t*>(base + o_hi);
    P.Qlo = reinterpret_cast<const uint16_t*>(base + o_lo);
    const long long qe = (long long)nblk * Lp * Lp;
    cudaError_t e = cudaSuccess;
    const int tr = trace_begin(ROT_KERNEL_GEMM_APPLY, m * (n - 1) * k, s);
    uint16_t* hi = const_cast<uint16_t*>(P.Qhi);
    uint16_t* lo = const_cast<uint16_t*>(P.Qlo);
    if (smode != ROT_GEMM_F64_DMMA && apply_tc_supported(L, Lp, nb, smode)) {
      // tcgen05: 64-row tiles, accumulator in tensor memory.
      if (G.q32) split_chunked(Q32, hi, lo, Lp, nblk, smode, s);
      else split_chunked(Q, hi, lo, Lp, nblk, smode, s);
      TcApplyParams T{};
      T.A = A; T.lda = lda; T.m = (int)m; T.n = (int)n; T.L = L; T.Lp = Lp; T.nb = nb;
      T.nblk = (int)nblk;
      T.c0 = P.c0;
      T.Qhi = P.Qhi;
      T.Qlo = P.Qlo;
      uint32_t cols = 32;
      while (cols < (uint32_t)Lp) cols <<= 1;
      T.tmem_cols = cols;
      T.status = reinterpret_cast<int*>(base + o_status);
      e = cudaMemsetAsync(T.status, 0, sizeof(int), s);
      if (e == cudaSuccess) e = launch_apply_tc(T, smode, s);
      if (e == cudaSuccess) {
        record_status_async(T.status, s);
        count_launches(1);
      }
    } else if (smode == ROT_GEMM_SPLIT_BF16) {
      if (G.q32) split_kernel<ROT_GEMM_SPLIT_BF16, float><<<1024, 256, 0, s>>>(Q32, hi, lo, qe);
      else split_kernel<ROT_GEMM_SPLIT_BF16, double><<<1024, 256, 0, s>>>(Q, hi, lo, qe);
      e = launch_apply<ROT_GEMM_SPLIT_BF16>(P, s);
    } else if (smode == ROT_GEMM_SPLIT_F16) {
      if (G.q32) split_kernel<ROT_GEMM_SPLIT_F16, float><<<1024, 256, 0, s>>>(Q32, hi, lo, qe);
      else split_kernel<ROT_GEMM_SPLIT_F16, double><<<1024, 256, 0, s>>>(Q, hi, lo, qe);
      e = launch_apply<ROT_GEMM_SPLIT_F16>(P, s);
    } else {
      e = launch_apply<ROT_GEMM_F64_DMMA>(P, s);
    }
    trace_end(tr, s);
    count_launches(mode == ROT_GEMM_F64_DMMA ? 1 : 2);
    if (e != cudaSuccess) st = cuda_failed(e, "rot_apply_gemm: apply kernel");
  }
  return st;
}

}  // namespace rs

extern "C" {

int64_t rot_form_blocks_count(int64_t n, int64_t k, int nb, int kb) {
  if (n < 2 || k < 1 || nb < 1 || kb < 1) return 0;
  return (int64_t)rs::block_schedule(n, k, nb, kb).size();
}

rot_status rot_form_blocks(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S, int64_t lds,
                           int nb, int kb, double* Q, void* stream) {
  bool quick;
  const void* dummy = reinterpret_cast<const void*>(0x100);
  rot_status v = rs::validate_gemm(1, n, k, dummy, 1, C, ldc, S, lds, nb, kb, &quick);
  if (v != ROT_OK || quick) return v;
  if (!Q) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rs::FormLayout F;
  rs::form_layout(n, k, nb, kb, &F);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, F.total, s) != cudaSuccess) { cudaGetLastError(); return ROT_ENOMEM; }
  rot_status st = rs::form_blocks_enqueue(n, k, C, ldc, S, lds, nb, kb, F, static_cast<unsigned char*>(ws), Q,
                                          nb + kb, s);
  cudaFreeAsync(ws, s);
  return st;
}

rot_status rot_form_blocks_f32(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S, int64_t lds,
                               int nb, int kb, float* Q, void* stream) {
  bool quick;
  const void* dummy = reinterpret_cast<const void*>(0x100);
  rot_status v = rs::validate_gemm(1, n, k, dummy, 1, C, ldc, S, lds, nb, kb, &quick);
  if (v != ROT_OK || quick) return v;
  if (!Q || kb > rs::kForm32MaxKb || (reinterpret_cast<uintptr_t>(Q) & 15u)) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rs::Form32Layout F;
  rs::form32_layout(n, k, nb, kb, nb + kb, &F);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, F.total, s) != cudaSuccess) { cudaGetLastError(); return ROT_ENOMEM; }
  rot_status st = rs::form32_enqueue(n, k, C, ldc, S, lds, nb, kb, F, static_cast<unsigned char*>(ws), Q, s);
  cudaFreeAsync(ws, s);
  return st;
}

rot_status rot_apply_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int nb, int kb, rot_gemm_mode mode,
                                         size_t* bytes) {
  if (!bytes) return ROT_EINVAL;
  *bytes = 0;
  bool quick;
  const void* dummy = reinterpret_cast<const void*>(0x100);
  rot_status v = rs::validate_gemm(m, n, k, dummy, std::max<int64_t>(1, m), dummy, std::max<int64_t>(1, n - 1),
                                   dummy, std::max<int64_t>(1, n - 1), nb, kb, &quick);
  if (v != ROT_OK || quick) return v;
  if (!rs::mode_ok(mode, kb)) return ROT_EINVAL;
  rs::GemmLayout G;
  rs::gemm_layout(n, k, nb, kb, mode, &G);
  *bytes = G.total;
  return ROT_OK;
}

rot_status rot_apply_gemm_ws(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                             int64_t ldc, const double* S, int64_t lds, int nb, int kb, rot_gemm_mode mode,
                             void* workspace, size_t workspace_bytes, void* stream) {
  bool quick;
  rot_status v = rs::validate_gemm(m, n, k, A, lda, C, ldc, S, lds, nb, kb, &quick);
  if (v != ROT_OK || quick) return v;
  if (!rs::mode_ok(mode, kb)) return ROT_EINVAL;
  rs::GemmLayout G;
  rs::gemm_layout(n, k, nb, kb, mode, &G);
  if (!workspace || workspace_bytes < G.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return ROT_EINVAL;
  return rs::gemm_enqueue(m, n, k, A, lda, C, ldc, S, lds, nb, kb, mode, G, static_cast<unsigned char*>(workspace),
                          static_cast<cudaStream_t>(stream));
}

rot_status rot_apply_gemm(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                          int64_t ldc, const double* S, int64_t lds, int nb, int kb, rot_gemm_mode mode,
                          void* stream) {
  bool quick;
  rot_status v = rs::validate_gemm(m, n, k, A, lda, C, ldc, S, lds, nb, kb, &quick);
  if (v != ROT_OK || quick) return v;
  if (!rs::mode_ok(mode, kb)) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rs::GemmLayout G;
  rs::gemm_layout(n, k, nb, kb, mode, &G);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, G.total, s) != cudaSuccess) { cudaGetLastError(); return ROT_ENOMEM; }
  rot_status st = rs::gemm_enqueue(m, n, k, A, lda, C, ldc, S, lds, nb, kb, mode, G, static_cast<unsigned char*>(ws), s);
  cudaFreeAsync(ws, s);
  return st;
}

}  // extern "C"
