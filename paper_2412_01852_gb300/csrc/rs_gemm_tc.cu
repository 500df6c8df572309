// rs_gemm_tc.cu -- the block apply of the accumulated-block variant (rs_gemm,
// Section 8) on the 5th-generation tensor cores: tcgen05.mma with operands in
// shared memory and the FP32 accumulator in tensor memory (TMEM).
//
// Split BF16: every FP64 entry x is written as hi + lo with hi = bf16(x) and
// lo = bf16(x - hi), and A_win * Q_b is formed as
//     A_hi*Q_hi + A_hi*Q_lo + A_lo*Q_hi
// in one FP32 accumulator (the lo*lo term, ~2^-16 relative, is dropped).
//
// One CTA owns a tile of 128 rows of A and walks the blocks in their order.
// Per block:
//   * the window (128 rows x Lp columns) sits in shared memory as hi and lo
//     BF16 operands in the K-major no-swizzle layout of 8x16-byte core
//     matrices;
//   * Q_b hi/lo (prepared in global memory, column n holding k contiguous) is
//     streamed in chunks of 16 k-rows through two buffers (cp.async);
//   * one thread issues, per chunk, the three products for the two halves of
//     N (N = Lp/2 each, at most 256) and commits them to the chunk buffer's
//     mbarrier, which releases the buffer;
//   * the epilogue reads the accumulator (tcgen05.ld, each warp its 32-lane
//     sub-partition), stores the block's finished columns to A in FP64 and,
//     when the next block continues the same p-block, keeps the kb columns
//     the two windows share in shared memory as the next window's first
//     columns (split again from FP32), so only nb new columns are read.
// Every wait is bounded; on a timeout the CTA records an error, stops, waits
// for its own copies and frees its tensor memory.
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "rs_device.cuh"
#include "rs_gemm_tc.h"

namespace rs {
namespace {

constexpr int kRows = 128;          // rows of A per CTA (the MMA's M)
constexpr int kThreads = 512;
constexpr int kKChunk = 16;         // k per MMA instruction (BF16)
constexpr uint32_t kCoreBytes = 128;  // one core matrix: 8 rows x 16 bytes

// ---- descriptors -------------------------------------------------------------
// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension
// byte offset (between core matrices adjacent in K) and stride-dimension byte
// offset (between core matrices adjacent in M or N), all in 16-byte units;
// descriptor version 1 at bits 46-47; no swizzle (bits 61-63 zero).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5
// = 1), A and B BF16 (bits 7-9 and 10-12 = 1), both K-major, N/8 at bits
// 17-22, M/16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- tcgen05 wrappers ----------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(smem_u32(slot)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}
// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3); v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- splitting ------------------------------------------------------------------
__device__ __forceinline__ void split_f64(double x, uint16_t& h, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn((float)x);
  const __nv_bfloat16 lb = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hb)));
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(lb);
}
__device__ __forceinline__ void split_f32(float x, uint16_t& h, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(x);
  const __nv_bfloat16 lb = __float2bfloat16_rn(x - __bfloat162float(hb));  // exact difference
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(lb);
}
__device__ __forceinline__ uint4 pack8(const uint16_t (&e)[8]) {
  uint4 u;
  u.x = (uint32_t)e[0] | ((uint32_t)e[1] << 16);
  u.y = (uint32_t)e[2] | ((uint32_t)e[3] << 16);
  u.z = (uint32_t)e[4] | ((uint32_t)e[5] << 16);
  u.w = (uint32_t)e[6] | ((uint32_t)e[7] << 16);
  return u;
}

struct Smem {
  // byte offsets from the dynamic shared-memory base
  uint32_t w_hi, w_lo, q, bar, slot, flag, total;
  uint32_t q_part;   // bytes of one staged operand (hi or lo) of one buffer: Lp x 16 k
};

__host__ __device__ inline Smem smem_plan(int Lp) {
  Smem s{};
  const uint32_t w = (uint32_t)kRows * Lp * 2;     // one BF16 operand of the window
  s.w_hi = 0;
  s.w_lo = w;
  s.q = 2 * w;
  s.q_part = (uint32_t)Lp * kKChunk * 2;
  s.bar = s.q + 4 * s.q_part;                       // 2 buffers x (hi, lo)
  s.slot = s.bar + 2 * 8;
  s.flag = s.slot + 4;
  s.total = s.flag + 4 + 16;
  return s;
}

// Write 8 consecutive window columns [k8*8, k8*8+8) of `row` (already split).
__device__ __forceinline__ void put_window8(unsigned char* smem, const Smem& L, int row, int k8, const uint4& hi,
                                            const uint4& lo) {
  const uint32_t off = (uint32_t)k8 * (kRows * 16) + (uint32_t)row * 16;
  *reinterpret_cast<uint4*>(smem + L.w_hi + off) = hi;
  *reinterpret_cast<uint4*>(smem + L.w_lo + off) = lo;
}

// Load window columns [g_lo*8, g_hi*8) of the block starting at global column
// c0 from A (FP64), split, into the window operands.  Columns outside [0, n)
// and rows outside [0, m) are zero; so are columns at or past L.
__device__ void load_window(unsigned char* smem, const Smem& L, const TcApplyParams& P, int r0, int c0, int g_lo,
                            int g_hi) {
  const int tid = threadIdx.x;
  const int row = tid % kRows;
  const int grow = r0 + row;
  const bool rok = grow < P.m;
  const double* arow = P.A + grow;
  for (int g = g_lo + tid / kRows; g < g_hi; g += kThreads / kRows) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int col = g * 8 + u;
      const int gc = c0 + col;
      v[u] = (rok && col < P.L && gc >= 0 && gc < P.n) ? __ldcg(arow + (int64_t)gc * P.lda) : 0.0;
    }
    uint16_t h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_f64(v[u], h[u], l[u]);
    put_window8(smem, L, row, g, pack8(h), pack8(l));
  }
}

__global__ void __launch_bounds__(kThreads, 1) apply_tc_kernel(const TcApplyParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int Lp = P.Lp, L = P.L;
  const Smem S = smem_plan(Lp);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S.bar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + S.slot);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + S.flag);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * kRows;
  const uint32_t ncols = P.tmem_cols;
  const int nk = Lp / kKChunk;
  const int nhalf = Lp / 2;
  const uint32_t idesc = idesc_bf16_f32(kRows, nhalf);
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) tmem_alloc(slot, ncols);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbarrier_init();
    *abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  uint32_t commits[2] = {0, 0}, waits[2] = {0, 0};
  bool fresh = true;   // the window must be loaded whole (first block of a p-block)
  for (int b = 0; b < P.nblk; ++b) {
    const int c0 = P.c0[b];
    if (fresh) load_window(smem, S, P, r0, c0, 0, Lp / 8);
    const bool contig = b + 1 < P.nblk && P.c0[b + 1] == c0 + P.nb;
    fence_async_smem();
    __syncthreads();

    // ---- the block's products, chunk by chunk ----------------------------------
    const uint16_t* Qh = P.Qhi + (int64_t)b * Lp * Lp;
    const uint16_t* Ql = P.Qlo + (int64_t)b * Lp * Lp;
    auto stage = [&](int kc, int buf) {
      // 16 k-rows of every column n of Q: two 16-byte pieces (k 0-7, 8-15) per n.
      const uint32_t dst = sbase + S.q + (uint32_t)buf * 2 * S.q_part;
      for (int e = tid; e < 2 * Lp; e += kThreads) {
        const int nn = e >> 1, half = e & 1;
        const uint32_t off = (uint32_t)half * (uint32_t)Lp * 16 + (uint32_t)nn * 16;
        const int64_t src = (int64_t)nn * Lp + kc * kKChunk + half * 8;
        cp_async16(dst + off, Qh + src);
        cp_async16(dst + S.q_part + off, Ql + src);
      }
      cp_async_commit();
    };
    stage(0, 0);
    for (int kc = 0; kc < nk; ++kc) {
      const int buf = kc & 1;
      if (kc + 1 < nk) {
        const int nbuf = buf ^ 1;
        if (commits[nbuf] > waits[nbuf]) {       // the MMAs of chunk kc-1 still read it
          if (!mbar_wait_bounded(&bar[nbuf], waits[nbuf] & 1)) {
            set_error(P.status, kDevTimeoutTma);
            *abort_flag = 1;
          }
          ++waits[nbuf];
        }
        stage(kc + 1, nbuf);
        cp_async_wait_1();
      } else {
        cp_async_wait_0();
      }
      fence_async_smem();
      __syncthreads();
      if (*abort_flag) break;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t q0 = sbase + S.q + (uint32_t)buf * 2 * S.q_part;
        const uint32_t a_off = (uint32_t)kc * 2 * (kRows * 16);
        const uint64_t ah = smem_desc(sbase + S.w_hi + a_off, kRows * 16, kCoreBytes);
        const uint64_t al = smem_desc(sbase + S.w_lo + a_off, kRows * 16, kCoreBytes);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t noff = (uint32_t)h * nhalf * 16;
          const uint64_t bh = smem_desc(q0 + noff, (uint32_t)Lp * 16, kCoreBytes);
          const uint64_t bl = smem_desc(q0 + S.q_part + noff, (uint32_t)Lp * 16, kCoreBytes);
          const uint32_t d = tmem + (uint32_t)(h * nhalf);
          tc_mma(d, ah, bh, idesc, kc > 0 ? 1u : 0u);
          tc_mma(d, ah, bl, idesc, 1u);
          tc_mma(d, al, bh, idesc, 1u);
        }
        tc_commit(&bar[buf]);
      }
      ++commits[buf];
    }
    // ---- wait for every MMA of the block -----------------------------------------
    for (int i = 0; i < 2; ++i) {
      while (commits[i] > waits[i]) {
        if (!mbar_wait_bounded(&bar[i], waits[i] & 1)) {
          set_error(P.status, kDevTimeoutTma);
          *abort_flag = 1;
        }
        ++waits[i];
      }
    }
    __syncthreads();
    if (*abort_flag) break;
    tc_fence_after();

    // ---- epilogue: finished columns to A, shared columns to the next window ------
    {
      const int q = warp & 3;                  // TMEM sub-partition = rows 32q .. 32q+31
      const int row = 32 * q + lane;
      const int grow = r0 + row;
      const bool rok = grow < P.m;
      const int per = Lp / 4;                  // columns per warp of the sub-partition
      const int cbeg = (warp >> 2) * per;
      const int keep = contig ? P.nb : L;      // columns at or past `keep` carry over
      for (int j0 = cbeg; j0 < cbeg + per; j0 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)j0, v);
        if (j0 >= L) continue;                 // padding columns
        if (j0 >= keep) {
          uint16_t h[8], l[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) split_f32(v[u], h[u], l[u]);
          put_window8(smem, S, row, (j0 - P.nb) / 8, pack8(h), pack8(l));
        } else if (rok) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int col = j0 + u;
            const int gc = c0 + col;
            if (col < keep && gc >= 0 && gc < P.n) __stcg(P.A + (int64_t)gc * P.lda + grow, (double)v[u]);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // the shared columns are in place; TMEM may be overwritten
    if (contig) {
      // The next window's columns [kb, L) are new: read them from A.
      load_window(smem, S, P, r0, P.c0[b + 1], (L - P.nb) / 8, L / 8);
    }
    fresh = !contig;
  }
  cp_async_wait_0();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

size_t apply_tc_smem_bytes(int Lp) { return smem_plan(Lp).total; }

bool apply_tc_supported(int L, int Lp, int nb) {
  // N = Lp/2 per MMA (a multiple of 16, at most 256); the window, two staged
  // chunks and the barriers fit in shared memory; nb and L - nb are whole
  // 8-column groups (the carried columns move in 16-byte pieces).
  return Lp % 32 == 0 && Lp <= 512 && nb % 8 == 0 && L % 8 == 0 && apply_tc_smem_bytes(Lp) <= 227 * 1024;
}

cudaError_t launch_apply_tc(const TcApplyParams& P, cudaStream_t s) {
  const size_t smem = apply_tc_smem_bytes(P.Lp);
  cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((P.m + kRows - 1) / kRows);
  apply_tc_kernel<<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace rs
