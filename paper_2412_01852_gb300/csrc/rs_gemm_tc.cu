// rs_gemm_tc.cu -- the block apply of the accumulated-block variant (rs_gemm,
// Section 8) on the 5th-generation tensor cores: tcgen05.mma with operands in
// shared memory and the FP32 accumulator in tensor memory (TMEM).
//
// Split BF16: every FP64 entry x is written as hi + lo with hi = bf16(x) and
// lo = bf16(x - hi), and A_win * Q_b is formed as
//     A_hi*Q_hi + A_hi*Q_lo + A_lo*Q_hi
// in one FP32 accumulator (the lo*lo term, ~2^-16 relative, is dropped).
// Split FP16: x = hi + 2^-11 lo with lo = fp16((x - hi) * 2^11) kept in
// FP16's normal range; hi*hi and hi*lo + lo*hi go to two accumulators,
// combined as acc0 + 2^-11 acc1.  Both accumulators of all Lp columns do not
// fit in TMEM, so each block runs as two passes of Lp/2 output columns.
//
// One CTA owns a tile of 64 rows of A (M = 64) and walks the blocks in their
// order with three roles:
//   * a TMA producer thread streams Q_b hi/lo (prepared in global memory,
//     column n holding k contiguous) in chunks of 16 k-rows through four
//     stages (full/empty mbarriers); the stream is latency-bound, so the
//     stage count matters (measured at L = 320: with three stages the apply
//     takes 8 % longer, with two a third longer);
//   * an MMA thread issues, per chunk, the three products for the two halves
//     of N (N = Lp/2 each, at most 256) into two TMEM accumulators and
//     commits each chunk to its stage's empty barrier;
//   * 16 worker warps keep the windows: the kb columns a block shares with
//     the previous one in buffer C, its nb new columns in one of two buffers
//     N0, N1.  While block b's products run they read the nb new columns of
//     block b+1 from A (FP64), split them and write them into the other N
//     buffer; when the accumulator is complete they read it (tcgen05.ld, each
//     warp its TMEM sub-partition), store block b's finished columns to A in
//     FP64 and write the kb columns that blocks b and b+1 share, split again
//     from FP32, into C (block b's products, C's readers, are done by then).
//     The first window of a p-block is read whole, after the previous
//     block's columns are stored.
// The window operands sit in shared memory in the K-major no-swizzle layout
// of 8-row x 16-byte core matrices.  Every wait is bounded; on a timeout the
// CTA records an error, every role stops, the producer waits for its copies
// and the tensor memory is freed.
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rs_device.cuh"
#include "rs_gemm_tc.h"
#include "rs_internal.h"

namespace rs {
namespace {

constexpr int kRows = 64;           // rows of A per CTA (the MMA's M)
constexpr int kWorkers = 16;        // warps that load windows and run the epilogue
constexpr int kThreads = (2 + kWorkers) * 32;   // + the TMA producer and MMA issuer warps
constexpr int kStages = 4;          // Q chunks in flight
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
// = 1), A and B BF16 (bits 7-9 and 10-12 = 1) or FP16 (0), both K-major, N/8
// at bits 17-22, M/16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f32acc(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
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

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- splitting ------------------------------------------------------------------
// FP64 <-> FP32 by integer bit operations.  GB300's FP64 pipe (2 lanes per
// clock per SM) would otherwise be this kernel's bottleneck: a conversion
// instruction there costs as much as a DFMA.
// FP64 -> FP32 rounding toward zero (relative error below 2^-23, far below the
// split's 2^-17): rebias the exponent in the high word, then one funnel shift
// moves exponent and mantissa into place.  Magnitudes below FP32's normal
// range become zero; above it Inf; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t ax = hi & 0x7fffffffu;
  const int32_t t = (int32_t)(ax - (896u << 20));          // exponent - (1023 - 127)
  uint32_t f = __funnelshift_l(lo, (uint32_t)t, 3);
  if (t <= 0) f = 0u;
  if (t >= (int32_t)(255u << 20)) f = (ax > 0x7ff00000u || (ax == 0x7ff00000u && lo)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(f | (hi & 0x80000000u));
}
// FP32 -> FP64, exact for zeros, normal numbers, Inf and NaN (FP32 subnormals
// become signed zero).
__device__ __forceinline__ double f32_to_f64(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t au = u & 0x7fffffffu;
  uint32_t dhi = (au >> 3) + (896u << 20), dlo = u << 29;
  if (au < 0x00800000u) dhi = dlo = 0u;
  if (au >= 0x7f800000u) dhi = 0x7ff00000u | (au >> 3);
  return __hiloint2double((int)(dhi | (u & 0x80000000u)), (int)dlo);
}
// Two FP32 values -> their hi parts and lo parts, each pair packed low-first.
//   BF16:  x = hi + lo + r,           |r| <= 2^-17 |x|
//   FP16:  x = hi + 2^-11 lo + r,     lo = RN16((x - hi) * 2^11), |r| <= 2^-22 |x|
//          (lo is kept scaled so that it stays in FP16's normal range).
template <int MODE>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  if constexpr (MODE == ROT_GEMM_SPLIT_BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xffff0000u);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - ha, b - hb);   // exact differences
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn((a - hf.x) * 2048.f, (b - hf.y) * 2048.f);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// Shared-memory plan (byte offsets from the dynamic base, Lp = padded width,
// kb = L - nb carried columns, a multiple of 16):
//   C         window columns [0, kb), hi then lo, 64 rows each
//   N[2]      window columns [kb, Lp), two buffers, each hi then lo
//             In each, 8-column group g of the part sits at g*1024, element
//             (m, k%8) of the group at m*16 + (k%8)*2 (K-major core matrices).
//   Q[4]      chunk stages, each hi then lo, each two k-groups of Lp rows x
//             16 bytes: element (n, k) at (k/8)*16*Lp + n*16 + (k%8)*2
//   barriers  see Bar
struct Smem {
  uint32_t c, c_part, n, n_buf, n_part, q, q_stage, q_part, bar, slot, flag, total;
};
__host__ __device__ inline Smem smem_plan(int Lp, int kb) {
  Smem s{};
  s.c = 0;
  s.c_part = (uint32_t)kRows * kb * 2;
  s.n = 2 * s.c_part;
  s.n_part = (uint32_t)kRows * (Lp - kb) * 2;
  s.n_buf = 2 * s.n_part;
  s.q_part = (uint32_t)Lp * kKChunk * 2;
  s.q_stage = 2 * s.q_part;
  s.q = s.n + 2 * s.n_buf;
  s.bar = s.q + kStages * s.q_stage;
  s.slot = s.bar + 16 * 8;
  s.flag = s.slot + 4;
  s.total = s.flag + 4 + 8;
  return s;
}
// Offset of 8-column group g (hi part) of the window in N buffer `buf`
// (groups below gc = kb/8 are in C), and the distance from hi to lo there.
__device__ __forceinline__ uint32_t win_group(const Smem& S, int buf, int g, int gc) {
  return g < gc ? S.c + (uint32_t)g * (kRows * 16) : S.n + (uint32_t)buf * S.n_buf + (uint32_t)(g - gc) * (kRows * 16);
}
__device__ __forceinline__ uint32_t win_lo(const Smem& S, int g, int gc) { return g < gc ? S.c_part : S.n_part; }

enum Bar {
  kQFull = 0,
  kQEmpty = kQFull + kStages,
  kWReady = kQEmpty + kStages,
  kWFree = kWReady + 2,
  kDFull = kWFree + 2,
  kDEmpty = kDFull + 1,
  kStored = kDEmpty + 1,
  kNumBars = kStored + 1
};
static_assert(kNumBars <= 16, "barrier area");

// A wait that gives up after the limit or once another role has given up.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity)) return true;
  set_error(status, kDevTimeoutTma);
  *abort_flag = 1;
  return false;
}

// Window columns [g_lo*8, g_hi*8) of the block whose window starts at global
// column c0: FP64 from A, split, into C and N buffer `wbuf`.  Columns outside [0, n),
// at or past L, and rows outside [0, m) are zero.  `wt` is the worker thread;
// each handles one row and up to kGroupsInFlight 8-column groups at a time,
// all of whose loads are issued before the first is used.
constexpr int kGroupsInFlight = 4;
template <int MODE>
__device__ void load_window(unsigned char* smem, const Smem& S, const TcApplyParams& P, int wbuf, int wt, int r0,
                            int c0, int g_lo, int g_hi) {
  const int row = wt % kRows;
  const int grow = r0 + row;
  const bool rok = grow < P.m;
  const double* arow = P.A + (rok ? grow : 0);
  const int gc = (P.L - P.nb) / 8;
  constexpr int kStep = kWorkers * 32 / kRows;   // threads per row
  for (int g0 = g_lo + wt / kRows; g0 < g_hi; g0 += kGroupsInFlight * kStep) {
    double v[kGroupsInFlight][8];
#pragma unroll
    for (int t = 0; t < kGroupsInFlight; ++t) {
      const int g = g0 + t * kStep;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = g * 8 + u;
        const int gc = c0 + col;
        v[t][u] = (g < g_hi && rok && col < P.L && gc >= 0 && gc < P.n) ? __ldcg(arow + (int64_t)gc * P.lda) : 0.0;
      }
    }
#pragma unroll
    for (int t = 0; t < kGroupsInFlight; ++t) {
      const int g = g0 + t * kStep;
      if (g >= g_hi) break;
      uint4 h, l;
      split_pair<MODE>(f64_to_f32_rz(v[t][0]), f64_to_f32_rz(v[t][1]), h.x, l.x);
      split_pair<MODE>(f64_to_f32_rz(v[t][2]), f64_to_f32_rz(v[t][3]), h.y, l.y);
      split_pair<MODE>(f64_to_f32_rz(v[t][4]), f64_to_f32_rz(v[t][5]), h.z, l.z);
      split_pair<MODE>(f64_to_f32_rz(v[t][6]), f64_to_f32_rz(v[t][7]), h.w, l.w);
      const uint32_t off = win_group(S, wbuf, g, gc) + (uint32_t)row * 16;
      *reinterpret_cast<uint4*>(smem + off) = h;
      *reinterpret_cast<uint4*>(smem + off + win_lo(S, g, gc)) = l;
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
apply_tc_kernel(const TcApplyParams P) {
  // Split BF16: one pass per block over all Lp output columns (both halves
  // of N per chunk), one accumulator.  Split FP16: one pass per half of the
  // columns, each with two accumulators (hi*hi and the scaled cross terms).
  constexpr bool kBF16 = MODE == ROT_GEMM_SPLIT_BF16;
  constexpr int kPasses = kBF16 ? 1 : 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int Lp = P.Lp, L = P.L;
  const int kb = L - P.nb;                  // carried columns
  const int gc = kb / 8, kcar = kb / kKChunk;
  // Q_b(k, n) is exactly zero for n < k - kb: each of the block's kb
  // sequences moves a row's first nonzero at most one column left.  So the
  // first half of the output columns (n < nhalf) gets nothing from chunks
  // kc >= kz, whose products are skipped (FP16: those chunks of its first
  // pass are not even fetched).
  const int kz = min(Lp / kKChunk, (Lp / 2 + kb + kKChunk - 1) / kKChunk);
  const Smem S = smem_plan(Lp, kb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S.bar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + S.slot);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + S.flag);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * kRows;
  const uint32_t ncols = P.tmem_cols;
  const int nk = Lp / kKChunk;
  const int nhalf = Lp / 2;
  const uint32_t sbase = smem_u32(smem);
  // bytes of one staged operand (hi or lo) of one chunk
  const uint32_t part_bytes = kBF16 ? S.q_part : S.q_part / 2;

  if (warp == 0) tmem_alloc(slot, ncols);
  if (tid == 32) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&bar[kQFull + i], 1);
      mbar_init(&bar[kQEmpty + i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar[kWReady + i], kWorkers * 32);
      mbar_init(&bar[kWFree + i], 1);
    }
    mbar_init(&bar[kDFull], 1);
    mbar_init(&bar[kDEmpty], kWorkers * 32);
    mbar_init(&bar[kStored], kWorkers * 32);
    fence_mbarrier_init();
    *abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  // The producer and MMA threads each issue one long stream of asynchronous
  // operations from a single thread; that thread's own arithmetic between two
  // issues does not overlap the tensor pipe, so both loops keep it minimal:
  // stages and parities advance by counters, copy sources by pointer
  // increments, and descriptors (whose start address is the low field, in
  // 16-byte units) by adding offsets to ones built once.
  if (warp == 0) {
    // ---- producer: Q chunks by bulk copy, four stages ahead --------------------------
    if (lane == 0) {
      const int64_t step = part_bytes / 2;   // elements of one operand of one chunk
      uint32_t cnt = 0, st = 0, ph = 0;      // ph: parity of the current round over the stages
      unsigned char* dst = smem + S.q;
      bool ok = true;
      for (int t = 0; t < P.nblk * kPasses && ok; ++t) {
        // FP16's first pass (t even) stops at chunk kz; everything else runs all nk
        const int nkt = (!kBF16 && (t & 1) == 0) ? kz : nk;
        const uint16_t* srch = P.Qhi + (int64_t)t * nk * step;
        const uint16_t* srcl = P.Qlo + (int64_t)t * nk * step;
        for (int kc = 0; kc < nkt; ++kc, ++cnt) {
          if (cnt >= (uint32_t)kStages && !mbar_try_wait(&bar[kQEmpty + st], ph ^ 1) &&
              !wait_phase(&bar[kQEmpty + st], ph ^ 1, abort_flag, P.status)) {
            ok = false;
            break;
          }
          // The chunk is stored in global memory in exactly its shared-memory
          // layout: one bulk copy each for hi and lo.
          mbar_arrive_expect_tx(&bar[kQFull + st], 2 * part_bytes);
          bulk_g2s(dst, srch, part_bytes, &bar[kQFull + st]);
          bulk_g2s(dst + S.q_part, srcl, part_bytes, &bar[kQFull + st]);
          srch += step;
          srcl += step;
          dst += S.q_stage;
          if (++st == (uint32_t)kStages) {
            st = 0;
            ph ^= 1;
            dst = smem + S.q;
          }
        }
      }
      // Leave no copy in flight: the last fill of each stage has landed.
      for (uint32_t s2 = 0; s2 < (uint32_t)kStages && s2 < cnt; ++s2) {
        const uint32_t fills = (cnt - s2 + kStages - 1) / kStages;   // fills of stage s2
        (void)mbar_wait_bounded(&bar[kQFull + s2], (fills - 1) & 1);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ------------------------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f32acc(kBF16, kRows, nhalf);
      // Window operand: C hi and N0 hi, chunk 0; Q operand of stage 0, hi, column 0.
      const uint64_t dc = smem_desc(sbase + S.c, kRows * 16, kCoreBytes);
      const uint64_t dn0 = smem_desc(sbase + S.n, kRows * 16, kCoreBytes);
      const uint64_t dq0 = smem_desc(sbase + S.q, kBF16 ? (uint32_t)Lp * 16 : (uint32_t)nhalf * 16, kCoreBytes);
      const uint64_t c_part16 = S.c_part >> 4, n_part16 = S.n_part >> 4, n_buf16 = S.n_buf >> 4;
      const uint64_t q_part16 = S.q_part >> 4, q_stage16 = S.q_stage >> 4;
      const uint64_t chunk16 = (2 * kRows * 16) >> 4;   // one chunk of the window: two k-groups
      const uint64_t half16 = (uint64_t)nhalf;          // nhalf columns of 16 bytes
      uint32_t st = 0, ph = 0;
      uint64_t dq = dq0;
      bool ok = true;
      for (int b = 0; b < P.nblk && ok; ++b) {
        const int wb = b & 1;
        if (!wait_phase(&bar[kWReady + wb], (b >> 1) & 1, abort_flag, P.status)) break;
        for (int h = 0; h < kPasses && ok; ++h) {
          const int t = b * kPasses + h;
          if (t >= 1 && !wait_phase(&bar[kDEmpty], (t - 1) & 1, abort_flag, P.status)) { ok = false; break; }
          tc_fence_after();
          uint64_t ah = dc, al = dc + c_part16;
          const int nkt = (!kBF16 && h == 0) ? kz : nk;
          for (int kc = 0; kc < nkt; ++kc) {
            if (kc == kcar) {                  // past the carried columns: the N buffer
              ah = dn0 + (uint64_t)wb * n_buf16;
              al = ah + n_part16;
            }
            if (!mbar_try_wait(&bar[kQFull + st], ph) && !wait_phase(&bar[kQFull + st], ph, abort_flag, P.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t acc = kc > 0 ? 1u : 0u;
            if constexpr (kBF16) {
              // both halves of N: hi*hi + hi*lo + lo*hi into each
              if (kc < kz) {
                tc_mma(tmem, ah, dq, idesc, acc);
                tc_mma(tmem, ah, dq + q_part16, idesc, 1u);
                tc_mma(tmem, al, dq, idesc, 1u);
              }
              tc_mma(tmem + (uint32_t)nhalf, ah, dq + half16, idesc, acc);
              tc_mma(tmem + (uint32_t)nhalf, ah, dq + q_part16 + half16, idesc, 1u);
              tc_mma(tmem + (uint32_t)nhalf, al, dq + half16, idesc, 1u);
            } else {
              // this half's columns: hi*hi into acc0, hi*lo + lo*hi into acc1
              tc_mma(tmem, ah, dq, idesc, acc);
              tc_mma(tmem + (uint32_t)nhalf, ah, dq + q_part16, idesc, acc);
              tc_mma(tmem + (uint32_t)nhalf, al, dq, idesc, 1u);
            }
            tc_commit(&bar[kQEmpty + st]);
            ah += chunk16;
            al += chunk16;
            dq += q_stage16;
            if (++st == (uint32_t)kStages) {
              st = 0;
              ph ^= 1;
              dq = dq0;
            }
          }
          if (!ok) break;
          tc_commit(&bar[kDFull]);
        }
        if (!ok) break;
        tc_commit(&bar[kWFree + wb]);
      }
    }
  } else {
    // ---- workers: window loads and the epilogue ------------------------------------------
    const int wt = tid - 64;
    const int sp = warp & 3;                   // TMEM sub-partition this warp may read
    const int cq = (warp - 2) >> 2;            // which quarter of the columns
    const int per = Lp / 4;
    // M = 64: accumulator row r sits in TMEM lane (r/16)*32 + r%16.
    load_window<MODE>(smem, S, P, 0, wt, r0, P.c0[0], 0, Lp / 8);
    // Columns [L, Lp) of the second buffer are only ever padding; a window
    // continued from the previous block never writes them, so zero them once
    // (Q's padding rows are zero, but 0 * NaN is not).
    for (int e = wt; e < (Lp - L) / 8 * kRows; e += kWorkers * 32) {
      const uint32_t off = win_group(S, 1, L / 8 + e / kRows, gc) + (uint32_t)(e % kRows) * 16;
      *reinterpret_cast<uint4*>(smem + off) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(smem + off + S.n_part) = make_uint4(0, 0, 0, 0);
    }
    fence_async_smem();
    mbar_arrive(&bar[kWReady + 0]);
    uint32_t fresh_loads = 0;
    for (int b = 0; b < P.nblk; ++b) {
      const int c0 = P.c0[b];
      const bool has_next = b + 1 < P.nblk;
      const bool contig = has_next && P.c0[b + 1] == c0 + P.nb;
      const int ib = (b + 1) & 1;
      if (contig) {
        // The next window's new columns [kb, L), into the other buffer once
        // the MMAs of block b-1 (its previous user) are done.
        if (b >= 1 && !wait_phase(&bar[kWFree + ib], ((b - 1) >> 1) & 1, abort_flag, P.status)) break;
        load_window<MODE>(smem, S, P, ib, wt, r0, P.c0[b + 1], (L - P.nb) / 8, L / 8);
      }
      const int keep = contig ? P.nb : L;      // columns at or past `keep` carry over
      // Lanes 0-15 of the warp hold rows 16sp .. 16sp+15 (M = 64); each
      // 8-column piece is shared with lanes 16-31, which take its upper half.
      const int half = lane >> 4;
      const int prow = 16 * sp + (lane & 15);
      const bool pvalid = r0 + prow < P.m;
      bool ok = true;
      for (int h = 0; h < kPasses; ++h) {
        const int t = b * kPasses + h;
        if (!wait_phase(&bar[kDFull], t & 1, abort_flag, P.status)) { ok = false; break; }
        tc_fence_after();
        // BF16: this warp's quarter of all Lp columns.  FP16: its share of
        // the half's nhalf columns, 8 at a time.
        const int jbeg = kBF16 ? cq * per : h * nhalf + cq * 8;
        const int jend = kBF16 ? (cq + 1) * per : (h + 1) * nhalf;
        const int jstep = kBF16 ? 8 : 32;
        for (int j0 = jbeg; j0 < jend; j0 += jstep) {
          float v[8];
          __syncwarp();
          const uint32_t tl = tmem + ((uint32_t)(32 * sp) << 16);
          if constexpr (kBF16) {
            tmem_ld8(tl + (uint32_t)j0, v);
          } else {
            float x[8];
            tmem_ld8(tl + (uint32_t)(j0 - h * nhalf), v);
            tmem_ld8(tl + (uint32_t)(nhalf + j0 - h * nhalf), x);
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = fmaf(x[u], 1.0f / 2048.0f, v[u]);
          }
          float w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] = __shfl_sync(0xffffffffu, v[4 + u], lane & 15);
          if (half) {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = w[u];
          }
          if (j0 >= L) continue;                 // padding columns
          const int jc = j0 + 4 * half;          // this lane's first column
          if (j0 >= keep) {
            uint2 hh, ll;
            split_pair<MODE>(v[0], v[1], hh.x, ll.x);
            split_pair<MODE>(v[2], v[3], hh.y, ll.y);
            // into C: this block's products, C's last readers, are complete
            const uint32_t off = S.c + (uint32_t)((j0 - P.nb) / 8) * (kRows * 16) + (uint32_t)prow * 16 + 8 * half;
            *reinterpret_cast<uint2*>(smem + off) = hh;
            *reinterpret_cast<uint2*>(smem + off + S.c_part) = ll;
          } else if (pvalid) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int gc = c0 + jc + u;
              if (gc >= 0 && gc < P.n) __stcg(P.A + (int64_t)gc * P.lda + r0 + prow, f32_to_f64(v[u]));
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&bar[kDEmpty]);
      }
      if (!ok) break;
      if (has_next && !contig) {
        // A new p-block: its first window overlaps columns just stored, so
        // every worker's stores come first.
        __threadfence_block();
        mbar_arrive(&bar[kStored]);
        if (!wait_phase(&bar[kStored], fresh_loads & 1, abort_flag, P.status)) break;
        ++fresh_loads;
        load_window<MODE>(smem, S, P, ib, wt, r0, P.c0[b + 1], 0, Lp / 8);
      }
      if (has_next) {
        fence_async_smem();
        mbar_arrive(&bar[kWReady + ib]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Issue-rate probe: one thread issues `mmas` products of one shape from zeroed
// shared-memory operands, cycling over `nacc` independent accumulators, and
// times first issue to last completion.
constexpr uint32_t kProbeSmem = 120 * 1024;   // more than half an SM: one CTA per SM
__global__ void __launch_bounds__(128, 1)
tc_issue_probe_kernel(int M, int N, int nacc, int mmas, unsigned long long* ns, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 16384);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 16384 + 8);
  const int tid = threadIdx.x;
  // A (M x 16) at 0 and B (N x 16) at 8192, K-major core matrices, all zero.
  for (int i = tid; i < 16384 / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 32) tmem_alloc(slot, 512);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbarrier_init();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    const uint32_t sb = smem_u32(smem);
    const uint64_t a = smem_desc(sb, (uint32_t)M * 16, kCoreBytes);
    const uint64_t b = smem_desc(sb + 8192, (uint32_t)N * 16, kCoreBytes);
    const uint32_t idesc = idesc_f32acc(true, M, N);
    const unsigned long long t0 = globaltimer_ns();
    int q = 0;
    for (int i = 0; i < mmas; ++i) {
      tc_mma(tmem + (uint32_t)(q * N), a, b, idesc, i >= nacc ? 1u : 0u);
      if (++q == nacc) q = 0;
    }
    tc_commit(bar);
    const bool ok = mbar_wait_bounded(bar, 0);
    ns[blockIdx.x] = ok ? globaltimer_ns() - t0 : 0ull;
    if (!ok) set_error(status, kDevTimeoutTma);
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

size_t apply_tc_smem_bytes(int Lp, int kb) { return smem_plan(Lp, kb).total; }

bool apply_tc_supported(int L, int Lp, int nb, int mode) {
  // N = Lp/2 per MMA (a multiple of 16, at most 256; one TMA box of Lp/2 rows);
  // two windows, three chunk stages and the barriers fit in shared memory; nb
  // and L - nb are whole 8-column groups (the carried columns move in 16-byte
  // pieces).
  // The carried columns are whole chunks of 16 (C is read by whole chunks)
  // and, in FP16's two passes, all in the second pass (C is rewritten in its
  // epilogue, after both passes' products).
  return Lp % 32 == 0 && Lp <= 512 && nb % 8 == 0 && L % 8 == 0 && nb < L && L <= Lp && (L - nb) % 16 == 0 &&
         (mode == ROT_GEMM_SPLIT_BF16 || nb >= Lp / 2) && apply_tc_smem_bytes(Lp, L - nb) <= 227 * 1024;
}

template <int MODE>
static cudaError_t launch_mode(const TcApplyParams& P, cudaStream_t s) {
  const size_t smem = apply_tc_smem_bytes(P.Lp, P.L - P.nb);
  cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((P.m + kRows - 1) / kRows);
  apply_tc_kernel<MODE><<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_apply_tc(const TcApplyParams& P, int mode, cudaStream_t s) {
  if (mode == ROT_GEMM_SPLIT_BF16) return launch_mode<ROT_GEMM_SPLIT_BF16>(P, s);
  if (mode == ROT_GEMM_SPLIT_F16) return launch_mode<ROT_GEMM_SPLIT_F16>(P, s);
  return cudaErrorInvalidValue;
}

// Q (nblk blocks of Lp x Lp FP64, column n holding k contiguous) split into
// hi/lo, written in the order the apply kernel stages it.
//   BF16: for block b, chunk kc of 16 k, k-group kg of 8 k and column n, the
//         8 values k = 16kc+8kg .. +7 form one 16-byte piece at
//         (((b*nk + kc)*2 + kg)*Lp + n)*8;  x = hi + lo.
//   FP16: the same per half h of the columns (N = Lp/2 of them): the piece of
//         column n of the half is at ((((2b + h)*nk + kc)*2 + kg)*N + n)*8;
//         x = hi + 2^-11 lo.
template <typename TQ>
__global__ void split_chunked_kernel(const TQ* __restrict__ Q, uint16_t* __restrict__ hi,
                                     uint16_t* __restrict__ lo, int Lp, int mode, long long total) {
  const int nk = Lp / kKChunk;
  const int W = mode == ROT_GEMM_SPLIT_BF16 ? Lp : Lp / 2;     // columns per staged chunk
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(e & 7);
    const long long r = e >> 3;
    const int n = (int)(r % W);
    const long long r2 = r / W;
    const int kg = (int)(r2 & 1);
    const long long r3 = r2 >> 1;
    const int kc = (int)(r3 % nk);
    const long long t = r3 / nk;
    long long b;
    int col;
    if (mode == ROT_GEMM_SPLIT_BF16) {
      b = t;
      col = n;
    } else {
      b = t >> 1;
      col = (int)(t & 1) * W + n;
    }
    const TQ q = Q[(b * Lp + col) * Lp + kc * kKChunk + kg * 8 + kk];
    if (mode == ROT_GEMM_SPLIT_BF16) {
      // From an FP32 block, q - hi is exact in FP32: the same halves as the
      // FP64 route gives for the same value.
      const __nv_bfloat16 hb = __float2bfloat16_rn((float)q);
      const __nv_bfloat16 lb = __float2bfloat16_rn((float)(q - (TQ)__bfloat162float(hb)));
      hi[e] = __bfloat16_as_ushort(hb);
      lo[e] = __bfloat16_as_ushort(lb);
    } else {
      const __half h = __float2half_rn((float)q);
      const __half l = __float2half_rn((float)((q - (TQ)__half2float(h)) * (TQ)2048));
      hi[e] = __half_as_ushort(h);
      lo[e] = __half_as_ushort(l);
    }
  }
}

void split_chunked(const double* Q, uint16_t* hi, uint16_t* lo, int Lp, long long nblk, int mode, cudaStream_t s) {
  split_chunked_kernel<double><<<1024, 256, 0, s>>>(Q, hi, lo, Lp, mode, nblk * Lp * Lp);
}

void split_chunked(const float* Q, uint16_t* hi, uint16_t* lo, int Lp, long long nblk, int mode, cudaStream_t s) {
  split_chunked_kernel<float><<<1024, 256, 0, s>>>(Q, hi, lo, Lp, mode, nblk * Lp * Lp);
}

}  // namespace rs

extern "C" rot_status rot_measure_tc_issue(int m, int n, int accumulators, int mmas, double* ns_per_mma) {
  if (!ns_per_mma || (m != 64 && m != 128) || n < 16 || n > 256 || n % 16 != 0 || accumulators < 1 ||
      accumulators * n > 512 || mmas < 1 || mmas > (1 << 20))
    return ROT_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROT_ECUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long* d_ns = nullptr;
  if (cudaMalloc(&d_ns, sizeof(unsigned long long) * nsm + sizeof(int)) != cudaSuccess) return ROT_ENOMEM;
  int* d_status = reinterpret_cast<int*>(d_ns + nsm);
  rot_status st = ROT_OK;
  cudaError_t e = cudaFuncSetAttribute(rs::tc_issue_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)rs::kProbeSmem);
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
  for (int r = 0; r < 2 && e == cudaSuccess; ++r) {   // the first launch warms up
    rs::tc_issue_probe_kernel<<<nsm, 128, rs::kProbeSmem>>>(m, n, accumulators, mmas, d_ns, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<unsigned long long> h(nsm);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), d_ns, sizeof(unsigned long long) * nsm, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = rs::cuda_failed(e, "rot_measure_tc_issue");
  else if (status != 0) st = ROT_ETIMEOUT;
  cudaFree(d_ns);
  rs::count_launches(2);
  if (st != ROT_OK) return st;
  double sum = 0;
  for (int i = 0; i < nsm; ++i) sum += (double)h[i];
  *ns_per_mma = sum / nsm / mmas;
  return ROT_OK;
}
