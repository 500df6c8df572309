// rs_chain.cuh -- FP32: one pass of up to KW*NW sequences as a chain of NW
// warps per 32-row strip (the column stream of rs_stream.cuh, its sequences
// dealt out to several warps).
//
// With one p-block there is no dependency between row strips, and a warp of
// the column stream owns a strip (one row per lane): 8192 rows make 256
// warps for GB300's 608 SM sub-partitions, so most of them idle and a pass
// of 8 sequences takes four times its HBM time.  Here warp w of a strip
// applies sequences w*KW .. w*KW + KW - 1 of the pass (Algorithm 2 applies
// sequence p entirely before p+1, and a column is final for sequences < p
// once sequence p-1 has rotated it with its right neighbour, so each warp
// runs the column stream's schedule on the columns its predecessor
// finished).  At global wave W (from -1 on) warp w takes in column
// W - w*KW + 1, rotates pairs (j, j+1), j = W - w*KW - l, for its l < KW,
// and passes column W - (w+1)*KW + 1 on (final for its sequences).  Every
// warp reads (c,s) row W of the same TMA stage: the repacked row of wave W
// holds sequence p's pair at position p for j = W - p.  Columns travel
// between consecutive warps through rings of RING tiles in shared memory
// (ready/free barriers); warp 0 reads A from the TMA stages, the last warp
// stores the finished columns, and a ninth, producer warp refills each
// stage once every compute warp is done with it.  Each element sees the
// column stream's operations on the same operands, in the same order:
// bit-identical.
//
// Measured at 8192 x 8192 (a clock64 timeline of one CTA's warps in a copy
// outside the product): the chain moves at the pace of its slowest warp,
// and a tile's barrier operations cost about as much as its rotations:
// each wait took about 400 cycles even on a barrier completed long before,
// and the last warp also refilled the stages.  Relaxed waits and arrivals on
// the barriers that carry no data (free, consumed) and a test before each
// suspending wait took a pass of 48 sequences from 1.79 to 1.31 ms in the
// timeline build; the refill on a producer warp, 1.25 to 1.04 ms without
// the timeline.  Issue is then about 70 % busy (about 4.5 warps per SM
// sub-partition), and the 256 strips of 8192 rows leave 104 SMs with two
// and 48 with one.
#pragma once
#include "rs_wave.cuh"

namespace rs {

template <int KW, int NW>
struct ChainShape {
  static constexpr int KR = KW * NW;                       // sequences per pass
  static constexpr int U = KW + 1;                         // window slots per warp
  static constexpr int CB = U * (16 / U);                  // columns per tile, a multiple of U
  // A warp starts a tile once its predecessor has handed the whole tile
  // over, so the last warp trails the first by a tile or more per warp; the
  // stages cover that lag and the copies' latency.  (Measured at 8192 x
  // 8192: rings of 3 to 6 tiles, or 8 to 12 more stages, changed nothing;
  // 10- or 5-column tiles were 10-40 % slower.)
  static constexpr int S = NW + 3;
  static constexpr int RING = 2;
  static constexpr int KP = KR >= 2 ? KR : 2;              // pairs per (c,s) row (rows of 16 bytes at least)
  static constexpr int kABytes = 32 * CB * (int)sizeof(float);
  static constexpr int kCsBytes = CB * 2 * KP * (int)sizeof(float);
  static constexpr int kAStage = (kABytes + 127) / 128 * 128;   // TMA destinations 128-byte aligned
  static constexpr int kStage = kAStage + (kCsBytes + 127) / 128 * 128;
  static constexpr int kRingTile = CB * 32 * (int)sizeof(float);
  static constexpr int kRingOff = S * kStage;
  static constexpr int kBarOff = kRingOff + (NW - 1) * RING * kRingTile;
  // barriers: full[S], consumed[S], ready[NW-1][RING], free[NW-1][RING]; then the abort flag
  static constexpr int kSmem = kBarOff + (2 * S + 2 * (NW - 1) * RING) * 8 + 16;
};

// Shared state of one CTA of chain_kernel.
struct ChainCta {
  const CUtensorMap* amap;
  const CUtensorMap* csmap;
  unsigned char* smem;
  uint64_t* full;
  uint64_t* consumed;
  uint64_t* ready;
  uint64_t* freed;
  volatile int* abort_flag;
  float* A;
  int64_t lda;
  int m, n, k, c, lane, ntiles;
  int* status;
};

// The KW pairs of one wave (128-bit loads where KW is even: KP and the
// warp's first sequence are then even, so the address is 16-byte aligned).
template <int KW>
__device__ __forceinline__ void chain_pairs(const float2* __restrict__ cs, float2 (&p)[KW]) {
  if constexpr (KW % 2 == 0) {
#pragma unroll
    for (int l = 0; l < KW; l += 2) {
      const float4 v = *reinterpret_cast<const float4*>(cs + l);
      p[l].x = v.x;
      p[l].y = v.y;
      p[l + 1].x = v.z;
      p[l + 1].y = v.w;
    }
  } else {
#pragma unroll
    for (int l = 0; l < KW; ++l) p[l] = cs[l];
  }
}

// One tile of warp w (first sequence wk): CB waves.  win: the last KW
// columns that entered the warp (columns wl0+1-KW .. wl0), carried from tile
// to tile; in: the tile's input columns ([slot][lane]); cs: the pairs of its
// waves, offset to the warp's first sequence; wl0: local wave (W - wk) of
// slot 0.  FULL: every rotation of the warp exists in the tile, so no
// predicates.  Every column of the tile has its own register (col[KW + i]
// enters at wave i), and the rotations run by anti-diagonals d = i + l:
// rotation (i, l) needs only (i, l-1) and (i-1, l), so the up to KW
// rotations of a diagonal are independent.  Wave i's output, column
// wl0 + 1 + i - KW (col[i]), is final after rotation (i, KW-1), on diagonal
// i + KW - 1.  The last warp stores it through ps; the others hand it on in
// out.
template <int KW, int NW, bool FULL, bool LAST>
__device__ __forceinline__ void chain_tile(float (&win)[KW], const float* __restrict__ in,
                                           const float2* __restrict__ cs, int wl0, int wk, int k, int n,
                                           float* __restrict__ out, float* ps, bool rowok, int64_t lda) {
  using CS = ChainShape<KW, NW>;
  constexpr int CB = CS::CB, KP = CS::KP;
  float col[KW + CB];
#pragma unroll
  for (int a = 0; a < KW; ++a) col[a] = win[a];
#pragma unroll
  for (int i = 0; i < CB; ++i) col[KW + i] = in[i * 32];
  float2 pw[CB][KW];
#pragma unroll
  for (int d = 0; d < CB + KW - 1; ++d) {
    if (d < CB) chain_pairs<KW>(cs + d * KP, pw[d]);
#pragma unroll
    for (int l = 0; l < KW; ++l) {
      const int i = d - l;
      if (i >= 0 && i < CB) {
        const int j = wl0 + i - l;
        if (FULL || (wk + l < k && j >= 0 && j <= n - 2))   // the same in every lane
          rotate(col[KW + i - 1 - l], col[KW + i - l], pw[i][l].x, pw[i][l].y);
      }
    }
    const int i = d - (KW - 1);                  // wave whose output is now final
    if (i >= 0) {
      if constexpr (LAST) {
        const int q = wl0 + 1 + i - KW;
        if ((FULL || (q >= 0 && q <= n - 1)) && rowok) st_cg(ps + (int64_t)i * lda, col[i]);
      } else {
        out[i * 32] = col[i];
      }
    }
  }
#pragma unroll
  for (int a = 0; a < KW; ++a) win[a] = col[CB + a];
}

// The tile loop of compute warp w (first or last of the chain fixed at
// compile time).
template <int KW, int NW, bool FIRST, bool LAST>
__device__ __forceinline__ void chain_role(const ChainCta& X, int w) {
  using CS = ChainShape<KW, NW>;
  constexpr int CB = CS::CB, S = CS::S, RING = CS::RING;
  const int lane = X.lane, n = X.n, k = X.k;
  const int wk = w * KW;
  auto ring = [&](int g, int q) {
    return reinterpret_cast<float*>(X.smem + CS::kRingOff) + ((size_t)g * RING + q) * CB * 32 + lane;
  };
  // Every lane's wait must succeed, else the warp leaves and the others
  // learn it from the abort flag.
  auto settle = [&](bool ok) {
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) {
      if (!*X.abort_flag) set_error(X.status, kDevTimeoutTma);
      *X.abort_flag = 1;
    }
    return ok;
  };
  const bool rowok = X.c * 32 + lane < X.m;
  float win[KW];                                // the last KW columns that entered
#pragma unroll
  for (int u = 0; u < KW; ++u) win[u] = 0.f;
  float* const arow = X.A + (int64_t)X.c * 32 + lane;
  for (int t = 0; t < X.ntiles; ++t) {
    const int s = t % S, q = t % RING;
    const uint32_t use = (uint32_t)(t / RING);
    if (*X.abort_flag) break;
    if (!settle(mbar_wait_data(&X.full[s], (uint32_t)(t / S) & 1u))) break;
    if (!FIRST && !settle(mbar_wait_data(&X.ready[(w - 1) * RING + q], use & 1u))) break;
    if (!LAST && t >= RING && !settle(mbar_wait_read(&X.freed[w * RING + q], (use - 1) & 1u))) break;
    const float* in = FIRST ? reinterpret_cast<const float*>(X.smem + s * CS::kStage) + lane : ring(w - 1, q);
    const float2* cs = reinterpret_cast<const float2*>(X.smem + s * CS::kStage + CS::kAStage) + wk;
    float* out = LAST ? nullptr : ring(w, q);
    const int wl0 = t * CB - 1 - wk;
    float* ps = arow + (int64_t)(wl0 + 1 - KW) * X.lda;   // the last warp's column of slot 0
    if (wk + KW <= k && wl0 - (KW - 1) >= 0 && wl0 + CB - 1 <= n - 2)
      chain_tile<KW, NW, true, LAST>(win, in, cs, wl0, wk, k, n, out, ps, rowok, X.lda);
    else
      chain_tile<KW, NW, false, LAST>(win, in, cs, wl0, wk, k, n, out, ps, rowok, X.lda);
    if constexpr (!LAST) mbar_arrive(&X.ready[w * RING + q]);   // release: the slot's columns
    if constexpr (!FIRST) mbar_arrive_relaxed(&X.freed[(w - 1) * RING + q]);
    mbar_arrive_relaxed(&X.consumed[s]);
  }
}

// The producer warp: refills stage s with tile t + S once every compute
// warp is done with tile t.
template <int KW, int NW>
__device__ __forceinline__ void chain_producer(const ChainCta& X) {
  using CS = ChainShape<KW, NW>;
  constexpr int CB = CS::CB, S = CS::S;
  int issued = X.ntiles < S ? X.ntiles : S;
  int t = 0;
  for (; t + S < X.ntiles; ++t) {
    const int s = t % S;
    bool ok = !*X.abort_flag && mbar_wait_read(&X.consumed[s], (uint32_t)(t / S) & 1u);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      if (X.lane == 0) {
        if (!*X.abort_flag) set_error(X.status, kDevTimeoutTma);
        *X.abort_flag = 1;
      }
      break;
    }
    if (X.lane == 0) {
      unsigned char* st = X.smem + s * CS::kStage;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&X.full[s], CS::kABytes + CS::kCsBytes);
      tma_load_2d(st, X.amap, &X.full[s], X.c * 32, (t + S) * CB);
      tma_load_2d(st + CS::kAStage, X.csmap, &X.full[s], 0, (t + S) * CB - 1);
    }
    ++issued;
  }
  // The last copies (all of them after a timeout) may still be in flight
  // when the compute warps leave; the CTA ends only once they have landed.
  if (X.lane == 0)
    for (int u = t; u < issued; ++u) (void)mbar_wait_bounded(&X.full[u % S], (uint32_t)(u / S) & 1u);
}

// NW compute warps and one producer warp per CTA, one CTA per 32-row strip.
template <int KW, int NW>
__global__ void __launch_bounds__(32 * (NW + 1))
chain_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap csmap, float* A,
             int64_t lda, int m, int n, int k, int* status) {
  static_assert(NW >= 2 && NW <= 8, "two to eight compute warps");
  using CS = ChainShape<KW, NW>;
  constexpr int CB = CS::CB, S = CS::S, RING = CS::RING, NR = NW - 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  ChainCta X;
  X.amap = &amap;
  X.csmap = &csmap;
  X.smem = smem;
  X.full = reinterpret_cast<uint64_t*>(smem + CS::kBarOff);
  X.consumed = X.full + S;
  X.ready = X.consumed + S;                     // ready[g * RING + q]: ring g, slot q written
  X.freed = X.ready + NR * RING;                // freed[g * RING + q]: ring g, slot q read
  X.abort_flag = reinterpret_cast<volatile int*>(X.freed + NR * RING);
  X.A = A;
  X.lda = lda;
  X.m = m;
  X.n = n;
  X.k = k;
  X.c = blockIdx.x;                             // strip of 32 rows
  X.lane = threadIdx.x & 31;
  X.ntiles = (n + CS::KR + CB - 1) / CB;        // waves -1 .. n-2+KR
  X.status = status;
  if (threadIdx.x == 0) {
    prefetch_tmap(&amap);
    prefetch_tmap(&csmap);
    for (int s = 0; s < S; ++s) {
      mbar_init(&X.full[s], 1);
      mbar_init(&X.consumed[s], 32 * NW);       // every compute warp
    }
    for (int g = 0; g < NR * RING; ++g) {
      mbar_init(&X.ready[g], 32);
      mbar_init(&X.freed[g], 32);
    }
    *X.abort_flag = 0;
    fence_mbarrier_init();
    for (int t = 0; t < S && t < X.ntiles; ++t) {
      unsigned char* st = smem + t * CS::kStage;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&X.full[t], CS::kABytes + CS::kCsBytes);
      tma_load_2d(st, &amap, &X.full[t], X.c * 32, t * CB);
      tma_load_2d(st + CS::kAStage, &csmap, &X.full[t], 0, t * CB - 1);
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  if (w == 0) chain_role<KW, NW, true, false>(X, 0);
  else if (w < NW - 1) chain_role<KW, NW, false, false>(X, w);
  else if (w == NW - 1) chain_role<KW, NW, false, true>(X, w);
  else chain_producer<KW, NW>(X);
}

}  // namespace rs
