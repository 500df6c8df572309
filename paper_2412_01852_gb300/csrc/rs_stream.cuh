// rs_stream.cuh -- the wavefront of a single p-block (k <= 8 sequences) as a
// column stream.
//
// With one p-block there is no dependency between row strips, and the only
// parallelism Algorithm 2 leaves is across rows (each row's rotations form
// one sequential chain, Section 1).  At small k a wave carries little
// arithmetic, so the kernel's time is the latency of bringing each column in.
// Each warp owns 32R rows (R per lane) and streams all columns through a
// ring of S stages in shared memory; each stage is filled by two TMA copies:
// CB columns of its rows, and the (c,s) pairs of the CB waves that take those
// columns in.  S*CB columns are in flight per warp, enough to hide the memory
// latency behind the rotations.  With one warp per SMSP or fewer, a wave's
// dependent FP chain is what a warp waits on; R = 2 gives it two independent
// chains per wave (and one (c,s) load and store address for two rows).
//
// Column q lives in window slot q % U (U = KR + 1).  Wave w (from -1, when
// column 0 enters, on) takes in column w + 1 and applies rotations
// l = 0..k-1 to columns (j, j+1), j = w - l, in increasing l, where
// 0 <= j <= n-2 (Algorithm 3's order, the same operations per element as
// Algorithm 2); column w + 1 - KR is then final and is stored.  Tiles hold a
// multiple of U columns, so every slot index is a compile-time constant.
#pragma once
#include "rs_wave.cuh"

namespace rs {

template <typename T, int KR, int R>
struct StreamShape {
  static constexpr int U = KR + 1;                      // window slots
  // Columns per tile, a multiple of U.  A tile costs about 0.2 us on top of
  // its waves (barrier, copies), so FP32 with small windows takes long tiles;
  // a window of 8 keeps the unrolled tile within the instruction cache, and
  // FP64 keeps its ring small enough for two CTAs per SM.
  static constexpr int kTarget = (sizeof(T) == 4 && KR <= 4) ? 60 : 20;
  static constexpr int CB = U * ((kTarget + U - 1) / U);
  static constexpr int S = 8;                           // tiles in flight
  // (c,s) rows are padded to 16 bytes (a TMA box's inner extent).
  static constexpr int KP = (int)(2 * KR * sizeof(T)) >= 16 ? KR : (int)(16 / (2 * sizeof(T)));
  static constexpr int kABytes = 32 * R * CB * (int)sizeof(T);
  static constexpr int kCsBytes = CB * 2 * KP * (int)sizeof(T);
  static constexpr int kAStage = (kABytes + 127) / 128 * 128;    // TMA destinations 128-byte aligned
  static constexpr int kCsStage = (kCsBytes + 127) / 128 * 128;
  static constexpr int kStage = kAStage + kCsStage;
  static constexpr int kSmem = S * kStage + S * 8;
};

// Rows per lane of the launch.  One (more warps: with a few warps per SM,
// each warp's issue rate bounds the stream).
template <typename T, int KR>
constexpr int stream_rows() { return 1; }

// One tile: CB waves.  FULL: every rotation of every wave exists (k == KR and
// the tile lies inside the triangle-free part), so no predicates.
template <typename T, int KR, int R, bool FULL>
__device__ __forceinline__ void stream_tile(T (&win)[R][KR + 1], const T* at, const typename Pair<T>::type* cs,
                                            int w0, int k, int n, const bool (&rowok)[R], T* arow, int64_t lda,
                                            int lane) {
  using SS = StreamShape<T, KR, R>;
  using V2 = typename Pair<T>::type;
  constexpr int U = SS::U, CB = SS::CB, KP = SS::KP;
  // Stores of the interior go through a pointer advanced one column per wave.
  T* ps = arow + (int64_t)(w0 + 1 - KR) * lda;
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int w = w0 + i;
#pragma unroll
    for (int r = 0; r < R; ++r) win[r][i % U] = at[(i * R + r) * 32 + lane];   // column w + 1
#pragma unroll
    for (int l = 0; l < KR; ++l) {
      const int j = w - l;
      if (FULL || (l < k && j >= 0 && j <= n - 2)) {   // the same in every lane
        const V2 p = cs[i * KP + l];
#pragma unroll
        for (int r = 0; r < R; ++r)
          rotate_dmul(win[r][((i - 1 - l) % U + U) % U], win[r][((i - l) % U + U) % U], p.x, p.y);
      }
    }
    const int q = w + 1 - KR;                    // final: its last rotation was at wave q + k - 1
    if (FULL || (q >= 0 && q <= n - 1)) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (rowok[r]) st_cg(ps + 32 * r, win[r][(i + 1) % U]);
    }
    ps += lda;
  }
}

template <typename T, int KR, int R>
__global__ void __launch_bounds__(32)
stream_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap csmap, T* A,
              int64_t lda, int m, int n, int k, int* status, int packed_n) {
  // packed_n != 0: A is in the packed layout (32-row strips, each a 32 x n
  // column-major panel, one after the other; lda = 32, R = 1) and amap views
  // it as a 32-wide tensor of strips * n rows.
  using SS = StreamShape<T, KR, R>;
  using V2 = typename Pair<T>::type;
  constexpr int U = SS::U, CB = SS::CB, S = SS::S;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * SS::kStage);
  const int lane = threadIdx.x;
  const int c = blockIdx.x;                     // strip of 32R rows
  bool rowok[R];
#pragma unroll
  for (int r = 0; r < R; ++r) rowok[r] = c * 32 * R + r * 32 + lane < m;
  // Row of slot r: arow + 32r (only dereferenced where rowok[r]).
  T* const arow = A + (packed_n ? (int64_t)c * 32 * packed_n : (int64_t)c * 32 * R) + lane;
  // Waves -1 .. n-2+KR: after the last one, column n-1 has been stored.
  const int ntiles = (n + KR + CB - 1) / CB;
  if (lane == 0) {
    prefetch_tmap(&amap);
    prefetch_tmap(&csmap);
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbarrier_init();
  }
  __syncwarp();
  // Tile t: columns [t*CB, (t+1)*CB) of the strip, and the (c,s) rows of
  // waves t*CB - 1 .. t*CB + CB - 2 (row -1 reads as zeros).
  auto issue = [&](int t) {
    const int s = t % S;
    unsigned char* st = smem + s * SS::kStage;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[s], SS::kABytes + SS::kCsBytes);
    if (packed_n) tma_load_2d(st, &amap, &bar[s], 0, c * packed_n + t * CB);
    else tma_load_2d(st, &amap, &bar[s], c * 32 * R, t * CB);
    tma_load_2d(st + SS::kAStage, &csmap, &bar[s], 0, t * CB - 1);
  };
  if (lane == 0)
    for (int t = 0; t < S && t < ntiles; ++t) issue(t);

  T win[R][U];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int u = 0; u < U; ++u) win[r][u] = T(0);
  int t = 0;
  for (; t < ntiles; ++t) {
    const int s = t % S;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(t / S) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) set_error(status, kDevTimeoutTma);
      break;
    }
    const T* at = reinterpret_cast<const T*>(smem + s * SS::kStage);             // [column i][row r][lane]
    const V2* cs = reinterpret_cast<const V2*>(smem + s * SS::kStage + SS::kAStage);  // [wave i][pair l]
    const int w0 = t * CB - 1;
    // Interior: every wave's rotations j = w-l, l < KR, lie in [0, n-2].
    if (k == KR && w0 - (KR - 1) >= 0 && w0 + CB - 1 <= n - 2)
      stream_tile<T, KR, R, true>(win, at, cs, w0, k, n, rowok, arow, lda, lane);
    else
      stream_tile<T, KR, R, false>(win, at, cs, w0, k, n, rowok, arow, lda, lane);
    __syncwarp();                                // every lane has read the stage
    if (lane == 0 && t + S < ntiles) issue(t + S);
  }
  // On a timeout, let the copies still in flight land before leaving.
  if (t < ntiles && lane == 0) {
    for (int r = t + 1; r < ntiles && r < t + S; ++r) (void)mbar_wait_bounded(&bar[r % S], (uint32_t)(r / S) & 1u);
  }
}

// ---------------------------------------------------------------------------
// FP64, one or two sequences: the column stream split over two warps.
//
// GB300's FP64 unit belongs to an SM sub-partition and takes 64 cycles for a
// warp instruction, whatever its active lanes.  A row's chain of rotations is
// sequential, so one warp streaming its 32 rows alone costs 4 instructions x
// 64 cycles per column at k = 1 (8 at k = 2) however many warps run beside
// it.  Two warps of one CTA, on different sub-partitions, share each column's
// instructions; the arithmetic is rotate_dmul's, every element sees the same
// operations on the same operands, so the result is bit-identical.
//   k = 1: warp A carries the chain, x <- fma(c, y, -RN(s*x)) (2
//          instructions a column), and hands each column's incoming x to
//          warp B, which forms the finished column fma(c, x, RN(s*y)).
//   k = 2: warp A applies sequence 0 (4 instructions a column) and hands its
//          finished columns to warp B, which applies sequence 1 to them.
// The hand-off is a ring of RING tiles of CB values per lane in shared
// memory (ready/free barriers); the TMA stages are read by both warps and
// refilled by warp B, their last reader, once warp A is done with them too.
// Measured at n = 8192 (kernel time the same for 76 to 304 strips, so a
// warp's own dependent chain is the bound): k = 1 1.20 ms, 302 cycles a
// column, two dependent FP64 instructions of about 151 cycles each (one warp
// alone: 1.26 ms); k = 2 1.83 ms (one warp: 2.32 ms).  The chain's product
// on the integer pipe (dmul_int) was slower: 1.67 ms at k = 1.
template <int KR>
struct SplitShape {
  using SS = StreamShape<double, KR, 1>;
  static constexpr int RING = 4;
  static constexpr int kRingTile = SS::CB * 32 * (int)sizeof(double);
  static constexpr int kRingOff = SS::S * SS::kStage;
  static constexpr int kBarOff = kRingOff + RING * kRingTile;
  // barriers: full[S], consumed[S], ready[RING], ring_free[RING]; then the abort flag
  static constexpr int kSmem = kBarOff + (2 * SS::S + 2 * RING) * 8 + 16;
};

template <int KR>
__global__ void __launch_bounds__(64)
stream_split_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap csmap, double* A,
                    int64_t lda, int m, int n, int* status) {
  static_assert(KR == 1 || KR == 2, "one or two sequences");
  using SS = StreamShape<double, KR, 1>;
  using SP = SplitShape<KR>;
  using V2 = typename Pair<double>::type;
  constexpr int CB = SS::CB, S = SS::S, KP = SS::KP, RING = SP::RING;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SP::kBarOff);
  uint64_t* consumed = full + S;
  uint64_t* ready = consumed + S;
  uint64_t* ring_free = ready + RING;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ring_free + RING);
  double* ring = reinterpret_cast<double*>(smem + SP::kRingOff);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x;                     // strip of 32 rows
  const bool rowok = c * 32 + lane < m;
  double* const arow = A + (int64_t)c * 32 + lane;
  const int ntiles = (n + KR + CB - 1) / CB;    // waves -1 .. n-2+KR
  auto issue = [&](int t) {
    const int s = t % S;
    unsigned char* st = smem + s * SS::kStage;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], SS::kABytes + SS::kCsBytes);
    tma_load_2d(st, &amap, &full[s], c * 32, t * CB);
    tma_load_2d(st + SS::kAStage, &csmap, &full[s], 0, t * CB - 1);
  };
  if (threadIdx.x == 0) {
    prefetch_tmap(&amap);
    prefetch_tmap(&csmap);
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&consumed[s], 32);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(&ready[r], 32);
      mbar_init(&ring_free[r], 32);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
    for (int t = 0; t < S && t < ntiles; ++t) issue(t);
  }
  __syncthreads();
  // A bounded wait that also gives up once the other warp has.
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    bool ok = !*abort_flag && mbar_wait_bounded(bar, parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) {
      if (!*abort_flag) set_error(status, kDevTimeoutTma);
      *abort_flag = 1;
    }
    return ok;
  };
  int issued = ntiles < S ? ntiles : S;         // tiles whose copies warp B has started (lane 0's count)
  if (warp == 0) {
    // ---- warp A: the upstream chain ------------------------------------------------
    double x = 0.0;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % S, r = t % RING;
      if (!wait(&full[s], (uint32_t)(t / S) & 1u)) break;
      if (t >= RING && !wait(&ring_free[r], (uint32_t)(t / RING - 1) & 1u)) break;
      const double* at = reinterpret_cast<const double*>(smem + s * SS::kStage);
      const V2* cs = reinterpret_cast<const V2*>(smem + s * SS::kStage + SS::kAStage);
      double* out = ring + (size_t)r * CB * 32 + lane;
      const int w0 = t * CB - 1;
#pragma unroll 4
      for (int i = 0; i < CB; ++i) {
        const int w = w0 + i;                   // wave w takes in column w + 1
        const double y = at[i * 32 + lane];
        if (w < 0) {
          x = y;                                // column 0
        } else if (w <= n - 2) {
          const V2 p = cs[i * KP];              // rotation (w, w+1) of the first sequence
          if constexpr (KR == 1) {
            out[i * 32] = x;                    // the column's incoming value, for warp B
            x = __fma_rn(p.x, y, -__dmul_rn(p.y, x));
          } else {
            const double sy = __dmul_rn(p.y, y);
            const double sx = __dmul_rn(p.y, x);
            out[i * 32] = __fma_rn(p.x, x, sy); // column w after the first sequence
            x = __fma_rn(p.x, y, -sx);
          }
        } else if (w == n - 1) {
          out[i * 32] = x;                      // the last column after the first sequence
        }
      }
      mbar_arrive(&ready[r]);
      mbar_arrive(&consumed[s]);
    }
  } else {
    // ---- warp B: finished columns, stores, and the stage refills -----------------------
    double x1 = 0.0;
    double* ps = arow;                          // column 0 of this lane's row
    int t = 0;
    for (; t < ntiles; ++t) {
      const int s = t % S, r = t % RING;
      if (!wait(&full[s], (uint32_t)(t / S) & 1u)) break;
      if (!wait(&ready[r], (uint32_t)(t / RING) & 1u)) break;
      const double* at = reinterpret_cast<const double*>(smem + s * SS::kStage);
      const V2* cs = reinterpret_cast<const V2*>(smem + s * SS::kStage + SS::kAStage);
      const double* in = ring + (size_t)r * CB * 32 + lane;
      const int w0 = t * CB - 1;
#pragma unroll 4
      for (int i = 0; i < CB; ++i) {
        const int w = w0 + i;
        if constexpr (KR == 1) {
          if (w >= 0 && w <= n - 2) {
            const V2 p = cs[i * KP];
            const double v = __fma_rn(p.x, in[i * 32], __dmul_rn(p.y, at[i * 32 + lane]));
            if (rowok) st_cg(ps, v);            // column w, final
            ps += lda;
          } else if (w == n - 1) {
            if (rowok) st_cg(ps, in[i * 32]);   // column n-1, final
            ps += lda;
          }
        } else {
          if (w == 0) {
            x1 = in[i * 32];                    // column 0 after the first sequence
          } else if (w >= 1 && w <= n - 1) {
            const V2 p = cs[i * KP + 1];        // rotation (w-1, w) of the second sequence
            const double y1 = in[i * 32];
            const double sy = __dmul_rn(p.y, y1);
            const double sx = __dmul_rn(p.y, x1);
            const double v = __fma_rn(p.x, x1, sy);
            x1 = __fma_rn(p.x, y1, -sx);
            if (rowok) st_cg(ps, v);            // column w-1, final
            ps += lda;
          } else if (w == n) {
            if (rowok) st_cg(ps, x1);           // column n-1, final
            ps += lda;
          }
        }
      }
      mbar_arrive(&ring_free[r]);
      __syncwarp();
      // Both warps are done with stage s: refill it with tile t + S.
      if (t + S < ntiles) {
        if (!wait(&consumed[s], (uint32_t)(t / S) & 1u)) break;
        if (lane == 0) issue(t + S);
        ++issued;
      }
    }
    // On a timeout, let the copies still in flight land before leaving.
    if (t < ntiles && lane == 0)
      for (int u = t + 1; u < issued; ++u) (void)mbar_wait_bounded(&full[u % S], (uint32_t)(u / S) & 1u);
  }
}

}  // namespace rs
