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
  // On a timeout, let the copies still in flight (from tile t on) land before
  // leaving; one that already landed returns at once.
  if (t < ntiles && lane == 0) {
    for (int r = t; r < ntiles && r < t + S; ++r) (void)mbar_wait_bounded(&bar[r % S], (uint32_t)(r / S) & 1u);
  }
}

// ---------------------------------------------------------------------------
// FP64, one to four sequences: the column stream split over warps.
//
// GB300's FP64 unit belongs to an SM sub-partition and takes 64 cycles for a
// warp instruction, whatever its active lanes, and a row's chain of
// rotations is sequential: column after column, x <- fma(c, y, -RN(s*x)).
// Issued in order, every other FP64 instruction of the warp (the finished
// column fma(c, x, RN(s*y)) and its product) delays that chain.  So each warp
// here carries only two FP64 instructions a column, two warps a sequence:
// warp 2p the chain of sequence p, handing each column's incoming x to warp
// 2p + 1, which forms the finished column from it and sequence p's input
// column (A itself for p = 0, else warp 2p - 1's finished columns); warp
// 2p + 1's columns go to the chain of sequence p + 1, and the last warp's
// are the result.
// Every element sees rotate_dmul's operations on the same operands, in the
// same order: bit-identical.  Values pass between warps through rings of
// RING tiles of CB values per lane in shared memory (ready/free barriers);
// the TMA stages are read by every warp and refilled by one more, producer
// warp once all of them are done with a stage.  Only the barriers that hand
// data over (a filled stage, a written ring slot) are waited on with
// acquire semantics, after a test that does not suspend; the free and
// consumed barriers, which only report reads, are arrived on and waited on
// relaxed (the reads have completed: their values were used before the
// arrive).
// Each warp's role is a template parameter, so a chain warp's per-column path
// holds nothing but its two FP64 instructions, their loads and the hand-off
// store (with the roles as runtime branches: k = 1 1.33 ms).  Measured at
// 8192 x 8192 (kernel time the same for 76 to 152 strips of 32 rows, so a
// warp's own dependent chain is the bound): k = 1 1.13 ms, 280 cycles a
// column (one warp per strip: 1.26 ms); k = 2 1.48 ms (one warp: 2.32 ms; two
// warps, one per sequence: 1.83 ms).  The chain's product on the integer pipe
// (dmul_int) was slower: 1.67 ms at k = 1 (two-warp build).  Whole calls of
// rot_apply at k = 3 and 4: 0.80 and 0.85 ms at 4096 x 4096 (one strip per
// SM), 1.90 and 2.37 ms at 8192 x 8192 (two strips on most SMs, whose FP64
// units then bound it).
template <int KR>
struct SplitShape {
  using SS = StreamShape<double, KR, 1>;
  static constexpr int NW = 2 * KR;                        // warps
  static constexpr int NRING = NW - 1;                     // rings between consecutive warps
  static constexpr int RING = KR == 1 ? 4 : 2;             // tiles per ring
  // A warp starts a tile once the warp before it has handed the whole tile
  // over, so the last warp trails the first by about a tile per chain; the
  // S stages cover that lag and the copies' latency.  From three sequences
  // on, tiles of 16 columns keep 8 stages and the rings within half an SM's
  // shared memory (two CTAs per SM).
  static constexpr int CB = KR <= 2 ? SS::CB : 16;         // columns per tile
  static constexpr int S = 8;                              // TMA stages
  static constexpr int KP = SS::KP;
  static constexpr int kABytes = 32 * CB * (int)sizeof(double);
  static constexpr int kCsBytes = CB * 2 * KP * (int)sizeof(double);
  static constexpr int kAStage = (kABytes + 127) / 128 * 128;
  static constexpr int kStage = kAStage + (kCsBytes + 127) / 128 * 128;
  static constexpr int kRingTile = CB * 32 * (int)sizeof(double);
  static constexpr int kRingOff = S * kStage;
  static constexpr int kBarOff = kRingOff + NRING * RING * kRingTile;
  // barriers: full[S], consumed[S], ready[NRING][RING], free[NRING][RING]; then the abort flag
  static constexpr int kSmem = kBarOff + (2 * S + 2 * NRING * RING) * 8 + 16;
};

// Shared state of one CTA of stream_split_kernel.
struct SplitCta {
  const CUtensorMap* amap;
  const CUtensorMap* csmap;
  unsigned char* smem;
  uint64_t* full;
  uint64_t* consumed;
  uint64_t* ready;
  uint64_t* freed;
  volatile int* abort_flag;
  double* A;
  int64_t lda;
  int m, n, c, lane, ntiles;
  int* status;
};

// The tile loop of warp W (its role fixed at compile time, so that a chain
// warp's per-column path holds nothing but its two FP64 instructions, the
// loads feeding them and the hand-off store).
template <int KR, int W>
__device__ __forceinline__ void split_role(const SplitCta& X) {
  using SP = SplitShape<KR>;
  using V2 = typename Pair<double>::type;
  constexpr int CB = SP::CB, S = SP::S, KP = SP::KP, RING = SP::RING, NW = SP::NW;
  constexpr bool kChain = (W & 1) == 0;         // a chain (else finished columns)
  constexpr int kSeq = W / 2;                   // its sequence
  constexpr bool kWrites = W < NW - 1;          // hands values to the next warp
  constexpr bool kReadsPrev = W > 0;            // ring W-1: the previous warp's hand-off
  constexpr bool kReadsIn = !kChain && kSeq > 0;  // ring W-2: its sequence's input columns
  constexpr bool kLast = W == NW - 1;
  const int lane = X.lane, n = X.n;
  auto ring = [&](int g, int q) {
    return reinterpret_cast<double*>(X.smem + SP::kRingOff) + ((size_t)g * RING + q) * CB * 32 + lane;
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
  double x = 0.0;                               // a chain's carried value
  double* ps = X.A + (int64_t)X.c * 32 + lane;  // the last warp's next column
  for (int t = 0; t < X.ntiles; ++t) {
    const int s = t % S, q = t % RING;
    const uint32_t use = (uint32_t)(t / RING);
    if (*X.abort_flag) break;
    if (!settle(mbar_wait_data(&X.full[s], (uint32_t)(t / S) & 1u))) break;
    if (kReadsPrev && !settle(mbar_wait_data(&X.ready[(W - 1) * RING + q], use & 1u))) break;
    if (kReadsIn && !settle(mbar_wait_data(&X.ready[(W - 2) * RING + q], use & 1u))) break;
    if (kWrites && t >= RING && !settle(mbar_wait_read(&X.freed[W * RING + q], (use - 1) & 1u))) break;
    const double* at = reinterpret_cast<const double*>(X.smem + s * SP::kStage) + lane;
    const V2* cs = reinterpret_cast<const V2*>(X.smem + s * SP::kStage + SP::kAStage) + kSeq;
    double* out = kWrites ? ring(W, q) : nullptr;
    const double* in = kReadsPrev ? ring(W - 1, q) : nullptr;
    const double* in1 = kReadsIn ? ring(W - 2, q) : nullptr;
    // Sequence kSeq takes its input column j + 1 at wave w = j + kSeq; its
    // rotation (j, j+1) has the pair of wave w, index kSeq.
    const int j0 = t * CB - 1 - kSeq;
#pragma unroll 4
    for (int i = 0; i < CB; ++i) {
      const int j = j0 + i;
      if constexpr (kChain) {
        const double y = kSeq == 0 ? at[i * 32] : in[i * 32];   // input column j + 1
        if (j >= 0 && j <= n - 2) {
          out[i * 32] = x;                      // column j's incoming value
          x = __fma_rn(cs[i * KP].x, y, -__dmul_rn(cs[i * KP].y, x));
        } else if (j == -1) {
          x = y;                                // input column 0
        } else if (j == n - 1) {
          out[i * 32] = x;                      // the last column, final for this sequence
        }
      } else {
        if (j >= 0 && j <= n - 1) {
          double v = in[i * 32];                // column j's incoming value (final at j = n-1)
          if (j <= n - 2) {
            const double y = kSeq == 0 ? at[i * 32] : in1[i * 32];
            v = __fma_rn(cs[i * KP].x, v, __dmul_rn(cs[i * KP].y, y));
          }
          if constexpr (kLast) {
            if (rowok) st_cg(ps, v);            // column j, final
            ps += X.lda;
          } else {
            out[i * 32] = v;                    // column j after sequence 0, for the next chain
          }
        }
      }
    }
    if constexpr (kWrites) mbar_arrive(&X.ready[W * RING + q]);   // release: the slot's values
    if constexpr (kReadsPrev) mbar_arrive_relaxed(&X.freed[(W - 1) * RING + q]);
    if constexpr (kReadsIn) mbar_arrive_relaxed(&X.freed[(W - 2) * RING + q]);
    mbar_arrive_relaxed(&X.consumed[s]);
  }
}

// The producer warp: refills stage s with tile t + S once every compute
// warp is done with tile t; the CTA ends only once its last copies (all of
// them after a timeout) have landed.
template <int KR>
__device__ __forceinline__ void split_producer(const SplitCta& X) {
  using SP = SplitShape<KR>;
  constexpr int CB = SP::CB, S = SP::S;
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
      unsigned char* st = X.smem + s * SP::kStage;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&X.full[s], SP::kABytes + SP::kCsBytes);
      tma_load_2d(st, X.amap, &X.full[s], X.c * 32, (t + S) * CB);
      tma_load_2d(st + SP::kAStage, X.csmap, &X.full[s], 0, (t + S) * CB - 1);
    }
    ++issued;
  }
  if (X.lane == 0)
    for (int u = t; u < issued; ++u) (void)mbar_wait_bounded(&X.full[u % S], (uint32_t)(u / S) & 1u);
}

template <int KR>
__global__ void __launch_bounds__(64 * KR + 32)
stream_split_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap csmap, double* A,
                    int64_t lda, int m, int n, int* status) {
  static_assert(KR >= 1 && KR <= 4, "one to four sequences");
  using SP = SplitShape<KR>;
  constexpr int CB = SP::CB, S = SP::S, RING = SP::RING, NW = SP::NW, NRING = SP::NRING;
  extern __shared__ __align__(1024) unsigned char smem[];
  SplitCta X;
  X.amap = &amap;
  X.csmap = &csmap;
  X.smem = smem;
  X.full = reinterpret_cast<uint64_t*>(smem + SP::kBarOff);
  X.consumed = X.full + S;
  X.ready = X.consumed + S;                     // ready[g * RING + q]: ring g, slot q written
  X.freed = X.ready + NRING * RING;             // freed[g * RING + q]: ring g, slot q read by all its readers
  X.abort_flag = reinterpret_cast<volatile int*>(X.freed + NRING * RING);
  X.A = A;
  X.lda = lda;
  X.m = m;
  X.n = n;
  X.c = blockIdx.x;                             // strip of 32 rows
  X.lane = threadIdx.x & 31;
  X.ntiles = (n + KR + CB - 1) / CB;            // waves -1 .. n-2+KR
  X.status = status;
  if (threadIdx.x == 0) {
    prefetch_tmap(&amap);
    prefetch_tmap(&csmap);
    for (int s = 0; s < S; ++s) {
      mbar_init(&X.full[s], 1);
      mbar_init(&X.consumed[s], 32 * NW);       // every compute warp
    }
    for (int g = 0; g < NRING; ++g)
      for (int q = 0; q < RING; ++q) {
        mbar_init(&X.ready[g * RING + q], 32);
        // an odd ring (a sequence's finished columns) is read by the next
        // sequence's two warps, an even one (a chain's hand-off) by one
        mbar_init(&X.freed[g * RING + q], (g & 1) ? 64 : 32);
      }
    *X.abort_flag = 0;
    fence_mbarrier_init();
    for (int t = 0; t < S && t < X.ntiles; ++t) {
      unsigned char* st = smem + t * SP::kStage;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&X.full[t], SP::kABytes + SP::kCsBytes);
      tma_load_2d(st, &amap, &X.full[t], X.c * 32, t * CB);
      tma_load_2d(st + SP::kAStage, &csmap, &X.full[t], 0, t * CB - 1);
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  switch (warp) {
    case 0: split_role<KR, 0>(X); break;
    case 1: split_role<KR, 1>(X); break;
    case 2: if constexpr (KR >= 2) split_role<KR, 2>(X); break;
    case 3: if constexpr (KR >= 2) split_role<KR, 3>(X); break;
    case 4: if constexpr (KR >= 3) split_role<KR, 4>(X); break;
    case 5: if constexpr (KR >= 3) split_role<KR, 5>(X); break;
    case 6: if constexpr (KR >= 4) split_role<KR, 6>(X); break;
    case 7: if constexpr (KR >= 4) split_role<KR, 7>(X); break;
    default: break;
  }
  if (warp == NW) split_producer<KR>(X);
}

}  // namespace rs
