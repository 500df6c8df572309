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

}  // namespace rs
