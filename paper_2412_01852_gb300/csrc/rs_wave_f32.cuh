// rs_wave_f32.cuh -- the FP32 wavefront kernel.
//
// Same work decomposition, ticket order, dependency counters and TMA-staged
// (c,s) tiles as the FP64 kernel (rs_wave.cuh), shaped for FP32 speed, where
// the rotation's 4 FP32 instructions are cheap and bookkeeping is not:
//   * R rows per lane (a chain is 32R rows), so each (c,s) pair loaded from
//     shared memory serves R rotations;
//   * tiles of KMAX+1 waves.  A tile whose waves are all interior (every
//     rotation of the wave exists, every column load and store is in range)
//     runs fully unrolled with the register window rotated by static indices:
//     after KMAX+1 waves the window is back in its canonical order, so no
//     register moves, no per-rotation branches.  The unrolled tile has to fit
//     the instruction cache, which bounds KMAX;
//   * the columns of the next tile are loaded one tile ahead;
//   * edge tiles (startup and shutdown triangles, short p-blocks, the ragged
//     last item) use the generic per-wave code with a shifted window.
// Both paths keep the window canonical at tile boundaries:
// slot s holds column ws + 1 - KMAX + s before wave ws.
#pragma once
#include "rs_wave.cuh"

namespace rs {

template <int KMAX, int R>
__device__ __forceinline__ bool run_item_f32(const WaveInstance& I, const void* tmap, int c, int g, int b,
                                             WarpTiles<float, KMAX, KMAX + 1>& wt, int lane, int* status) {
  using T = float;
  using V2 = float2;
  constexpr int NBT = KMAX + 1;
  constexpr int U = KMAX + 1;
  using SM = WaveSmem<T, KMAX, NBT>;
  const int n = I.n;
  const int p0 = g * I.K;
  const int kr = min(I.K, I.k - p0);
  const int nw = n + kr - 2;
  const int w0 = b * I.NB;
  if (w0 >= nw) return true;
  const int w1 = min(w0 + I.NB, nw);
  int* const done = I.done + (int64_t)c * I.G;

  bool ok = true;
  if (lane == 0) {
    if (b > 0) ok = wait_flag_geq(done + g, b, status);
    if (ok && g > 0) {
      const int krp = I.K;
      const int Bp = (n + krp - 2 + I.NB - 1) / I.NB;
      int need = (w1 + krp + I.NB - 1) / I.NB;
      if (need > Bp) need = Bp;
      ok = wait_flag_geq(done + g - 1, need, status);
    }
    if (!ok) set_error(status, kDevTimeoutDependency);
  }
  ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
  if (!ok) return false;

  const int64_t lda = I.lda;
  const int64_t cstr = I.chain_stride ? I.chain_stride : 32;   // between 32-row strips
  // Retired columns are read again by the next p-block about two items
  // later; storing them as evict_last keeps more of them in L2 (measured:
  // 2.5 % less time at 8192 x 8192, k = 192; the p-blocks in flight span
  // more columns than L2 holds).
  const unsigned long long keep = l2_evict_last_policy();
  T* arow[R];
  bool rowok[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = c * (32 * R) + r * 32 + lane;
    rowok[r] = row < I.m;
    arow[r] = reinterpret_cast<T*>(I.A) + (int64_t)(c * R + r) * cstr + lane;
  }
  const int own_lo = w0 - kr + 1;
  // Columns enter the window one per wave (column w+1 at wave w).  At FP32
  // speed a wave is ~100 issue cycles, shorter than an L2 round trip, so the
  // U columns of the next tile are loaded one tile ahead into `pre`:
  // pre[r][u] holds column ws+u+1 when tile ws starts.  Only columns <= w1 are
  // loaded: the dependency wait above made exactly those final.
  const int col_hi = min(w1, n - 1);
  T win[R][KMAX + 1];
  T pre[R][U];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
      const int q = w0 + 1 - KMAX + s;
      win[r][s] = (rowok[r] && q >= own_lo && q >= 0 && q <= n - 1) ? ld_cg(arow[r] + (int64_t)q * lda) : T(0);
    }
    win[r][KMAX] = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = w0 + 1 + u;
      pre[r][u] = (rowok[r] && q <= col_hi) ? ld_cg(arow[r] + (int64_t)q * lda) : T(0);
    }
  }

  const int ntiles = (w1 - w0 + NBT - 1) / NBT;
  const int tx = 2 * (I.p_base + p0);
  const int ty0 = I.cs_row0 + w0 + p0;
  if (lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&wt.bar[0], SM::kBoxBytes);
    tma_load_2d(wt.tile(0), tmap, &wt.bar[0], tx, ty0);
  }
  for (int st = 0; st < ntiles; ++st) {
    const int cur = st & 1;
    if (st + 1 < ntiles && lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&wt.bar[cur ^ 1], SM::kBoxBytes);
      tma_load_2d(wt.tile(cur ^ 1), tmap, &wt.bar[cur ^ 1], tx, ty0 + (st + 1) * NBT);
    }
    const uint32_t ph = cur ? wt.phase1 : wt.phase0;
    if (!mbar_wait_bounded(&wt.bar[cur], ph)) {
      if (lane == 0) set_error(status, kDevTimeoutTma);
      ok = false;
    }
    if (cur) wt.phase1 ^= 1u; else wt.phase0 ^= 1u;
    if (!__all_sync(0xffffffffu, ok)) {
      if (st + 1 < ntiles) (void)mbar_wait_bounded(&wt.bar[cur ^ 1], cur ? wt.phase0 : wt.phase1);
      return false;
    }
    const V2* tl = reinterpret_cast<const V2*>(wt.tile(cur));
    const int ws = w0 + st * NBT;
    const int wend = min(ws + NBT, w1);
    // A tile is interior when it holds all U waves, every wave has all KMAX
    // rotations (kr == KMAX, ws >= KMAX-1, last wave <= n-2) and every
    // column load w+2 stays below n (ws + U + 1 <= n - 1).  The instance has
    // no wave window and no j restriction (plain problems only).
    const bool interior = (wend - ws == U) && kr == KMAX && ws >= KMAX - 1 && ws + U + 1 <= n - 1;
    if (interior) {
      // Column pointers advance by one column per wave (no per-access
      // multiply).  Whether the next tile's columns all exist is decided
      // once for the tile: if it is not whole, only its first column (the
      // one an edge tile takes from `pre`) is fetched.
      const bool next_whole = ws + 2 * U <= col_hi;
      const bool next_first = ws + U + 1 <= col_hi;
      const T* pl = reinterpret_cast<const T*>(I.A) + (int64_t)(ws + U + 1) * lda + (int64_t)c * R * cstr + lane;
      T* ps = reinterpret_cast<T*>(I.A) + (int64_t)(ws + 1 - KMAX) * lda + (int64_t)c * R * cstr + lane;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool fetch = u == 0 ? next_first : next_whole;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          win[r][(KMAX + u) % U] = pre[r][u];
          pre[r][u] = T(0);
          if (fetch && rowok[r]) pre[r][u] = ld_cg(pl + r * cstr);
        }
        pl += lda;
        const V2* trow = tl + u * KMAX;
#pragma unroll
        for (int l = 0; l < KMAX; ++l) {
          const V2 cs = trow[l];
#pragma unroll
          for (int r = 0; r < R; ++r)
            rotate(win[r][(KMAX - 1 - l + u) % U], win[r][(KMAX - l + u) % U], cs.x, cs.y);
        }
        // column w + 1 - KMAX (>= own_lo and >= 0 in an interior tile) retires
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (rowok[r]) st_l2_keep(ps + r * cstr, win[r][u % U], keep);
        ps += lda;
      }
    } else {
      T nextcol[R];
#pragma unroll
      for (int r = 0; r < R; ++r) nextcol[r] = pre[r][0];
      for (int w = ws; w < wend; ++w) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          win[r][KMAX] = nextcol[r];
          nextcol[r] = (rowok[r] && w + 2 <= col_hi) ? ld_cg(arow[r] + (int64_t)(w + 2) * lda) : T(0);
        }
        const int l_lo = max(0, w - (n - 2));
        const int l_hi = min(kr - 1, w);
        const V2* trow = tl + (w - ws) * KMAX;
#pragma unroll
        for (int l = 0; l < KMAX; ++l) {
          if (l > l_hi) break;
          if (l >= l_lo) {
            const V2 cs = trow[l];
#pragma unroll
            for (int r = 0; r < R; ++r) rotate(win[r][KMAX - 1 - l], win[r][KMAX - l], cs.x, cs.y);
          }
        }
        const int q = w + 1 - KMAX;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (rowok[r] && q >= own_lo && q >= 0) st_cg(arow[r] + (int64_t)q * lda, win[r][0]);
#pragma unroll
          for (int s = 0; s < KMAX; ++s) win[r][s] = win[r][s + 1];
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = wend + 1 + u;
          pre[r][u] = (rowok[r] && q <= col_hi) ? ld_cg(arow[r] + (int64_t)q * lda) : T(0);
        }
      }
    }
    __syncwarp();
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
      const int q = w1 + 1 - KMAX + s;
      if (rowok[r] && q >= own_lo && q >= 0 && q <= n - 1) st_cg(arow[r] + (int64_t)q * lda, win[r][s]);
    }
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    st_release_gpu(done + g, b + 1);
  }
  return true;
}

// Single FP32 instance; same ticket decode as wave_kernel.
template <int KMAX, int R, int WARPS, int MINB = 1>
__global__ void __launch_bounds__(WARPS * 32, MINB)
wave_f32_kernel(const __grid_constant__ CUtensorMap tmap, const WaveProblem P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  auto wt = warp_tiles_init<float, KMAX, KMAX + 1, WARPS>(smem_raw, lane);
  if (lane == 0) prefetch_tmap(&tmap);
  int kappa = 0;
  long long kstart = 0;
  int kglo = 0;
  int kcount = pairs_in_key(0, P.G, P.B, P.delta, &kglo) * P.nchains;
  const int last_key = (P.B - 1) + P.delta * (P.G - 1);
  while (true) {
    const long long t = next_ticket(P.ticket, P.total, P.status, lane);
    if (t < 0) break;
    while (t >= kstart + kcount && kappa <= last_key) {
      kstart += kcount;
      ++kappa;
      kcount = pairs_in_key(kappa, P.G, P.B, P.delta, &kglo) * P.nchains;
    }
    if (kappa > last_key) {
      if (lane == 0) set_error(P.status, kDevBadItem);
      break;
    }
    const long long r = t - kstart;
    const int gi = (int)(r / P.nchains);
    const int c = (int)(r - (long long)gi * P.nchains);
    const int g = kglo + gi;
    const int b = kappa - P.delta * g;
    if (!run_item_f32<KMAX, R>(P, &tmap, c, g, b, wt, lane, P.status)) break;
  }
}

}  // namespace rs
