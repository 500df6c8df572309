// rs_wave.cuh -- the row-parallel wavefront kernel that applies a sequence of
// planar rotations to the columns of a column-major matrix (Algorithm 2's
// result, computed in Algorithm 3's wave order, Section 1.1).
//
// Work decomposition (GB300 design; the paper's blocking of Section 2 recast
// for warps):
//   chain c      : 32 consecutive rows of one instance, one row per lane.
//   p-block g    : sequences [g*K, g*K + kr), kr = min(K, k - g*K).
//   wave-block b : waves [b*NB, (b+1)*NB) of that p-block; wave w holds the
//                  rotations (j = w - l, p = g*K + l), l = 0..kr-1, in
//                  increasing l (Section 1.1: (i,j), (i-1,j+1), ...).
// An item (c, g, b) is one warp's unit of work.  Item (c,g,b) needs item
// (c,g,b-1) (the same rows' earlier waves of the same sequences) and enough
// of p-block g-1 to have finished every column it touches (the dependency
// rule of Section 2: block (j_b, p_b) before (j_b + n_b, p_b) and before
// (j_b - k_b, p_b + k_b)).  Items are handed out in increasing key
// b + delta*g by an atomic ticket, so every dependency holds a smaller ticket
// and is held by a running warp: no co-residency is needed and no deadlock
// can occur.  Between items the partially rotated columns live in A itself.
//
// Inside an item a warp keeps a window of KMAX+1 columns in registers.  Each
// wave loads one new column (coalesced: 32 lanes x one element), applies kr
// rotations to the window and retires the oldest column.  (c, s) pairs for the
// item's waves come from a wave-major repacked copy of C and S, staged into
// shared memory per warp by TMA (cp.async.bulk.tensor, double-buffered,
// completion on an mbarrier), and are read back with broadcast loads.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#include <cuda.h>
#include "rs_device.cuh"

namespace rs {

template <typename T> struct Pair;
template <> struct Pair<double> { using type = double2; };
template <> struct Pair<float> { using type = float2; };

// -0.0, computed afresh from s by two integer operations (opaque to the
// compiler, so it is neither folded into a constant nor hoisted).
__device__ __forceinline__ double neg_zero_from(double s) {
  unsigned long long r;
  asm volatile("{\n\tand.b64 %0, %1, 0x8000000000000000;\n\tor.b64 %0, %0, 0x8000000000000000;\n\t}"
               : "=l"(r)
               : "l"((unsigned long long)__double_as_longlong(s)));
  return __longlong_as_double((long long)r);
}

// RN(a*b) as a fused multiply-add with a -0 addend.  Bit-identical to the
// rounded product for every input: the exact product v is rounded once in
// both, v + (-0) = v for v != 0, and +0 + (-0) = +0, -0 + (-0) = -0 under
// round-to-nearest; infinities, NaN, overflow and subnormal results come out
// the same.  On GB300 the FP64 pipe issues DFMA faster than DMUL: measured on
// the rotation's own mix (registers only, (c, s) from shared memory), 2 DMUL
// + 2 DFMA reach 0.91 of the nominal pipe rate, 4 DFMA 0.95-0.99, but only
// when the -0 comes from a freshly computed register (a loop-invariant
// register operand, or a constant, issues at the DMUL rate).
__device__ __forceinline__ double mul_as_fma(double a, double b, double neg_zero) {
  return __fma_rn(a, b, neg_zero);
}

// Algorithm 1 with the fixed FMA placement:
//   x' = fma(c, x, RN(s*y)),  y' = fma(c, y, -RN(s*x)),
// the two rounded products taken as fma(s, ., -0) (see mul_as_fma).
__device__ __forceinline__ void rotate(double& x, double& y, double c, double s) {
  const double nz = neg_zero_from(s);
  const double sy = mul_as_fma(s, y, nz);
  const double sx = mul_as_fma(s, x, nz);
  const double xn = __fma_rn(c, x, sy);
  y = __fma_rn(c, y, -sx);
  x = xn;
}
// The rotation with DMUL products (bit-identical to rotate).  For kernels
// bound by the latency of one row's chain of rotations rather than by the
// FP64 pipe's issue rate (the column stream at one or two sequences), where
// the DFMA form measured slower (8192 x 8192, k = 1: 1.36 ms against 1.25).
__device__ __forceinline__ void rotate_dmul(double& x, double& y, double c, double s) {
  const double sy = __dmul_rn(s, y);
  const double sx = __dmul_rn(s, x);
  const double xn = __fma_rn(c, x, sy);
  y = __fma_rn(c, y, -sx);
  x = xn;
}
__device__ __forceinline__ void rotate(float& x, float& y, float c, float s) {
  const float sy = __fmul_rn(s, y);
  const float sx = __fmul_rn(s, x);
  const float xn = __fmaf_rn(c, x, sy);
  y = __fmaf_rn(c, y, -sx);
  x = xn;
}
__device__ __forceinline__ void rotate_dmul(float& x, float& y, float c, float s) { rotate(x, y, c, s); }

// RN(a*b) computed on the integer pipe, bit-identical to DMUL (IEEE round to
// nearest even) whenever a and b are normal and the product is a normal
// number that cannot overflow; `special` is set otherwise and the caller
// must use DMUL.  GB300 issues FP64 at 2 lanes per clock per SM but integer
// multiply-adds at 64, so moving the rotation's two products here leaves the
// FP64 pipe only the two fused multiply-adds.
//   a = Ma * 2^(ea-1075), b = Mb * 2^(eb-1075) with Ma, Mb in [2^52, 2^53).
//   Ma*Mb = P in [2^104, 2^106); with ma = Ma<<11, mb = Mb<<11 the 128-bit
//   product ma*mb = P*2^22, whose high word hi = floor(P/2^42) has its top
//   bit t set iff P >= 2^105.  The rounded mantissa is hi >> (10+t) plus the
//   round-to-even increment from the guard bit and the sticky bits (the rest
//   of hi and the whole low word); the biased exponent is ea + eb - 1023 + t,
//   and adding the 53-bit mantissa to (exponent-1)<<52 lets a rounding carry
//   (mantissa 2^53) move into the exponent field exactly as IEEE requires.
__host__ __device__ __forceinline__ unsigned long long umul64hi(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

__host__ __device__ __forceinline__ double dmul_int(double a, double b, bool& special) {
  const unsigned long long A = bits_of(a);
  const unsigned long long B = bits_of(b);
  const int ea = (int)(A >> 52) & 0x7ff;
  const int eb = (int)(B >> 52) & 0x7ff;
  const unsigned long long sign = (A ^ B) & 0x8000000000000000ull;
  const unsigned long long ma = ((A & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;
  const unsigned long long mb = ((B & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;
  const unsigned long long hi = umul64hi(ma, mb);
  const unsigned long long lo = ma * mb;
  const unsigned t = (unsigned)(hi >> 63);
  const unsigned sh = 10u + t;
  unsigned long long mant = hi >> sh;
  const unsigned long long guard = (hi >> (sh - 1u)) & 1ull;
  const unsigned long long rest = (hi & ((1ull << (sh - 1u)) - 1ull)) | lo;
  mant += guard & ((unsigned long long)(rest != 0ull) | (mant & 1ull));
  const int e = ea + eb - 1023 + (int)t;
  special = ((unsigned)(ea - 1) >= 2046u) | ((unsigned)(eb - 1) >= 2046u) | ((unsigned)(e - 1) >= 2045u);
  return double_of(sign | ((((unsigned long long)(unsigned)(e - 1)) << 52) + mant));
}

// The FP64 rotation with both products on the integer pipe (same result as
// rotate(double&, ...)); warps with any special lane recompute those
// products with DMUL.
__device__ __forceinline__ void rotate_intmul(double& x, double& y, double c, double s) {
  bool sp1, sp2;
  double sy = dmul_int(s, y, sp1);
  double sx = dmul_int(s, x, sp2);
  if (__any_sync(0xffffffffu, sp1 | sp2)) {
    if (sp1) sy = __dmul_rn(s, y);
    if (sp2) sx = __dmul_rn(s, x);
  }
  const double xn = __fma_rn(c, x, sy);
  y = __fma_rn(c, y, -sx);
  x = xn;
}

// A 2x2 reflector H = I - tau*v*v^T, v = (1, nu), applied to the row pair
// (Section 6: three multiplications and three additions), with the fixed
// placement t = fma(nu, y, x), w = RN(tau*t), x' = RN(x - w), y' = fma(-nu, w, y).
// In FP64 the product and the difference are DFMAs with freshly computed
// constants: RN(tau*t) = fma(tau, t, -0) and RN(x - w) = fma(w, -1, x), both
// bit-identical (the product by -1 is exact), issued at the DFMA rate.
__device__ __forceinline__ void reflect(double& x, double& y, double tau, double nu) {
  const double nz = neg_zero_from(tau);
  unsigned long long m1b;
  asm volatile("{\n\tand.b64 %0, %1, 0;\n\tor.b64 %0, %0, 0xBFF0000000000000;\n\t}"
               : "=l"(m1b)
               : "l"((unsigned long long)__double_as_longlong(nu)));
  const double m1 = __longlong_as_double((long long)m1b);   // -1.0
  const double t = __fma_rn(nu, y, x);
  const double w = mul_as_fma(tau, t, nz);
  const double xn = __fma_rn(w, m1, x);
  y = __fma_rn(-nu, w, y);
  x = xn;
}
__device__ __forceinline__ void reflect(float& x, float& y, float tau, float nu) {
  const float t = __fmaf_rn(nu, y, x);
  const float w = __fmul_rn(tau, t);
  const float xn = __fsub_rn(x, w);
  y = __fmaf_rn(-nu, w, y);
  x = xn;
}

// What a wave kernel applies to each row pair.
enum WaveOp : int {
  kOpRotate = 1,        // rotation (c, s), products with DMUL
  kOpRotateIntmul = 2,  // rotation (c, s), products on the integer pipe
  kOpReflect = 3,       // 2x2 reflector (tau, nu)
};

// One instance of the problem as the wave kernel sees it.
struct WaveInstance {
  void* A;          // column-major m x n, leading dimension lda (elements)
  int64_t lda;
  // Elements from row 0 of one 32-row strip to row 0 of the next: 0 means 32
  // (plain column-major).  The packed layout (strips of 32 rows stored one
  // after the other, each a 32 x n column-major panel) has lda = 32 and
  // chain_stride = 32 n.
  int64_t chain_stride;
  int m, n, k;
  int K;            // sequences per p-block
  int NB;           // waves per item
  int delta;        // key stride between p-blocks: 1 + ceil(K / NB)
  int nchains;      // ceil(m / 32)
  int G;            // p-blocks: ceil(k / K)
  int B;            // wave-blocks of a full p-block: ceil((n + K - 2) / NB)
  int cs_row0;      // (c,s) tensor row of rotation (j, p) is cs_row0 + j + p
  int p_base;       // (c,s) tensor column pair of sequence p is p_base + p
  int j_lo, j_hi;   // rotations exist for j_lo <= j <= j_hi (normally 0, n-2)
  int W_lo, W_hi;   // and for j + p in [W_lo, W_hi) (normally everything)
  int unit_rows;    // 1: row r of A starts as the unit vector e_r (accumulated blocks)
  int* done;        // [nchains * G] completed wave-blocks per (chain, p-block)
  const void* tmap; // TMA descriptor of the (c,s) tensor (global memory), batched kernel only
  unsigned long long wait_ns;  // limit of one dependency wait (0: kWaitLimitNs)
  // Streaming A in and out while the kernel runs (both optional, null = off):
  const int* arrived;  // arrived[c / arrive_cols] != 0 once columns of that chunk are in A
  int arrive_cols;
  int* last_done;      // last_done[b]: chains that finished wave-block b of the last p-block
};

// The whole problem: every rotation (j, p) with 0 <= j <= n-2, 0 <= p < k.
__host__ __device__ inline void set_full_range(WaveInstance& I) {
  I.p_base = 0;
  I.j_lo = 0;
  I.j_hi = I.n - 2;
  I.W_lo = 0;
  I.W_hi = 0x7fffffff;
  I.unit_rows = 0;
}

// Kernel-wide state of one launch.
struct WaveLaunch {
  unsigned long long* ticket;  // next ticket to hand out
  int* status;                 // first device error of this launch (0 = none)
  long long total;             // number of tickets
};

// Backwards-compatible name for the single-instance kernel's parameters.
struct WaveProblem : WaveInstance {
  unsigned long long* ticket;
  int* status;
  long long total;
};

// One run of consecutive tickets that belong to one (key, instance).
struct WaveSegment {
  long long start;  // first ticket of the run
  int inst;         // instance index
  int key;          // key kappa = b + delta * g
};

// Number of (g, b) pairs whose key b + delta*g equals kappa.
__device__ __forceinline__ int pairs_in_key(int kappa, int G, int B, int delta, int* g_lo) {
  int hi = kappa / delta;
  if (hi > G - 1) hi = G - 1;
  int lo = kappa - (B - 1);
  lo = lo <= 0 ? 0 : (lo + delta - 1) / delta;
  *g_lo = lo;
  return hi >= lo ? hi - lo + 1 : 0;
}

// Repack C, S ((n-1) x k, column-major) into rows of (c, s) pairs indexed by
// j + p: out[(row0 + j + p) * W2 + 2p + {0,1}] = (C(j,p), S(j,p)).  Item
// (c,g,b) then finds all pairs of its wave w in row w + g*K, columns
// [2gK, 2gK + 2kr): a rectangle that TMA can fetch.
template <typename T>
__global__ void repack_cs_kernel(const T* __restrict__ C, int64_t ldc, const T* __restrict__ S,
                                 int64_t lds, int n, int k, T* __restrict__ out, int64_t W2,
                                 int row0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= n - 1 || p >= k) return;
  typename Pair<T>::type v;
  v.x = C[j + (int64_t)p * ldc];
  v.y = S[j + (int64_t)p * lds];
  *reinterpret_cast<typename Pair<T>::type*>(out + (int64_t)(row0 + j + p) * W2 + 2 * p) = v;
}

template <typename T, int KMAX, int NBT>
struct WaveSmem {
  static constexpr int kTileElems = NBT * 2 * KMAX;              // one buffer
  static constexpr int kBoxBytes = kTileElems * (int)sizeof(T);   // bytes one TMA copy delivers
  // A TMA destination in shared memory must be 128-byte aligned, so each
  // buffer occupies a whole number of 128-byte lines.
  static constexpr int kTileBytes = (kBoxBytes + 127) / 128 * 128;
  static constexpr int kWarpBytes = 2 * kTileBytes + 128;         // 2 buffers + barriers
  static_assert(kWarpBytes % 128 == 0, "per-warp tile buffers must stay 128-byte aligned");
};

// Per-warp shared-memory resources: two (c,s) tile buffers and their mbarriers.
template <typename T, int KMAX, int NBT>
struct WarpTiles {
  unsigned char* base;
  uint64_t* bar;
  uint32_t phase0, phase1;
  __device__ __forceinline__ T* tile(int i) const {
    return reinterpret_cast<T*>(base + i * WaveSmem<T, KMAX, NBT>::kTileBytes);
  }
};

template <typename T, int KMAX, int NBT, int WARPS>
__device__ __forceinline__ WarpTiles<T, KMAX, NBT> warp_tiles_init(unsigned char* smem_raw, int lane) {
  using SM = WaveSmem<T, KMAX, NBT>;
  const int warp = threadIdx.x >> 5;
  WarpTiles<T, KMAX, NBT> wt;
  wt.base = smem_raw + warp * SM::kWarpBytes;
  wt.bar = reinterpret_cast<uint64_t*>(wt.base + 2 * SM::kTileBytes);
  wt.phase0 = 0;
  wt.phase1 = 0;
  if (lane == 0) {
    mbar_init(&wt.bar[0], 1);
    mbar_init(&wt.bar[1], 1);
    fence_mbarrier_init();
  }
  __syncwarp();
  return wt;
}

// Work item (c, g, b) of instance I.  Returns false if the launch must stop
// (an error was recorded in *status).
// OP (a WaveOp) selects the operation on each row pair: a rotation with its
// products on DMUL or on the integer pipe (bit-identical), or a reflector.
template <typename T, int KMAX, int NBT, int OP>
__device__ __forceinline__ bool run_item(const WaveInstance& I, const void* tmap, int c, int g,
                                         int b, WarpTiles<T, KMAX, NBT>& wt, int lane,
                                         int* status) {
  using V2 = typename Pair<T>::type;
  using SM = WaveSmem<T, KMAX, NBT>;
  const int n = I.n;
  const int p0 = g * I.K;
  const int kr = min(I.K, I.k - p0);
  const int nw = n + kr - 2;                 // waves of this p-block
  const int w0 = b * I.NB;
  if (w0 >= nw) return true;                 // empty tail item of a short p-block
  const int w1 = min(w0 + I.NB, nw);
  int* const done = I.done + (int64_t)c * I.G;

  // ---- wait for dependencies ------------------------------------------------
  bool ok = true;
  if (lane == 0) {
    const unsigned long long lim = I.wait_ns ? I.wait_ns : kWaitLimitNs;
    if (b > 0) ok = wait_flag_geq(done + g, b, status, lim);
    if (ok && g > 0) {
      const int krp = I.K;                   // every p-block but the last is full
      const int Bp = (n + krp - 2 + I.NB - 1) / I.NB;
      int need = (w1 + krp + I.NB - 1) / I.NB;
      if (need > Bp) need = Bp;
      ok = wait_flag_geq(done + g - 1, need, status, lim);
    }
    // The first p-block reads columns up to w1 + 1 straight from A: when A is
    // being uploaded while the kernel runs, wait for the chunk holding them
    // (chunks arrive in column order).
    if (ok && g == 0 && I.arrived)
      ok = wait_flag_geq(I.arrived + min(w1 + 1, n - 1) / I.arrive_cols, 1, status, lim);
    if (!ok) set_error(status, kDevTimeoutDependency);
  }
  ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
  if (!ok) return false;

  // ---- load the window: columns [w0-kr+1, w0] owned by this p-block ---------
  const int row = c * 32 + lane;
  const bool rowok = row < I.m;
  T* const arow = reinterpret_cast<T*>(I.A) + (int64_t)c * (I.chain_stride ? I.chain_stride : 32) + lane;
  const int64_t lda = I.lda;
  const int own_lo = w0 - kr + 1;
  T win[KMAX + 1];
#pragma unroll
  for (int s = 0; s < KMAX; ++s) {
    const int q = w0 + 1 - KMAX + s;
    win[s] = (rowok && q >= own_lo && q >= 0 && q <= n - 1) ? ld_cg(arow + (int64_t)q * lda) : T(0);
  }
  T nextcol = (rowok && w0 + 1 <= n - 1) ? ld_cg(arow + (int64_t)(w0 + 1) * lda) : T(0);

  // Waves of this p-block that hold rotations: the full-sequence wave
  // j + p = w + p0 must lie in [W_lo, W_hi).
  int wr_lo = I.W_lo - p0;
  const int wr_hi = I.W_hi - p0;
  // Rows that start as unit vectors e_r: before rotation (j, p) (p counted
  // from the instance's first sequence) row r can be non-zero only in columns
  // >= r - p - 1, because each sequence spreads a row's support at most one
  // column to the left.  So for every row r >= 32c of this chain, rotation
  // (j = w - l, p = p0 + l) acts on two zeros when w < 32c - p0 - 2, whatever
  // l is: such waves are skipped.  Skipping changes at most the sign of zeros.
  if (I.unit_rows) wr_lo = max(wr_lo, c * 32 - p0 - 2);

  // ---- stream (c,s) tiles and run the waves ---------------------------------
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
      // Let the copy already issued into the other buffer land before leaving.
      if (st + 1 < ntiles) (void)mbar_wait_bounded(&wt.bar[cur ^ 1], cur ? wt.phase0 : wt.phase1);
      return false;
    }
    const V2* tl = reinterpret_cast<const V2*>(wt.tile(cur));
    const int ws = w0 + st * NBT;
    const int wend = min(ws + NBT, w1);
    for (int w = ws; w < wend; ++w) {
      win[KMAX] = nextcol;
      nextcol = (rowok && w + 2 <= n - 1) ? ld_cg(arow + (int64_t)(w + 2) * lda) : T(0);
      // Rotations l = l_lo..l_hi in increasing l, j = w - l in [j_lo, j_hi].
      // The bounds are the same for all lanes, so the early exit is a
      // uniform branch and a short p-block issues only its own kr rotations.
      const int l_lo = max(0, w - I.j_hi);
      const int l_hi = (w >= wr_lo && w < wr_hi) ? min(kr - 1, w - I.j_lo) : -1;
      const V2* trow = tl + (w - ws) * KMAX;
#pragma unroll
      for (int l = 0; l < KMAX; ++l) {
        if (l > l_hi) break;
        if (l >= l_lo) {
          const V2 cs = trow[l];
          if constexpr (OP == kOpRotateIntmul && sizeof(T) == 8)
            rotate_intmul(win[KMAX - 1 - l], win[KMAX - l], cs.x, cs.y);
          else if constexpr (OP == kOpReflect)
            reflect(win[KMAX - 1 - l], win[KMAX - l], cs.x, cs.y);
          else
            rotate(win[KMAX - 1 - l], win[KMAX - l], cs.x, cs.y);
        }
      }
      const int q = w + 1 - KMAX;            // column leaving the window
      if (rowok && q >= own_lo && q >= 0) st_cg(arow + (int64_t)q * lda, win[0]);
#pragma unroll
      for (int s = 0; s < KMAX; ++s) win[s] = win[s + 1];
    }
    __syncwarp();
  }

  // ---- flush the window: columns [w1+1-KMAX, w1] ----------------------------
#pragma unroll
  for (int s = 0; s < KMAX; ++s) {
    const int q = w1 + 1 - KMAX + s;
    if (rowok && q >= own_lo && q >= 0 && q <= n - 1) st_cg(arow + (int64_t)q * lda, win[s]);
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    st_release_gpu(done + g, b + 1);
    if (I.last_done && g == I.G - 1) {
      // Columns this item finished may now be copied out by another engine.
      __threadfence_system();
      atomicAdd(I.last_done + b, 1);
    }
  }
  return true;
}

// Hand out the next ticket to the whole warp; -1 when the launch is over.
__device__ __forceinline__ long long next_ticket(unsigned long long* ticket, long long total,
                                                 const int* status, int lane) {
  long long t = 0;
  if (lane == 0) {
    t = (long long)atomicAdd(ticket, 1ull);
    if (t >= total || ld_relaxed_gpu(status) != 0) t = -1;
  }
  return __shfl_sync(0xffffffffu, t, 0);
}

// Single instance: tickets decode in closed form (keys b + delta*g, within a
// key p-block-major then chain-minor).  Every warp runs the ticket loop
// independently; warps of a CTA share nothing but the CTA's shared memory.
template <typename T, int KMAX, int NBT, int WARPS, int OP = kOpRotate>
__global__ void __launch_bounds__(WARPS * 32)
wave_kernel(const __grid_constant__ CUtensorMap tmap, const WaveProblem P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  auto wt = warp_tiles_init<T, KMAX, NBT, WARPS>(smem_raw, lane);
  if (lane == 0) prefetch_tmap(&tmap);

  // Ticket -> key cursor (tickets a warp receives only increase).
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
    if (kappa > last_key) {                    // cannot happen: keys cover every ticket
      if (lane == 0) set_error(P.status, kDevBadItem);
      break;
    }
    const long long r = t - kstart;
    const int gi = (int)(r / P.nchains);
    const int c = (int)(r - (long long)gi * P.nchains);
    const int g = kglo + gi;
    const int b = kappa - P.delta * g;
    if (!run_item<T, KMAX, NBT, OP>(P, &tmap, c, g, b, wt, lane, P.status)) break;
  }
}

// Many instances in one launch: tickets run through a host-built table of
// segments (key, instance, first ticket), ordered by key and then instance,
// so that every dependency of an item has a smaller ticket.
template <typename T, int KMAX, int NBT, int WARPS, int OP = kOpRotate>
__global__ void __launch_bounds__(WARPS * 32)
wave_batched_kernel(const WaveInstance* __restrict__ insts, const WaveSegment* __restrict__ segs,
                    int nseg, const WaveLaunch L) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  auto wt = warp_tiles_init<T, KMAX, NBT, WARPS>(smem_raw, lane);
  int s = 0;
  while (true) {
    const long long t = next_ticket(L.ticket, L.total, L.status, lane);
    if (t < 0) break;
    while (s + 1 < nseg && t >= segs[s + 1].start) ++s;
    const WaveSegment sg = segs[s];
    const WaveInstance I = insts[sg.inst];
    int glo = 0;
    const int npairs = pairs_in_key(sg.key, I.G, I.B, I.delta, &glo);
    const long long r = t - sg.start;
    const int gi = (int)(r / I.nchains);
    if (gi >= npairs || t < sg.start) {        // cannot happen: segments cover every ticket
      if (lane == 0) set_error(L.status, kDevBadItem);
      break;
    }
    const int c = (int)(r - (long long)gi * I.nchains);
    const int g = glo + gi;
    const int b = sg.key - I.delta * g;
    if (!run_item<T, KMAX, NBT, OP>(I, I.tmap, c, g, b, wt, lane, L.status)) break;
  }
}

}  // namespace rs
