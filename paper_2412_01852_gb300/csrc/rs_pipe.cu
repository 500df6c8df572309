// rs_pipe.cu -- rotations as a pipeline of sequences across the lanes of a
// warp (FP32 and FP64).
//
// One sequence's sweep over a row (Algorithm 2's inner loop) needs a single
// value of state: at column q it rotates the carried column q-1 with the
// incoming column q, emits column q-1 (final for this sequence) and carries
// the new column q.  Sequences p, p+1, ... are therefore stages of a
// pipeline: sequence l works on column t - 2l at step t, and its output
// reaches sequence l+1 one step later.  Each rotation sees the operands it
// sees in Algorithm 2, so the result is bit-exact with the sequential loop.
//
// A warp is G groups of 32/G lanes.  Lane i of a group holds sequences
// SPL*i .. SPL*i + SPL - 1 (KS stages per group) and the group streams its R
// rows through all n columns, a shuffle per row and step handing each value
// to the next lane of the group.  The group's first lane takes the columns
// in, its last lane emits the finished ones; both go through 32-column tiles
// in shared memory that the whole warp loads and stores (the next tile is
// fetched one tile ahead).  The (c,s) of step t are one row of a table in
// which every lane finds its SPL pairs side by side.  Tiles where every
// stage has its rotation run without predicates; at the two ends of the
// stream a stage without a rotation passes its values through unchanged, so
// zeros keep their sign and infinities stay.
//
// FP32 (k >= 32): one group, up to 192 stages per pass, 7 rows, 4 warps per
// CTA.  FP64 (3 <= k <= 32): GB300's FP64
// unit takes as long for a warp instruction whatever its active lanes, so
// every lane holds a stage: k is rounded up to a power of two KS and the warp
// holds 32/KS independent groups; CTAs of one warp up to KS = 16, of 4 warps
// at KS = 32.
//
// The warps of a CTA run in step and share the (c,s) table through shared
// memory: one bulk copy per 32-step tile, two or three tiles in flight,
// waits bounded (a timeout sets the status).
#include <algorithm>
#include <cuda_runtime.h>

#include "rs_device.cuh"
#include "rs_internal.h"
#include "rs_wave.cuh"

namespace rs {
namespace {

constexpr int kPTC = 32;      // steps (columns) per tile
constexpr int kPMaxSpl = 6;   // FP32 sequences per lane: 192 per pass

// W: warps per CTA.
template <typename T, int SPL, int G, int R, int W = 4>
struct Pipe {
  using P2 = typename Pair<T>::type;
  static constexpr int LPG = 32 / G;                             // lanes per group
  static constexpr int KS = LPG * SPL;                           // stages per group
  static constexpr int ROWS = G * R;                             // rows per warp
  static constexpr int EPC = 16 / (int)sizeof(T);                // elements per 16-byte chunk
  static constexpr int CPG = (R + EPC - 1) / EPC;                // chunks per group in a column slot
  static constexpr int NCH = G * CPG;                            // chunks per column slot
  static constexpr int SLOT = NCH * EPC;                         // elements per column slot
  static constexpr int kTabBytes = kPTC * KS * (int)sizeof(P2);  // (c,s) of one 32-step tile
  static constexpr int NS = kTabBytes >= 32768 ? 2 : 3;          // table tiles in flight
  static constexpr int kWarpElems = 3 * kPTC * SLOT;             // two input tiles, one output tile
  static constexpr int kSmem = NS * kTabBytes + W * kWarpElems * (int)sizeof(T) + NS * 8;
  static_assert(NCH == 1 || NCH == 2 || NCH == 4 || NCH == 8, "column slot of 1, 2, 4 or 8 chunks");
  static_assert(32 % G == 0, "groups split the warp evenly");
};

// Column q's slot in a staging tile holds the warp's rows, group g's in
// chunks g*CPG ...; chunk c sits at position c ^ swz(q), so that eight lanes
// storing or loading chunk c of their columns with 128-bit accesses hit
// distinct banks.
template <int NCH>
__device__ __forceinline__ int chunk_at(int q, int c) {
  if constexpr (NCH == 1) return q;
  else return q * NCH + (c ^ ((q / (8 / NCH)) & (NCH - 1)));
}

// tab[t][l] = (c, s) of rotation (j, p0 + l), j = t - 2l - 1, where
// 0 <= j <= n-2 and l < kp; (1, 0) elsewhere (never used).  32 x 32 tiles
// through shared memory: reads run along j, writes along l.
template <typename T>
__global__ void pipe_table_kernel(const T* __restrict__ C, int64_t ldc, const T* __restrict__ S, int64_t lds, int n,
                                  int kp, int NT, int KS, typename Pair<T>::type* __restrict__ tab) {
  using P2 = typename Pair<T>::type;
  __shared__ P2 tile[32][33];
  const int t0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += blockDim.y) {
    const int l = l0 + i, t = t0 + tx;
    const int j = t - 2 * l - 1;
    P2 v;
    v.x = T(1);
    v.y = T(0);
    if (l < kp && j >= 0 && j <= n - 2) {
      v.x = C[j + (int64_t)l * ldc];
      v.y = S[j + (int64_t)l * lds];
    }
    tile[i][tx] = v;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {
    const int t = t0 + i, l = l0 + tx;
    if (t < NT && l < KS) tab[(int64_t)t * KS + l] = tile[tx][i];
  }
}

template <typename P2, int SPL>
__device__ __forceinline__ void load_pairs(const P2* p, P2 (&cs)[SPL]) {
  if constexpr (sizeof(P2) == 8 && SPL % 2 == 0) {
#pragma unroll
    for (int s = 0; s < SPL; s += 2) {
      const float4 v = *reinterpret_cast<const float4*>(p + s);
      cs[s].x = v.x; cs[s].y = v.y;
      cs[s + 1].x = v.z; cs[s + 1].y = v.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < SPL; ++s) cs[s] = p[s];
  }
}

template <typename T, int SPL, int R>
struct PipeState {
  T carry[SPL][R];                     // column each stage carries
  T prev[SPL > 1 ? SPL - 1 : 1][R];    // stage s's last output, stage s+1's next input
  T last[R];                           // the lane's last stage's output
};

// RN(a*b): FMUL in FP32 (an FFMA with a freshly computed -0 addend measured
// no faster there: 2.744 ms against 2.733 at 8192 x 8192, k = 192); in FP64 a
// DFMA with a freshly computed -0 addend (bit-identical, and issued faster
// than DMUL on GB300; see mul_as_fma).
__device__ __forceinline__ float mul_rn(float a, float b, float) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b, double nz) { return mul_as_fma(a, b, nz); }
__device__ __forceinline__ float neg_zero_for(float) { return -0.0f; }
__device__ __forceinline__ double neg_zero_for(double s) { return neg_zero_from(s); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// One stage on the group's rows: x' = fma(c, x, RN(s*y)),
// y' = fma(c, y, -RN(s*x)), or (stage without a rotation) the values passed
// through unchanged.
template <typename T, int R, bool FAST>
__device__ __forceinline__ void pipe_stage(T (&carry)[R], const T (&y)[R], T (&out)[R], T c, T sn, bool on) {
  const T nz = neg_zero_for(sn);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const T x = carry[i];
    if (FAST || on) {
      out[i] = fma_rn(c, x, mul_rn(sn, y[i], nz));
      carry[i] = fma_rn(c, y[i], -mul_rn(sn, x, nz));
    } else {
      out[i] = x;
      carry[i] = y[i];
    }
  }
}

// 16 bytes of a staging slot (one 128-bit shared-memory access).
template <typename T>
struct alignas(16) Chunk {
  T e[16 / sizeof(T)];
};

// Load R elements of group g from chunk slots of column q (the group's
// first lane then uses them as stage 0's input).
template <typename T, int SPL, int G, int R>
__device__ __forceinline__ void read_group(const T* buf, int q, int g, T (&v)[R]) {
  using PC = Pipe<T, SPL, G, R>;
#pragma unroll
  for (int c = 0; c < PC::CPG; ++c) {
    const Chunk<T> x = *reinterpret_cast<const Chunk<T>*>(buf + chunk_at<PC::NCH>(q, g * PC::CPG + c) * PC::EPC);
#pragma unroll
    for (int e = 0; e < PC::EPC; ++e)
      if (c * PC::EPC + e < R) v[c * PC::EPC + e < R ? c * PC::EPC + e : 0] = x.e[e];
  }
}

template <typename T, int SPL, int G, int R>
__device__ __forceinline__ void write_group(T* buf, int q, int g, const T (&v)[R]) {
  using PC = Pipe<T, SPL, G, R>;
#pragma unroll
  for (int c = 0; c < PC::CPG; ++c) {
    Chunk<T> x;
#pragma unroll
    for (int e = 0; e < PC::EPC; ++e) {
      const int i = c * PC::EPC + e;
      x.e[e] = i < R ? v[i < R ? i : 0] : T(0);
    }
    *reinterpret_cast<Chunk<T>*>(buf + chunk_at<PC::NCH>(q, g * PC::CPG + c) * PC::EPC) = x;
  }
}

// 16 bytes into shared memory, stored only where `on` holds: a predicated
// store, so the warp takes no branch around the group's last lane.
__device__ __forceinline__ void st_shared_if(float* p, const Chunk<float>& x, bool on) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n @q st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n}\n"
               ::"r"(smem_u32(p)), "f"(x.e[0]), "f"(x.e[1]), "f"(x.e[2]), "f"(x.e[3]), "r"((int)on) : "memory");
}
__device__ __forceinline__ void st_shared_if(double* p, const Chunk<double>& x, bool on) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n @q st.shared.v2.f64 [%0], {%1, %2};\n}\n"
               ::"r"(smem_u32(p)), "d"(x.e[0]), "d"(x.e[1]), "r"((int)on) : "memory");
}

// write_group by the lanes where `on` holds (every lane computes the slots).
template <typename T, int SPL, int G, int R>
__device__ __forceinline__ void write_group_if(T* buf, int q, int g, const T (&v)[R], bool on) {
  using PC = Pipe<T, SPL, G, R>;
#pragma unroll
  for (int c = 0; c < PC::CPG; ++c) {
    Chunk<T> x;
#pragma unroll
    for (int e = 0; e < PC::EPC; ++e) {
      const int i = c * PC::EPC + e;
      x.e[e] = i < R ? v[i < R ? i : 0] : T(0);
    }
    st_shared_if(buf + chunk_at<PC::NCH>(q, g * PC::CPG + c) * PC::EPC, x, on);
  }
}

template <typename T>
constexpr bool kLateSelect = sizeof(T) == 4;

// One step t = t0 + u.  cs / in: this step's pairs and stage-0 input;
// ncs / nin receive the next step's (the pairs from shared memory, the
// input as the shuffle of this step's last-stage output, for a group's
// first lane column nq of nin_buf).  The lane's last stage runs first, so
// the shuffles overlap the other stages.  FAST: every stage of every lane
// has its rotation.
//
// FP32 (kLateSelect): the group's last lane stores its output with a
// predicated store instead of a branch, and the first lane's choice of its
// next input comes last, after the shuffle and shared-memory results have
// arrived (with four steps per iteration, 2.93 -> 2.73 ms at 8192 x 8192,
// k = 192).  FP64 keeps the branch and the early choice: the late form
// made k = 16 slower by 1.5 %.
template <typename T, int SPL, int G, int R, bool FAST>
__device__ __forceinline__ void pipe_step(PipeState<T, SPL, R>& st, const typename Pair<T>::type (&cs)[SPL],
                                          const T (&in)[R], typename Pair<T>::type (&ncs)[SPL], T (&nin)[R],
                                          bool load_next, const typename Pair<T>::type* ncs_src, const T* nin_buf,
                                          int nq, T* outb, int u, int t, int n, int kp, int g, int pl) {
  using PC = Pipe<T, SPL, G, R>;
  if (load_next) load_pairs<typename PC::P2, SPL>(ncs_src, ncs);
  T nv[R];
  read_group<T, SPL, G, R>(nin_buf, nq, g, nv);
  bool on[SPL];
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    on[s] = true;
    if (!FAST) {
      const int l = SPL * pl + s;
      on[s] = l < kp && (unsigned)(t - 2 * l - 1) <= (unsigned)(n - 2);
    }
  }
  if constexpr (SPL > 1)
    pipe_stage<T, R, FAST>(st.carry[SPL - 1], st.prev[SPL - 2], st.last, cs[SPL - 1].x, cs[SPL - 1].y, on[SPL - 1]);
  else
    pipe_stage<T, R, FAST>(st.carry[0], in, st.last, cs[0].x, cs[0].y, on[0]);
#pragma unroll
  for (int i = 0; i < R; ++i) nin[i] = __shfl_up_sync(0xffffffffu, st.last[i], 1, PC::LPG);
  if constexpr (!kLateSelect<T>) {
    if (pl == 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) nin[i] = nv[i];
    }
  }
  // Then stage SPL-2 down to 0: stage s reads stage s-1's output of the
  // previous step before stage s-1 replaces it.
#pragma unroll
  for (int s = SPL - 2; s >= 1; --s)
    pipe_stage<T, R, FAST>(st.carry[s], st.prev[s - 1], st.prev[s], cs[s].x, cs[s].y, on[s]);
  if constexpr (SPL > 1) pipe_stage<T, R, FAST>(st.carry[0], in, st.prev[0], cs[0].x, cs[0].y, on[0]);
  if constexpr (kLateSelect<T>) {
    write_group_if<T, SPL, G, R>(outb, u, g, st.last, pl == PC::LPG - 1);
#pragma unroll
    for (int i = 0; i < R; ++i) nin[i] = pl == 0 ? nv[i] : nin[i];
  } else {
    if (pl == PC::LPG - 1) write_group<T, SPL, G, R>(outb, u, g, st.last);
  }
}

// 32 steps t0 .. t0+31, the current and next registers trading places
// every step (no copies): four steps per iteration in FP32, two in FP64 (at
// 8192 x 8192, four made FP32 6 % faster and FP64 at k = 8 3 % slower).
// cst: this lane's pairs of the tile's first step (shared memory); inb /
// inb_next: this tile's and the next tile's input columns; in: stage 0's
// input of step t0, on return that of step t0 + 32.
template <typename T, int SPL, int G, int R, bool FAST>
__device__ __forceinline__ void pipe_tile(PipeState<T, SPL, R>& st, T (&in)[R], const T* inb, const T* inb_next,
                                          T* outb, const typename Pair<T>::type* cst, int t0, int n, int kp, int g,
                                          int pl) {
  using PC = Pipe<T, SPL, G, R>;
  constexpr int KS = PC::KS;
  typename PC::P2 csA[SPL], csB[SPL];
  T inB[R];
  load_pairs<typename PC::P2, SPL>(cst, csA);
  if constexpr (sizeof(T) == 4) {
#pragma unroll 1
    for (int u = 0; u < kPTC; u += 4) {
      pipe_step<T, SPL, G, R, FAST>(st, csA, in, csB, inB, true, cst + (u + 1) * KS, inb, u + 1, outb, u, t0 + u, n,
                                    kp, g, pl);
      pipe_step<T, SPL, G, R, FAST>(st, csB, inB, csA, in, true, cst + (u + 2) * KS, inb, u + 2, outb, u + 1,
                                    t0 + u + 1, n, kp, g, pl);
      pipe_step<T, SPL, G, R, FAST>(st, csA, in, csB, inB, true, cst + (u + 3) * KS, inb, u + 3, outb, u + 2,
                                    t0 + u + 2, n, kp, g, pl);
      const bool end = u + 4 >= kPTC;
      pipe_step<T, SPL, G, R, FAST>(st, csB, inB, csA, in, !end, cst + (u + 4) * KS, end ? inb_next : inb,
                                    (u + 4) & (kPTC - 1), outb, u + 3, t0 + u + 3, n, kp, g, pl);
    }
  } else {
#pragma unroll 1
    for (int u = 0; u < kPTC; u += 2) {
      pipe_step<T, SPL, G, R, FAST>(st, csA, in, csB, inB, true, cst + (u + 1) * KS, inb, u + 1, outb, u, t0 + u, n,
                                    kp, g, pl);
      const bool end = u + 2 >= kPTC;
      pipe_step<T, SPL, G, R, FAST>(st, csB, inB, csA, in, !end, cst + (u + 2) * KS, end ? inb_next : inb,
                                    (u + 2) & (kPTC - 1), outb, u + 1, t0 + u + 1, n, kp, g, pl);
    }
  }
}

// One CTA: W warps of G*R rows each, in step with each other; the (c,s)
// table flows through NS shared tiles (one bulk copy per 32 steps, bounded
// waits).
template <typename T, int SPL, int G, int R, int W>
__global__ void __launch_bounds__(W * 32)
pipe_kernel(const typename Pair<T>::type* __restrict__ tab, int NT, T* __restrict__ A, int64_t lda, int m, int n,
            int kp, int* status) {
  using PC = Pipe<T, SPL, G, R, W>;
  using P2 = typename PC::P2;
  constexpr int KS = PC::KS, NS = PC::NS, ROWS = PC::ROWS, SLOT = PC::SLOT;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * PC::kTabBytes + W * PC::kWarpElems * sizeof(T));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = lane / PC::LPG, pl = lane % PC::LPG;
  const int r0 = (blockIdx.x * W + wid) * ROWS;
  const bool active = r0 < m;                   // idle warps still take part in the barriers
  const int nrow = active ? min(ROWS, m - r0) : 0;
  T* wb = reinterpret_cast<T*>(smem + NS * PC::kTabBytes) + wid * PC::kWarpElems;
  // wb: input tiles 0 and 1, then the output tile.
  T* const outb = wb + 2 * kPTC * SLOT;
  T* const Ar = A + r0;
  const int ntiles = (NT + kPTC - 1) / kPTC;

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  auto issue = [&](int Tn) {
    const int s = Tn % NS;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[s], PC::kTabBytes);
    bulk_g2s(smem + s * PC::kTabBytes, tab + (int64_t)Tn * kPTC * KS, PC::kTabBytes, &bar[s]);
  };
  if (tid == 0)
    for (int Tn = 0; Tn < NS && Tn < ntiles; ++Tn) issue(Tn);

  // Column q of the warp's rows (zeros past the matrix), staged by this
  // lane as column `lane` of a tile.
  auto load_col = [&](int q, T (&v)[ROWS]) {
#pragma unroll
    for (int i = 0; i < ROWS; ++i) v[i] = (q < n && i < nrow) ? Ar[(int64_t)q * lda + i] : T(0);
  };
  auto stage_col = [&](T* buf, const T (&v)[ROWS]) {
#pragma unroll
    for (int gg = 0; gg < G; ++gg) {
      T part[R];
#pragma unroll
      for (int i = 0; i < R; ++i) part[i] = v[gg * R + i];
      write_group<T, SPL, G, R>(buf, lane, gg, part);
    }
  };
  T pf[ROWS];
  load_col(lane, pf);
  stage_col(wb, pf);
  load_col(kPTC + lane, pf);

  PipeState<T, SPL, R> st;
  T in[R];                                       // stage 0's input of the coming step
  {
    T c0[R];                                     // column 0 of the group's rows
#pragma unroll
    for (int i = 0; i < R; ++i) c0[i] = (n > 0 && g * R + i < nrow) ? Ar[g * R + i] : T(0);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      in[i] = pl == 0 ? c0[i] : T(0);
      st.last[i] = T(0);
#pragma unroll
      for (int s = 0; s < SPL; ++s) st.carry[s][i] = T(0);
#pragma unroll
      for (int s = 0; s < (SPL > 1 ? SPL - 1 : 1); ++s) st.prev[s][i] = T(0);
    }
  }
  int Ti = 0;
  for (; Ti < ntiles; ++Ti) {
    // The next tile's columns go to the other buffer; the one after is fetched.
    stage_col(wb + ((Ti + 1) & 1) * kPTC * SLOT, pf);
    load_col(kPTC * (Ti + 2) + lane, pf);
    const int s = Ti % NS;
    bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(Ti / NS) & 1u);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) set_error(status, kDevTimeoutTma);
      break;
    }
    const int t0 = kPTC * Ti;
    const P2* cst = reinterpret_cast<const P2*>(smem + s * PC::kTabBytes) + SPL * pl;
    T* inb = wb + (Ti & 1) * kPTC * SLOT;
    T* inb_next = wb + ((Ti + 1) & 1) * kPTC * SLOT;
    if (active) {
      if (kp == KS && t0 >= 2 * KS - 1 && t0 + kPTC - 1 <= n - 1)
        pipe_tile<T, SPL, G, R, true>(st, in, inb, inb_next, outb, cst, t0, n, kp, g, pl);
      else
        pipe_tile<T, SPL, G, R, false>(st, in, inb, inb_next, outb, cst, t0, n, kp, g, pl);
    }
    __syncthreads();                             // stage s read by every warp; outputs complete
    if (tid == 0 && Ti + NS < ntiles) issue(Ti + NS);
    // The groups' last lanes emitted columns t - 2KS + 1 of this tile's steps.
    const int q = t0 + lane - 2 * KS + 1;
    if (active && q >= 0 && q < n) {
      T* dst = Ar + (int64_t)q * lda;
#pragma unroll
      for (int gg = 0; gg < G; ++gg) {
        T v[R];
        read_group<T, SPL, G, R>(outb, lane, gg, v);
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (gg * R + i < nrow) dst[gg * R + i] = v[i];
      }
    }
  }
  // On a timeout, let the copies still in flight (tiles Ti .. Ti+NS-1) land
  // before leaving.
  if (Ti < ntiles && tid == 0)
    for (int r = Ti; r < ntiles && r < Ti + NS; ++r) (void)mbar_wait_bounded(&bar[r % NS], (uint32_t)(r / NS) & 1u);
}

template <typename T, int SPL, int G, int R, int W = 4>
cudaError_t launch_pipe(const typename Pair<T>::type* tab, int NT, T* A, int64_t lda, int m, int n, int kp,
                        int* status, cudaStream_t s) {
  using PC = Pipe<T, SPL, G, R, W>;
  const int rows = W * PC::ROWS;
  auto kfn = pipe_kernel<T, SPL, G, R, W>;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(kfn), PC::kSmem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)((m + rows - 1) / rows), W * 32, PC::kSmem, s>>>(tab, NT, A, lda, m, n, kp, status);
  return cudaGetLastError();
}

// Scratch of a pipelined call: the widest pass's table (whole 32-step
// tiles) and a status word.
template <typename T>
struct PipeScratch {
  void* base = nullptr;
  typename Pair<T>::type* tab = nullptr;
  int* status = nullptr;
};

template <typename T>
rot_status pipe_scratch(int64_t n, int64_t KSmax, cudaStream_t s, PipeScratch<T>* ps) {
  const int64_t NTmax = (n + 2 * KSmax - 1 + kPTC - 1) / kPTC * kPTC;
  const size_t tab_bytes = (size_t)NTmax * KSmax * sizeof(typename Pair<T>::type);
  if (cudaMallocAsync(&ps->base, tab_bytes + 256, s) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  ps->tab = static_cast<typename Pair<T>::type*>(ps->base);
  ps->status = reinterpret_cast<int*>(static_cast<unsigned char*>(ps->base) + tab_bytes);
  cudaError_t e = cudaMemsetAsync(ps->status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(ps->base, s);
    return cuda_failed(e, "pipe: memset");
  }
  return ROT_OK;
}

// One pass of kp sequences (C, S at their first column) with KS stages per group.
template <typename T>
rot_status pipe_table(int64_t n, int kp, int KS, const T* C, int64_t ldc, const T* S, int64_t lds,
                      const PipeScratch<T>& ps, cudaStream_t s, int* NT) {
  *NT = (int)n + 2 * KS - 1;
  dim3 tg((unsigned)((*NT + 31) / 32), (unsigned)((KS + 31) / 32));
  pipe_table_kernel<T><<<tg, dim3(32, 8), 0, s>>>(C, ldc, S, lds, (int)n, kp, *NT, KS, ps.tab);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROT_OK : cuda_failed(e, "pipe: table kernel");
}

}  // namespace

bool pipe_f32_fits(int64_t m, int64_t n, int64_t k) {
  // At least 20 sequences, over columns well beyond the fill and drain of up
  // to 2 x 192 steps.  (rot_apply_f32 keeps k <= 41 on the column stream
  // where it applies and the matrix has more than 4096 rows: 8192 x 8192,
  // k = 41, 1.78 ms against 1.82.)
  return k >= 20 && n >= 1024 && m >= 1 && m < (int64_t(1) << 31) && n < (int64_t(1) << 30);
}

rot_status pipe_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C, int64_t ldc,
                          const float* S, int64_t lds, cudaStream_t s) {
  // Passes of whole lanes of sequences (32 stages per lane of the group),
  // as even as possible.  The r = k mod 32 left over either fill one more,
  // part-filled lane (its stages past k pass their values through) or run
  // on the column stream afterwards, whichever measured faster.  At
  // 8192 x 8192 a full pass takes 1.34 ms with 32 stages, 1.55 with 64,
  // 1.94 with 96, 2.30 with 128, 2.64 with 160 and 2.87 with 192; a
  // part-filled one costs more the wider it is (64: +17 %, 96: +29 %, 160
  // and 192: +35 %: its tiles take every stage's predicate at every step);
  // the stream takes about 0.3 ms per 8 sequences.  So one more lane when
  // r reaches kRoundUp[u] after u whole lanes (k = 95: 2.53 ms, against 3.0
  // with 31 on the stream; k = 42..63: 1.82 against up to 2.69), the stream
  // otherwise (k = 65: 1.79 ms, against 2.53 as a part-filled pass of 96),
  // and never past six lanes, where the extra lane would start a second
  // pass.  With no whole lane (20 <= k < 32, few rows) the one pass is
  // part-filled.  Each pass applies its sequences entirely before the next, as
  // Algorithm 2 does.
  // Seven rows per warp: 8192 rows then make 1171 warps, 1.93 per SM
  // subpartition of a GB300 (eight rows: 1.68, so the busiest subpartitions
  // would carry two warps of 8 rows while others idle).
  constexpr int R = 7;
  // r needed after u whole lanes (33: never); below one lane, only where
  // rot_apply_f32 sends k >= 20 here (up to 4096 rows)
  constexpr int kRoundUp[6] = {20, 10, 22, 25, 29, 30};
  const int64_t r = k % 32, u = k / 32;
  // With few rows the stream is relatively slower, so after one lane the
  // part-filled pass pays from r = 7 (4096 x 4096, k = 39: 0.64 ms against
  // 0.71 as 32 stages and 7 on the stream).
  const int r_min = (u == 1 && m <= 4096) ? 7 : (u < 6 ? kRoundUp[u] : 33);
  const bool round_up = r >= r_min;
  const int64_t units = k / 32 + (round_up ? 1 : 0);
  const int64_t kpipe = round_up ? k : k - r;                 // sequences the passes apply
  const int64_t npass = (units + kPMaxSpl - 1) / kPMaxSpl;
  const int64_t KSmax = 32 * ((units + npass - 1) / npass);              // stages of the widest pass
  PipeScratch<float> ps;
  rot_status st = pipe_scratch<float>(n, KSmax, s, &ps);
  if (st != ROT_OK) return st;
  int64_t p0 = 0;
  for (int64_t gi = 0; gi < npass && st == ROT_OK; ++gi) {
    const int64_t left = units - p0 / 32;                     // lanes of sequences still to apply
    const int spl = (int)((left + (npass - gi) - 1) / (npass - gi));
    const int KS = 32 * spl;
    const int kp = (int)std::min<int64_t>(KS, kpipe - p0);    // short only in the last pass
    int NT = 0;
    st = pipe_table<float>(n, kp, KS, C + p0 * ldc, ldc, S + p0 * lds, lds, ps, s, &NT);
    if (st != ROT_OK) break;
    const int tr = trace_begin(ROT_KERNEL_PIPE_F32, m * (n - 1) * kp, s);
    cudaError_t e;
    switch (spl) {
      case 1: e = launch_pipe<float, 1, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
      case 2: e = launch_pipe<float, 2, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
      case 3: e = launch_pipe<float, 3, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
      case 4: e = launch_pipe<float, 4, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
      case 5: e = launch_pipe<float, 5, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
      default: e = launch_pipe<float, 6, 1, R>(ps.tab, NT, A, lda, (int)m, (int)n, kp, ps.status, s); break;
    }
    trace_end(tr, s);
    if (e != cudaSuccess) { st = cuda_failed(e, "pipe_f32: kernel launch"); break; }
    count_launches(2);
    p0 += kp;
  }
  if (st == ROT_OK) record_status_async(ps.status, s);
  cudaFreeAsync(ps.base, s);
  if (st != ROT_OK || p0 == k) return st;
  if (stream_fits<float>(m, n, k - p0, A, lda))
    return stream_apply<float>(m, n, k - p0, A, lda, C + p0 * ldc, ldc, S + p0 * lds, lds, s);
  return wave_apply_f32(m, n, k - p0, A, lda, C + p0 * ldc, ldc, S + p0 * lds, lds, s, WaveOptions{});
}

// SMs of the current device (0 if it cannot be read).
static int device_sms() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nsm;
}

rot_status apply_f64(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C, int64_t ldc,
                     const double* S, int64_t lds, cudaStream_t s) {
  // The split column stream (passes of up to 4 sequences, two warps a
  // sequence per 32-row strip) while its strips fit one CTA per SM (each
  // chain then waits only on its own latency), or for three sequences with
  // two strips per SM.  Measured against the lane pipeline (rot_apply, the
  // same box, median of 5 calls): k = 3..8 at 4096 x 4096 0.81-1.59 ms
  // against 1.18-1.83, at 1024 x 8192 1.48-3.02 against 2.05-3.35; k = 3 at
  // 8192 x 8192 1.92 against 2.37, at 6144 x 6144 1.47 against 1.78.  With
  // two strips per SM from k = 4 on the pipeline is ahead (8192 x 8192,
  // k = 4: 2.42 against 2.38; k = 8: 4.73 against 4.02).
  const int64_t strips = (m + 31) / 32;
  const int64_t nsm = device_sms();
  if (stream_fits<double>(m, n, k, A, lda) && ((k <= 8 && strips <= nsm) || (k == 3 && strips <= 2 * nsm)))
    return stream_apply<double>(m, n, k, A, lda, C, ldc, S, lds, s);
  if (pipe_f64_fits(m, n, k)) return pipe_apply_f64(m, n, k, A, lda, C, ldc, S, lds, s);
  if (stream_fits<double>(m, n, k, A, lda)) return stream_apply<double>(m, n, k, A, lda, C, ldc, S, lds, s);
  // The wavefront kernel, with the tiling the autotuner recorded for this
  // shape (rot_batch_autotune on a batch of this one problem), else the
  // defaults (p-blocks as long as the resident warps allow, wave_apply).
  // Above 32 sequences it beats the lane pipeline in chunks of 32 nearly
  // everywhere (2048 x 2048, k = 64: 3.37 ms against 4.68; 8192 x 8192,
  // k = 33: 15.0 against 16.5).
  rot_problem p{m, n, k, A, lda, C, ldc, S, lds};
  rot_tuning tu{};
  tuning_lookup(1, &p, &tu);
  WaveOptions o{};
  o.K = tu.K;
  o.NB = tu.NB;
  o.ctas_per_sm = tu.ctas_per_sm;
  o.fp64_products = tu.fp64_products;
  return wave_apply<double>(m, n, k, A, lda, C, ldc, S, lds, s, o);
}

bool pipe_f64_fits(int64_t m, int64_t n, int64_t k) {
  return k >= 3 && k <= 32 && n >= 256 && m >= 1 && m < (int64_t(1) << 31) && n < (int64_t(1) << 30);
}

// FP64 passes for k sequences: the stages per group and the sequences of
// each lane-pipeline pass (np of them, at most 3), and the sequences left to
// the split column stream at the end (tail, at most 7).
struct PipePlan64 {
  int np = 0;
  int KS[4] = {0, 0, 0, 0};
  int kp[4] = {0, 0, 0, 0};
  int tail = 0;
};

static PipePlan64 pipe_f64_plan(int64_t m, int64_t k, bool tail_ok, int64_t nsm) {
  // Every lane holds one stage, so a pass costs its KS (a power of two from
  // 4 to 32) whatever the sequences it applies, and a pass short of its KS
  // more (its stages past k pass values through: 4096 x 4096, KS = 32 with
  // 21..31 sequences 5.33 ms, with 32 4.55).
  PipePlan64 p;
  auto pass = [&](int KS, int64_t kp) {
    p.KS[p.np] = KS;
    p.kp[p.np] = (int)kp;
    ++p.np;
  };
  const int64_t strips = (m + 31) / 32;
  if (tail_ok && nsm > 0 && strips <= nsm) {
    // At most one 32-row strip per SM: the split stream takes up to 7
    // sequences for less than a pass of 8 (4096 x 4096: 5..7 in 1.42-1.55
    // ms, a pass of 8 1.76; 4864 x 8192: 2.67-2.94 against 3.34).  So full
    // passes of 8, 16 and 32 for the multiple of 8, the rest on the stream.
    // From 29 sequences on and up to 4096 rows one pass of 32 short of its
    // stages is cheaper (4096 x 4096: 5.34 ms against 5.96-6.11 for
    // k = 29..31; 2048 x 2048: 2.77 against 3.02-3.08), with more rows it is
    // not (4864 x 8192: 15.6 against 11.7-12.0).
    if (k >= 29 && m <= 4096) {
      pass(32, k);
      return p;
    }
    const int64_t q = k / 8 * 8;
    for (int b = 32; b >= 8; b /= 2)
      if (q & b) pass(b, b);
    p.tail = (int)(k - q);
    return p;
  }
  // Otherwise the FP64 units bound every pass (8192 x 8192: KS = 4, 8, 16, 32
  // take 2.37, 4.01, 7.79, 15.3 ms) and k runs as passes of powers of two
  // from 32 down to 4 (the binary digits of k rounded up to a multiple of 4),
  // the last one short by that rounding.  A remainder of 1 (k = 4j + 1) or,
  // past a pass of 8, of 2 goes to the split stream (1.25 and 1.60 ms), and
  // one of 3 too while there are at most two strips per SM (1.92 ms, where
  // strips run in several rounds it is slower than a pass of 4).
  if (tail_ok) {
    if (k % 4 == 1) p.tail = 1;
    else if (k >= 10 && k % 8 == 2) p.tail = 2;
    else if (k >= 10 && k % 8 == 3 && nsm > 0 && strips <= 2 * nsm) p.tail = 3;
  }
  const int64_t kt = k - p.tail;
  const int64_t q = (kt + 3) / 4 * 4;
  for (int b = 32; b >= 4; b /= 2)
    if (q & b) pass(b, b);
  if (p.np > 0) p.kp[p.np - 1] -= (int)(q - kt);
  return p;
}

rot_status pipe_apply_f64(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C, int64_t ldc,
                          const double* S, int64_t lds, cudaStream_t s) {
  // Passes (pipe_f64_plan), each applying its sequences entirely before
  // the next, as Algorithm 2 does.  Every lane holds one stage of a group
  // of KS lanes (stages past a pass's sequences pass their values through),
  // 32/KS groups per warp, about 8 rows per warp.  Up to 16 stages a CTA is
  // one warp: 8192 rows then make 1024 CTAs, at most 7 (56 rows) per SM
  // where 4-warp CTAs put 64 rows on some SMs and 32 on others, and the
  // SM's FP64 unit takes time in proportion to its rows (k = 8: 4.86 ->
  // 4.09 ms, k = 16: 9.33 -> 8.04 ms at 8192 x 8192).  At 32 stages the
  // table tiles leave room for only 4 one-warp CTAs per SM (18.4 ms against
  // 16.3).  The plan leaves up to 7 sequences to the split column stream
  // where it applies (A 16-byte aligned, an even lda, m and n >= 64).
  const PipePlan64 plan = pipe_f64_plan(m, k, stream_fits<double>(m, n, 4, A, lda), device_sms());
  const int np = plan.np;
  const int* KS = plan.KS;
  const int* kp = plan.kp;
  int64_t p0 = 0;
  rot_status st = ROT_OK;
  if (np > 0) {
    PipeScratch<double> ps;
    st = pipe_scratch<double>(n, KS[0], s, &ps);
    if (st != ROT_OK) return st;
    for (int i = 0; i < np && st == ROT_OK; ++i) {
      int NT = 0;
      st = pipe_table<double>(n, kp[i], KS[i], C + p0 * ldc, ldc, S + p0 * lds, lds, ps, s, &NT);
      if (st != ROT_OK) break;
      const int tr = trace_begin(ROT_KERNEL_PIPE_F64, m * (n - 1) * kp[i], s);
      cudaError_t e;
      switch (KS[i]) {
        case 4: e = launch_pipe<double, 1, 8, 1, 1>(ps.tab, NT, A, lda, (int)m, (int)n, kp[i], ps.status, s); break;
        case 8: e = launch_pipe<double, 1, 4, 2, 1>(ps.tab, NT, A, lda, (int)m, (int)n, kp[i], ps.status, s); break;
        case 16: e = launch_pipe<double, 1, 2, 4, 1>(ps.tab, NT, A, lda, (int)m, (int)n, kp[i], ps.status, s); break;
        default: e = launch_pipe<double, 1, 1, 7, 4>(ps.tab, NT, A, lda, (int)m, (int)n, kp[i], ps.status, s); break;
      }
      trace_end(tr, s);
      if (e != cudaSuccess) { st = cuda_failed(e, "pipe_f64: kernel launch"); break; }
      count_launches(2);
      p0 += kp[i];
    }
    if (st == ROT_OK) record_status_async(ps.status, s);
    cudaFreeAsync(ps.base, s);
  }
  if (st != ROT_OK || plan.tail == 0) return st;
  return stream_apply<double>(m, n, plan.tail, A, lda, C + p0 * ldc, ldc, S + p0 * lds, lds, s);
}

}  // namespace rs
