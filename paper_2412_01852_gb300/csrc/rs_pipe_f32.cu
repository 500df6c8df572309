// rs_pipe_f32.cu -- FP32 rotations as a pipeline of sequences across the
// lanes of a warp.
//
// One sequence's sweep over a row (Algorithm 2's inner loop) needs a single
// value of state: at column q it rotates the carried column q-1 with the
// incoming column q, emits column q-1 (final for this sequence) and carries
// the new column q.  Sequences p, p+1, ... are therefore stages of a
// pipeline: sequence l works on column t - 2l at step t, and its output
// reaches sequence l+1 one step later.  Each rotation sees the operands it
// sees in Algorithm 2, so the result is bit-exact with the sequential FP32
// loop.
//
// Lane i holds sequences SPL*i .. SPL*i + SPL - 1 (up to 192 per pass); a
// warp streams 7 rows through all n columns, with one shuffle per row and
// step handing each value to the next lane.  Lane 0 takes the columns in,
// lane 31 emits the finished ones; both go through 32-column tiles in shared
// memory that the whole warp loads and stores (the next tile is fetched one
// tile ahead).  The (c,s) of step t are one row of a table in which lane i
// finds its SPL pairs side by side.  Tiles where every stage has a rotation
// run without predicates; at the two ends of the stream a stage without a
// rotation passes its values through unchanged, so zeros keep their sign
// and infinities stay.
//
// Passes of at most 192 sequences (whole lanes of them) apply them in
// Algorithm 2's order, each pass reading and writing A once; fewer than 32
// left over run on the column stream or the wavefront kernel.  The warps of a CTA run in step and share
// the (c,s) table through shared memory: one bulk copy per 32-step tile,
// two or three tiles in flight, waits bounded (a timeout sets the status).
#include <algorithm>
#include <cuda_runtime.h>

#include "rs_device.cuh"
#include "rs_internal.h"

namespace rs {
namespace {

// Rows per warp.  Seven: 8192 rows then make 1171 warps, 1.93 per SM
// subpartition of a GB300 (eight rows: 1.68, so the busiest subpartitions
// carry two warps of 8 rows while others idle).
constexpr int kPR = 7;
constexpr int kPS = 8;        // floats per column in the staging tiles (kPR rows, padded)

// Staging tiles hold column q's rows in 32 bytes at q * 8 floats, the two
// 16-byte halves swapped for q & 4: eight lanes storing or loading their
// columns' halves with 128-bit accesses then hit distinct banks.
__device__ __forceinline__ int half_at(int q, int h) { return q * kPS + 4 * (h ^ ((q >> 2) & 1)); }
constexpr int kPTC = 32;      // steps (columns) per tile
constexpr int kPWarps = 4;    // warps per CTA
constexpr int kPMaxSpl = 6;   // sequences per lane: 192 per pass

// tab[t][l] = (c, s) of rotation (j, p0 + l), j = t - 2l - 1, where
// 0 <= j <= n-2 and l < kp; (1, 0) elsewhere (never used).  32 x 32 tiles
// through shared memory: reads run along j, writes along l.
__global__ void pipe_table_kernel(const float* __restrict__ C, int64_t ldc, const float* __restrict__ S,
                                  int64_t lds, int n, int kp, int NT, int KS, float2* __restrict__ tab) {
  __shared__ float2 tile[32][33];
  const int t0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += blockDim.y) {
    const int l = l0 + i, t = t0 + tx;
    const int j = t - 2 * l - 1;
    float2 v = make_float2(1.0f, 0.0f);
    if (l < kp && j >= 0 && j <= n - 2) v = make_float2(C[j + (int64_t)l * ldc], S[j + (int64_t)l * lds]);
    tile[i][tx] = v;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {
    const int t = t0 + i, l = l0 + tx;
    if (t < NT) tab[(int64_t)t * KS + l] = tile[tx][i];
  }
}

template <int SPL>
struct PipeShape {
  static constexpr int KS = 32 * SPL;                                   // stages
  static constexpr int kTabBytes = kPTC * KS * (int)sizeof(float2);     // (c,s) of one 32-step tile
  static constexpr int NS = SPL >= 4 ? 2 : 3;                           // table tiles in flight
  static constexpr int kWarpFloats = 3 * kPTC * kPS;                    // two input tiles, one output tile
  static constexpr int kSmem = NS * kTabBytes + kPWarps * kWarpFloats * 4 + NS * 8;
};

template <int SPL>
__device__ __forceinline__ void load_pairs(const float2* p, float2 (&cs)[SPL]) {
  if constexpr (SPL % 2 == 0) {
#pragma unroll
    for (int s = 0; s < SPL; s += 2) {
      const float4 v = *reinterpret_cast<const float4*>(p + s);
      cs[s] = make_float2(v.x, v.y);
      cs[s + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int s = 0; s < SPL; ++s) cs[s] = p[s];
  }
}

template <int SPL>
struct PipeState {
  float carry[SPL][kPR];                     // column each stage carries
  float prev[SPL > 1 ? SPL - 1 : 1][kPR];    // stage s's last output, stage s+1's next input
  float last[kPR];                           // the lane's last stage's output
};

// One stage on the warp's rows: rotation, or (stage without one) the
// values passed through unchanged.
template <bool FAST>
__device__ __forceinline__ void pipe_stage(float (&carry)[kPR], const float (&y)[kPR], float (&out)[kPR], float c,
                                           float sn, bool on) {
#pragma unroll
  for (int i = 0; i < kPR; ++i) {
    const float x = carry[i];
    if (FAST || on) {
      out[i] = fmaf(c, x, __fmul_rn(sn, y[i]));
      carry[i] = fmaf(c, y[i], -__fmul_rn(sn, x));
    } else {
      out[i] = x;
      carry[i] = y[i];
    }
  }
}

// One step t = t0 + u.  cs / in: this step's pairs and stage-0 input;
// ncs / nin receive the next step's (the pairs from shared memory, the
// input as the shuffle of this step's last-stage output, for lane 0 column
// nq of nin_buf).  The lane's last stage runs first, so the shuffles overlap
// the other stages.  FAST: every stage of every lane has its rotation.
template <int SPL, bool FAST>
__device__ __forceinline__ void pipe_step(PipeState<SPL>& st, const float2 (&cs)[SPL], const float (&in)[kPR],
                                          float2 (&ncs)[SPL], float (&nin)[kPR], bool load_next,
                                          const float2* ncs_src, const float* nin_buf, int nq, float* outb, int u,
                                          int t, int n, int kp, int lane) {
  if (load_next) load_pairs<SPL>(ncs_src, ncs);
  const float4 na = *reinterpret_cast<const float4*>(nin_buf + half_at(nq, 0));
  const float4 nb = *reinterpret_cast<const float4*>(nin_buf + half_at(nq, 1));
  bool on[SPL];
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    on[s] = true;
    if (!FAST) {
      const int l = SPL * lane + s;
      on[s] = l < kp && (unsigned)(t - 2 * l - 1) <= (unsigned)(n - 2);
    }
  }
  if constexpr (SPL > 1)
    pipe_stage<FAST>(st.carry[SPL - 1], st.prev[SPL - 2], st.last, cs[SPL - 1].x, cs[SPL - 1].y, on[SPL - 1]);
  else
    pipe_stage<FAST>(st.carry[0], in, st.last, cs[0].x, cs[0].y, on[0]);
#pragma unroll
  for (int i = 0; i < kPR; ++i) nin[i] = __shfl_up_sync(0xffffffffu, st.last[i], 1);
  if (lane == 0) {
    const float v[kPS] = {na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w};
#pragma unroll
    for (int i = 0; i < kPR; ++i) nin[i] = v[i];
  }
  // Then stage SPL-2 down to 0: stage s reads stage s-1's output of the
  // previous step before stage s-1 replaces it.
#pragma unroll
  for (int s = SPL - 2; s >= 1; --s)
    pipe_stage<FAST>(st.carry[s], st.prev[s - 1], st.prev[s], cs[s].x, cs[s].y, on[s]);
  if constexpr (SPL > 1) pipe_stage<FAST>(st.carry[0], in, st.prev[0], cs[0].x, cs[0].y, on[0]);
  if (lane == 31) {
    float v[kPS];
#pragma unroll
    for (int i = 0; i < kPS; ++i) v[i] = i < kPR ? st.last[i < kPR ? i : 0] : 0.0f;
    *reinterpret_cast<float4*>(outb + half_at(u, 0)) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(outb + half_at(u, 1)) = make_float4(v[4], v[5], v[6], v[7]);
  }
}

// 32 steps t0 .. t0+31, two per iteration with the current and next
// registers trading places (no copies).  cst: this lane's pairs of the
// tile's first step (shared memory); inb / inb_next: this tile's and the
// next tile's input columns; in: stage 0's input of step t0, on return that
// of step t0 + 32.
template <int SPL, bool FAST>
__device__ __forceinline__ void pipe_tile(PipeState<SPL>& st, float (&in)[kPR], const float* inb,
                                          const float* inb_next, float* outb, const float2* cst, int t0, int n,
                                          int kp, int lane) {
  constexpr int KS = 32 * SPL;
  float2 csA[SPL], csB[SPL];
  float inB[kPR];
  load_pairs<SPL>(cst, csA);
#pragma unroll 1
  for (int u = 0; u < kPTC; u += 2) {
    pipe_step<SPL, FAST>(st, csA, in, csB, inB, true, cst + (u + 1) * KS, inb, u + 1, outb, u, t0 + u, n, kp,
                         lane);
    const bool end = u + 2 >= kPTC;
    pipe_step<SPL, FAST>(st, csB, inB, csA, in, !end, cst + (u + 2) * KS, end ? inb_next : inb,
                         (u + 2) & (kPTC - 1), outb, u + 1, t0 + u + 1, n, kp, lane);
  }
}

// One CTA: kPWarps warps of kPR rows each, in step with each other; the
// (c,s) table flows through NS shared tiles (one bulk copy per 32 steps,
// bounded waits).
template <int SPL>
__global__ void __launch_bounds__(kPWarps * 32)
pipe_f32_kernel(const float2* __restrict__ tab, int NT, float* __restrict__ A, int64_t lda, int m, int n, int kp,
                int* status) {
  using PS = PipeShape<SPL>;
  constexpr int KS = PS::KS, NS = PS::NS;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * PS::kTabBytes + kPWarps * PS::kWarpFloats * 4);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = (blockIdx.x * kPWarps + wid) * kPR;
  const bool active = r0 < m;                   // idle warps still take part in the barriers
  const int nrow = active ? min(kPR, m - r0) : 0;
  float* wb = reinterpret_cast<float*>(smem + NS * PS::kTabBytes) + wid * PS::kWarpFloats;
  // wb: input tiles 0 and 1, then the output tile.
  float* const outb = wb + 2 * kPTC * kPS;
  float* const Ar = A + r0;
  const int ntiles = (NT + kPTC - 1) / kPTC;

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  auto issue = [&](int T) {
    const int s = T % NS;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[s], PS::kTabBytes);
    bulk_g2s(smem + s * PS::kTabBytes, tab + (int64_t)T * kPTC * KS, PS::kTabBytes, &bar[s]);
  };
  if (tid == 0)
    for (int T = 0; T < NS && T < ntiles; ++T) issue(T);

  // Column q of the warp's rows (zeros past the matrix).
  auto load_col = [&](int q, float (&v)[kPR]) {
#pragma unroll
    for (int i = 0; i < kPR; ++i) v[i] = (q < n && i < nrow) ? Ar[(int64_t)q * lda + i] : 0.0f;
  };
  auto stage_col = [&](float* buf, const float (&v)[kPR]) {
    float w[kPS];
#pragma unroll
    for (int i = 0; i < kPS; ++i) w[i] = i < kPR ? v[i < kPR ? i : 0] : 0.0f;
    *reinterpret_cast<float4*>(buf + half_at(lane, 0)) = make_float4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<float4*>(buf + half_at(lane, 1)) = make_float4(w[4], w[5], w[6], w[7]);
  };
  float pf[kPR];
  load_col(lane, pf);
  stage_col(wb, pf);
  float pf0[kPR];                                // column 0, lane 0's first input
  load_col(0, pf0);
  load_col(kPTC + lane, pf);

  PipeState<SPL> st;
  float in[kPR];                                 // stage 0's input of the coming step
#pragma unroll
  for (int i = 0; i < kPR; ++i) {
    in[i] = lane == 0 ? pf0[i] : 0.0f;
    st.last[i] = 0.0f;
#pragma unroll
    for (int s = 0; s < SPL; ++s) st.carry[s][i] = 0.0f;
#pragma unroll
    for (int s = 0; s < (SPL > 1 ? SPL - 1 : 1); ++s) st.prev[s][i] = 0.0f;
  }
  int T = 0;
  for (; T < ntiles; ++T) {
    // The next tile's columns go to the other buffer; the one after is fetched.
    stage_col(wb + ((T + 1) & 1) * kPTC * kPS, pf);
    load_col(kPTC * (T + 2) + lane, pf);
    const int s = T % NS;
    bool ok = mbar_wait_bounded(&bar[s], (uint32_t)(T / NS) & 1u);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) set_error(status, kDevTimeoutTma);
      break;
    }
    const int t0 = kPTC * T;
    const float2* cst = reinterpret_cast<const float2*>(smem + s * PS::kTabBytes) + SPL * lane;
    if (active) {
      if (kp == KS && t0 >= 2 * KS - 1 && t0 + kPTC - 1 <= n - 1)
        pipe_tile<SPL, true>(st, in, wb + (T & 1) * kPTC * kPS, wb + ((T + 1) & 1) * kPTC * kPS, outb, cst, t0, n,
                             kp, lane);
      else
        pipe_tile<SPL, false>(st, in, wb + (T & 1) * kPTC * kPS, wb + ((T + 1) & 1) * kPTC * kPS, outb, cst, t0,
                              n, kp, lane);
    }
    __syncthreads();                             // stage s read by every warp; outputs complete
    if (tid == 0 && T + NS < ntiles) issue(T + NS);
    // Lane 31 emitted columns t - 2KS + 1 of this tile's steps.
    const int q = t0 + lane - 2 * KS + 1;
    if (active && q >= 0 && q < n) {
      const float4 a = *reinterpret_cast<const float4*>(outb + half_at(lane, 0));
      const float4 b = *reinterpret_cast<const float4*>(outb + half_at(lane, 1));
      const float v[kPS] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      float* dst = Ar + (int64_t)q * lda;
#pragma unroll
      for (int i = 0; i < kPR; ++i)
        if (i < nrow) dst[i] = v[i];
    }
  }
  // On a timeout, let the copies still in flight (tiles T .. T+NS-1) land
  // before leaving.
  if (T < ntiles && tid == 0)
    for (int r = T; r < ntiles && r < T + NS; ++r) (void)mbar_wait_bounded(&bar[r % NS], (uint32_t)(r / NS) & 1u);
}

template <int SPL>
cudaError_t launch_pipe(const float2* tab, int NT, float* A, int64_t lda, int m, int n, int kp, int* status,
                        cudaStream_t s) {
  const int rows = kPWarps * kPR;
  auto kfn = pipe_f32_kernel<SPL>;
  cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(kfn), PipeShape<SPL>::kSmem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)((m + rows - 1) / rows), kPWarps * 32, PipeShape<SPL>::kSmem, s>>>(tab, NT, A, lda, m, n, kp,
                                                                                     status);
  return cudaGetLastError();
}

}  // namespace

bool pipe_f32_fits(int64_t m, int64_t n, int64_t k) {
  // Worth it where most tiles run without predicates: at least 32
  // sequences, over columns well beyond the fill and drain of up to
  // 2 x 192 steps.
  return k >= 32 && n >= 1024 && m >= 1 && m < (int64_t(1) << 31) && n < (int64_t(1) << 30);
}

rot_status pipe_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C, int64_t ldc,
                          const float* S, int64_t lds, cudaStream_t s) {
  // The first k32 = 32*floor(k/32) sequences run as passes of whole lanes
  // of sequences, as even as possible (a pass of 32 stages costs almost as
  // much as one of 64); the k - k32 left over follow on the column stream,
  // or the wavefront kernel where the stream does not apply.  Each pass
  // applies its sequences entirely before the next, as Algorithm 2 does.
  const int64_t units = k / 32;
  const int64_t npass = (units + kPMaxSpl - 1) / kPMaxSpl;
  const int64_t KSmax = 32 * ((units + npass - 1) / npass);              // stages of the widest pass
  // The kernel copies whole 32-step tiles of the table; rows past NT are never used.
  const int64_t NTmax = (n + 2 * KSmax - 1 + kPTC - 1) / kPTC * kPTC;
  const size_t tab_bytes = (size_t)NTmax * KSmax * sizeof(float2);
  void* tab = nullptr;
  if (cudaMallocAsync(&tab, tab_bytes + 256, s) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  int* status = reinterpret_cast<int*>(static_cast<unsigned char*>(tab) + tab_bytes);
  rot_status st = ROT_OK;
  cudaError_t e0 = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e0 != cudaSuccess) st = cuda_failed(e0, "pipe_f32: memset");
  int64_t p0 = 0;
  for (int64_t g = 0; g < npass && st == ROT_OK; ++g) {
    const int64_t left = units - p0 / 32;                     // lanes of sequences still to apply
    const int spl = (int)((left + (npass - g) - 1) / (npass - g));
    const int kp = 32 * spl;
    const int KS = 32 * spl;
    const int NT = (int)n + 2 * KS - 1;
    float2* t2 = static_cast<float2*>(tab);
    dim3 tg((unsigned)((NT + 31) / 32), (unsigned)(KS / 32));
    pipe_table_kernel<<<tg, dim3(32, 8), 0, s>>>(C + p0 * ldc, ldc, S + p0 * lds, lds, (int)n, kp, NT, KS, t2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_failed(e, "pipe_f32: table kernel"); break; }
    const int tr = trace_begin(ROT_KERNEL_PIPE_F32, m * (n - 1) * kp, s);
    switch (spl) {
      case 1: e = launch_pipe<1>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
      case 2: e = launch_pipe<2>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
      case 3: e = launch_pipe<3>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
      case 4: e = launch_pipe<4>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
      case 5: e = launch_pipe<5>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
      default: e = launch_pipe<6>(t2, NT, A, lda, (int)m, (int)n, kp, status, s); break;
    }
    trace_end(tr, s);
    if (e != cudaSuccess) { st = cuda_failed(e, "pipe_f32: kernel launch"); break; }
    count_launches(2);
    p0 += kp;
  }
  if (st == ROT_OK) record_status_async(status, s);
  cudaFreeAsync(tab, s);
  if (st != ROT_OK || p0 == k) return st;
  const int64_t r = k - p0;
  if (stream_fits<float>(m, n, r, A, lda))
    return stream_apply<float>(m, n, r, A, lda, C + p0 * ldc, ldc, S + p0 * lds, lds, s);
  return wave_apply_f32(m, n, r, A, lda, C + p0 * ldc, ldc, S + p0 * lds, lds, s, WaveOptions{});
}

}  // namespace rs
