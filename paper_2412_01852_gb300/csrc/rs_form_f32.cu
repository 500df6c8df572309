// rs_form_f32.cu -- the accumulated blocks of rs_gemm (Section 8) formed in
// FP32 as a systolic pipeline across the lanes of a warp.
//
// A row of Q_b starts as a unit vector and passes, column by column, through
// the block's kb sequences.  One sequence's sweep over a row needs one value
// of state (the running column of Algorithm 1's pair (j, j+1)): it takes in
// column q, rotates it with the carried column q-1, emits column q-1 and
// carries the new column q.  So the sequences form a pipeline: sequence l
// works on column t - 2l at step t, its output reaching sequence l+1 one
// step later.  Each rotation sees the same two operands as in Algorithm 2
// (the same dependency order per element), so the result equals the
// sequential FP32 block, except that rotations outside the block act as
// (c,s) = (1,0) and may change the sign of a zero.
//
// Lane i holds sequences spl*i .. spl*i + spl - 1 (KS = 32 spl stages; those
// past kb are (1,0) too); a warp runs 8 rows of Q_b through the pipeline in
// step, a shuffle handing each row's value from lane to lane.  The (c,s) of
// step t are one row of a per-block table (every lane reads its own spl
// pairs), written beforehand with (1,0) wherever the block has no rotation.
// A warp starts at the step of its first row's unit entry: before it, every
// value in its pipeline is zero.
//
// Work at 8192 x 8192, k = 192, nb = 256, kb = 64 (99 blocks of 320 x 320):
// about 1.1 M warp-steps of 16 rotations on 8 rows.
#include <cuda_runtime.h>

#include "rs_form_f32.h"

namespace rs {
namespace {

constexpr int kRows = 8;        // rows of Q_b per warp
constexpr int kWarps = 4;       // warps per CTA
constexpr int kTabRows = 4;     // table steps per thread row of the table kernel

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// table[b][t][l] = (c, s) of rotation (j, p) = (c0 + t - 2l - 1, p0 + l) of
// block b when it exists in the block (l < kbe, wave t - l - 1 in
// [kb - 1, kb - 1 + nb), 0 <= j <= n - 2), else (1, 0).  Also c0 per block.
__global__ void form32_table_kernel(const double* __restrict__ C, int64_t ldc, const double* __restrict__ S,
                                    int64_t lds, int n, int k, int nb, int kb, int NT, int KS,
                                    float2* __restrict__ tab, int* __restrict__ c0s) {
  const int b = blockIdx.y;
  int c0, p0, kbe;
  block_at(b, n, k, nb, kb, &c0, &p0, &kbe);
  const int l = threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.y == 0 && l == 0) c0s[b] = c0;
  const int t_lo = (blockIdx.x * blockDim.y + threadIdx.y) * kTabRows;
  float2* row = tab + ((int64_t)b * NT) * KS + l;
#pragma unroll
  for (int i = 0; i < kTabRows; ++i) {
    const int t = t_lo + i;
    if (t >= NT) break;
    const int j = c0 + t - 2 * l - 1;
    const int u = t - l - kb;
    float2 v = make_float2(1.0f, 0.0f);
    if (l < kbe && u >= 0 && u < nb && j >= 0 && j <= n - 2) {
      v.x = __double2float_rn(C[j + (int64_t)(p0 + l) * ldc]);
      v.y = __double2float_rn(S[j + (int64_t)(p0 + l) * lds]);
    }
    row[(int64_t)t * KS] = v;
  }
}

template <int SPL>
__device__ __forceinline__ void load_pairs(const float2* p, float2 (&cs)[SPL]) {
  if constexpr (SPL % 2 == 0) {
#pragma unroll
    for (int s = 0; s < SPL; s += 2) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + s));
      cs[s] = make_float2(v.x, v.y);
      cs[s + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int s = 0; s < SPL; ++s) cs[s] = __ldg(p + s);
  }
}

__device__ __forceinline__ void store_rows(float* dst, const float (&v)[kRows]) {
  reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void store_zero_rows(float* dst) {
  const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  reinterpret_cast<float4*>(dst)[0] = z;
  reinterpret_cast<float4*>(dst)[1] = z;
}

template <int SPL>
__global__ void __launch_bounds__(kWarps * 32)
form32_kernel(const float2* __restrict__ tab, int NT, int L, int Lq, float* __restrict__ Q) {
  constexpr int KS = 32 * SPL;
  constexpr int NP = SPL > 1 ? SPL - 1 : 1;
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int r0 = (blockIdx.x * kWarps + (threadIdx.x >> 5)) * kRows;
  if (r0 >= Lq) return;
  float* Qb = Q + (int64_t)b * Lq * Lq + r0;
  if (r0 >= L) {                                 // padding rows
    for (int q = lane; q < Lq; q += 32) store_zero_rows(Qb + (int64_t)q * Lq);
    return;
  }
  // Columns left of the first one this warp's pipeline emits are zero
  // (row r of Q_b is zero left of column r - kb).
  const int qfirst = r0 - 2 * KS + 1;
  for (int q = lane; q < qfirst; q += 32) store_zero_rows(Qb + (int64_t)q * Lq);

  float carry[SPL][kRows], prev[NP][kRows], last[kRows];
#pragma unroll
  for (int i = 0; i < kRows; ++i) {
    last[i] = 0.0f;
#pragma unroll
    for (int s = 0; s < SPL; ++s) carry[s][i] = 0.0f;
#pragma unroll
    for (int s = 0; s < NP; ++s) prev[s][i] = 0.0f;
  }
  const float2* tp = tab + (int64_t)b * NT * KS + SPL * lane + (int64_t)r0 * KS;
  float2 cs[SPL], nx[SPL];
  load_pairs<SPL>(tp, nx);
  for (int t = r0; t < NT; ++t) {
#pragma unroll
    for (int s = 0; s < SPL; ++s) cs[s] = nx[s];
    tp += KS;
    if (t + 1 < NT) load_pairs<SPL>(tp, nx);
    float in[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) in[i] = __shfl_up_sync(0xffffffffu, last[i], 1);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kRows; ++i) in[i] = (t == r0 + i) ? 1.0f : 0.0f;
    }
    // Stages from the last to the first, so that stage s reads stage s-1's
    // output of the previous step.
#pragma unroll
    for (int s = SPL - 1; s >= 0; --s) {
      const float c = cs[s].x, sn = cs[s].y;
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        const float x = carry[s][i];
        const float y = s == 0 ? in[i] : prev[s > 0 ? s - 1 : 0][i];
        const float out = fmaf(c, x, __fmul_rn(sn, y));
        carry[s][i] = fmaf(c, y, -__fmul_rn(sn, x));
        if (s < SPL - 1) prev[s][i] = out;
        else last[i] = out;
      }
    }
    const int q = t - 2 * KS + 1;                // column the last stage emitted
    if (lane == 31 && q >= 0) store_rows(Qb + (int64_t)q * Lq, last);
  }
}

template <int SPL>
cudaError_t launch_form32(const float2* tab, const Form32Layout& F, float* Q, cudaStream_t s) {
  dim3 grid((unsigned)((F.Lq + kWarps * kRows - 1) / (kWarps * kRows)), (unsigned)F.nblk);
  form32_kernel<SPL><<<grid, kWarps * 32, 0, s>>>(tab, F.NT, F.L, F.Lq, Q);
  return cudaGetLastError();
}

}  // namespace

void form32_layout(int64_t n, int64_t k, int nb, int kb, int Lq, Form32Layout* F) {
  const int64_t B0 = (n + kb - 2 + nb - 1) / nb;
  const int64_t G = (k + kb - 1) / kb;
  const int64_t kl = k - (G - 1) * kb;
  F->nblk = (G - 1) * B0 + (n + kl - 2 + nb - 1) / nb;
  F->L = nb + kb;
  F->Lq = Lq;
  F->spl = (kb + 31) / 32;
  F->KS = 32 * F->spl;
  F->NT = Lq + 2 * F->KS - 1;
  F->o_c0 = 0;
  F->o_tab = (size_t)round_up((int64_t)sizeof(int) * F->nblk, 256);
  F->total = F->o_tab + (size_t)round_up((int64_t)F->nblk * F->NT * F->KS * (int64_t)sizeof(float2), 256);
}

rot_status form32_enqueue(int64_t n, int64_t k, const double* C, int64_t ldc, const double* S, int64_t lds,
                          int nb, int kb, const Form32Layout& F, unsigned char* ws, float* Q, cudaStream_t s) {
  if (kb > kForm32MaxKb || F.Lq < F.L || F.Lq % kRows != 0) return ROT_EINVAL;
  float2* tab = reinterpret_cast<float2*>(ws + F.o_tab);
  int* c0s = reinterpret_cast<int*>(ws + F.o_c0);
  const int ty = 256 / F.KS;
  dim3 tb((unsigned)F.KS, (unsigned)ty);
  dim3 tg((unsigned)((F.NT + ty * kTabRows - 1) / (ty * kTabRows)), (unsigned)F.nblk);
  form32_table_kernel<<<tg, tb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, nb, kb, F.NT, F.KS, tab, c0s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks_f32: table kernel");
  // Executed work: every warp of rows r0 .. r0+7 (r0 < L) runs steps
  // r0 .. NT-1 of all KS stages on its 8 rows, padding stages included.
  long long executed = 0;
  for (int r0 = 0; r0 < F.L; r0 += kRows) executed += (long long)(F.NT - r0) * F.KS * kRows;
  const int tr = trace_begin(ROT_KERNEL_FORM_BLOCKS, executed * F.nblk, s);
  switch (F.spl) {
    case 1: e = launch_form32<1>(tab, F, Q, s); break;
    case 2: e = launch_form32<2>(tab, F, Q, s); break;
    case 3: e = launch_form32<3>(tab, F, Q, s); break;
    default: e = launch_form32<4>(tab, F, Q, s); break;
  }
  trace_end(tr, s);
  if (e != cudaSuccess) return cuda_failed(e, "form_blocks_f32: formation kernel");
  count_launches(2);
  return ROT_OK;
}

}  // namespace rs
