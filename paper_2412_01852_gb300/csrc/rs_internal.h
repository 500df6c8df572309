// rs_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda.h>
#include "../../include/rotseq.h"

namespace rs {

// Per-call overrides of the wavefront kernel's tiling (0 = planner default).
struct WaveOptions {
  int K = 0;              // sequences per p-block (<= the kernel's window KMAX)
  int NB = 0;             // waves per work item
  int ctas_per_sm = 0;    // resident CTAs per SM (<= occupancy limit)
  int fp64_products = 0;  // 0 default, 1 DMUL, 2 integer pipe
  bool reflectors = false; // the pairs are 2x2 reflectors (tau, nu) instead of (c, s)
  const int* arrived = nullptr;  // upload progress flags per chunk of arrive_cols columns (FP64 only)
  int arrive_cols = 0;
  int* last_done = nullptr;      // per wave-block completion counts of the last p-block
  int64_t chain_stride = 0;      // between 32-row strips (0: column-major; packed layout: 32 n)
};

// The FP64 products used when a caller leaves the choice to the library.
// Measured on GB300 (A 8192x8192, k = 192): on the FP64 pipe as DFMAs with a
// -0 addend (value 1) 83.3 ms, as DMUL 90.7 ms, on the integer pipe (value 2)
// 95.7 ms.
constexpr int kDefaultFp64Products = 1;

struct WavePlan {
  int K, NB, delta, nchains, G, B, kpad, cs_rows;
  long long total;
};

// Sequences per p-block of the FP64 wavefront kernel when the caller leaves
// the choice to the library (rs_wave_host.cu).
int wave_default_K_f64(int64_t m, int64_t k, int ctas_per_sm_req);
WavePlan plan_wave(int64_t m, int64_t n, int64_t k, int kmax, int nbt, int K_req, int NB_req,
                   int elem_bytes, int rows_per_chain = 32);

rot_status wave_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C,
                          int64_t ldc, const float* S, int64_t lds, cudaStream_t stream, const WaveOptions& opt);

template <typename T>
rot_status wave_apply(int64_t m, int64_t n, int64_t k, T* A, int64_t lda, const T* C, int64_t ldc,
                      const T* S, int64_t lds, cudaStream_t stream, const WaveOptions& opt);

// The column stream (rs_stream.cu), one pass per 8 sequences: whether it
// takes this problem, and the call.
template <typename T>
bool stream_fits(int64_t m, int64_t n, int64_t k, const T* A, int64_t lda);
// packed: A is in the packed layout (32-row strips; lda is ignored).
template <typename T>
rot_status stream_apply(int64_t m, int64_t n, int64_t k, T* A, int64_t lda, const T* C, int64_t ldc,
                        const T* S, int64_t lds, cudaStream_t stream, bool packed = false);

// FP32 warp chain (rs_chain.cu): whether it takes this problem (16 <= k <=
// 55, A TMA-addressable as for the column stream), and the call.
bool chain_f32_fits(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda);
rot_status chain_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C, int64_t ldc,
                           const float* S, int64_t lds, cudaStream_t stream);

// Rotations as a pipeline of sequences across a warp's lanes (rs_pipe.cu):
// whether it takes this problem, and the call (FP32: k >= 32; FP64:
// 3 <= k <= 32).
bool pipe_f32_fits(int64_t m, int64_t n, int64_t k);
rot_status pipe_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C, int64_t ldc,
                          const float* S, int64_t lds, cudaStream_t stream);
bool pipe_f64_fits(int64_t m, int64_t n, int64_t k);
// rot_apply's choice of FP64 kernel (also rot_apply_left's, on the
// transpose): the lane pipeline for 3 <= k <= 32, the column stream for
// fewer sequences, the wavefront kernel otherwise.
rot_status apply_f64(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C, int64_t ldc,
                     const double* S, int64_t lds, cudaStream_t stream);
rot_status pipe_apply_f64(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C, int64_t ldc,
                          const double* S, int64_t lds, cudaStream_t stream);

bool encode_tile_map_2d(CUtensorMap* map, const void* base, bool is_double, uint64_t inner,
                        uint64_t outer, uint64_t row_pitch_bytes, uint32_t box_inner,
                        uint32_t box_outer);

bool encode_tile_map_2d_b16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                            uint64_t row_pitch_bytes, uint32_t box_inner, uint32_t box_outer);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device): function attributes belong to a
// device's context.
cudaError_t smem_opt_in(const void* kernel, int bytes);

// Record a failed CUDA call for rot_last_error(); returns ROT_ECUDA.
rot_status cuda_failed(cudaError_t e, const char* where);
void note_error(const char* what);

// Launch counting and event tracing (rs_util.cu).
void count_launches(int n);
int trace_begin(int kind, long long work, cudaStream_t s);
void trace_end(int id, cudaStream_t s);

// Autotuner cache (rs_tune.cu): the tiling recorded for a batch of this shape,
// or the defaults.
void tuning_lookup(int count, const rot_problem* problems, rot_tuning* out);

rot_status selftest_dependency_timeout(int wait_ms, cudaStream_t stream, int* device_status);

// Sticky device status (first error recorded by any launch since the last read).
int take_sticky_status();
void record_status_async(const int* status, cudaStream_t stream);

}  // namespace rs
