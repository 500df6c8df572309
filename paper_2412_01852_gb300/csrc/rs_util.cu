// rs_util.cu -- tracing (CUDA events around the library's main kernels), the
// kernel launch counter, the FP64 throughput probe used as the roofline
// denominator, and the host-buffer entry point.
#include <atomic>
#include <mutex>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>
#include "rs_internal.h"
#include "rs_wave.cuh"

namespace rs {

static std::atomic<long long> g_launches{0};

static thread_local char g_last_error[256] = "";

rot_status cuda_failed(cudaError_t e, const char* where) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
  cudaGetLastError();
  return ROT_ECUDA;
}

void note_error(const char* what) { snprintf(g_last_error, sizeof g_last_error, "%s", what); }

cudaError_t smem_opt_in(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> done;   // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& d : done)
    if (d.first.first == kernel && d.first.second == dev && d.second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.push_back({{kernel, dev}, bytes});
  return e;
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct TraceEntry {
  int kind;
  long long work;
  cudaEvent_t e0, e1;
};
static std::mutex g_trace_mu;
static bool g_trace_on = false;
static std::vector<TraceEntry> g_trace;

int trace_begin(int kind, long long work, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on) return -1;
  TraceEntry t{kind, work, nullptr, nullptr};
  if (cudaEventCreate(&t.e0) != cudaSuccess || cudaEventCreate(&t.e1) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaEventRecord(t.e0, s);
  g_trace.push_back(t);
  return (int)g_trace.size() - 1;
}

void trace_end(int id, cudaStream_t s) {
  if (id < 0) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (id < (int)g_trace.size()) cudaEventRecord(g_trace[id].e1, s);
}

// FP64 throughput probe: every thread runs NC independent DFMA chains.
template <int NC>
__global__ void dfma_probe_kernel(double* out, double b, double c, int iters) {
  double a[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) a[i] = 1.0 + threadIdx.x * 1e-9 + i * 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NC; ++i) a[i] = __fma_rn(a[i], b, c);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < NC; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 instruction-mix probe: every thread keeps NP independent (x, y) pairs
// in registers and updates each pair per iteration with
//   KIND 0: two DFMA      x = fma(x, c, s), y = fma(y, c, s)
//   KIND 1: two DMUL      x = x*c, y = y*c
//   KIND 2: a rotation    2 DMUL + 2 DFMA with the wave kernel's placement
//   KIND 3: a rotation whose (c, s) pair comes from shared memory (one
//           broadcast 16-byte load per rotation, as in the wave kernel)
//   KIND 4: KIND 3 with the two products as DFMAs with a freshly computed -0
//           addend (the form the FP64 kernels use)
//   KIND 5: two DFMA per pair, multiplier and addend from shared memory
// Values stay bounded: |c| < 1 and the rotation is orthogonal.  c and s pass
// through an opaque move so that they sit in registers (an FP64 instruction
// that reads a kernel parameter straight from the constant bank issues more
// slowly, which would make the probe a poor ceiling).
template <int KIND, int NP>
__global__ void fp64_mix_probe_kernel(double* out, double c_arg, double s_arg, int iters) {
  double c, s;
  asm volatile("mov.b64 %0, %1;" : "=d"(c) : "d"(c_arg));
  asm volatile("mov.b64 %0, %1;" : "=d"(s) : "d"(s_arg));
  __shared__ double2 tab[64];
  if (KIND >= 3) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = make_double2(c, s * (1.0 - 1e-9 * i));
    __syncthreads();
  }
  double x[NP], y[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    x[i] = 1.0 + threadIdx.x * 1e-9 + i * 1e-7;
    y[i] = 0.5 - threadIdx.x * 1e-9 + i * 1e-7;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if constexpr (KIND == 0) {
        x[i] = __fma_rn(x[i], c, s);
        y[i] = __fma_rn(y[i], c, s);
      } else if constexpr (KIND == 1) {
        x[i] = __dmul_rn(x[i], c);
        y[i] = __dmul_rn(y[i], c);
      } else if constexpr (KIND == 2) {
        const double sy = __dmul_rn(s, y[i]);
        const double sx = __dmul_rn(s, x[i]);
        const double xn = __fma_rn(c, x[i], sy);
        y[i] = __fma_rn(c, y[i], -sx);
        x[i] = xn;
      } else if constexpr (KIND == 3) {
        const double2 cs = tab[(it * NP + i) & 63];
        const double sy = __dmul_rn(cs.y, y[i]);
        const double sx = __dmul_rn(cs.y, x[i]);
        const double xn = __fma_rn(cs.x, x[i], sy);
        y[i] = __fma_rn(cs.x, y[i], -sx);
        x[i] = xn;
      } else if constexpr (KIND == 4) {
        const double2 cs = tab[(it * NP + i) & 63];
        rotate(x[i], y[i], cs.x, cs.y);
      } else {
        const double2 cs = tab[(it * NP + i) & 63];
        x[i] = __fma_rn(x[i], cs.x, cs.y);
        y[i] = __fma_rn(y[i], cs.x, cs.y);
      }
    }
  }
  double acc = 0;
#pragma unroll
  for (int i = 0; i < NP; ++i) acc += x[i] + y[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace rs

extern "C" {

const char* rot_last_error(void) { return rs::g_last_error; }

rot_status rot_trace_start(void) {
  std::lock_guard<std::mutex> lk(rs::g_trace_mu);
  for (auto& t : rs::g_trace) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  rs::g_trace.clear();
  rs::g_trace_on = true;
  return ROT_OK;
}

rot_status rot_trace_stop(rot_trace_record* out, int capacity, int* count) {
  std::lock_guard<std::mutex> lk(rs::g_trace_mu);
  rs::g_trace_on = false;
  rot_status st = ROT_OK;
  int n = 0;
  for (auto& t : rs::g_trace) {
    float ms = -1.f;
    if (cudaEventSynchronize(t.e1) != cudaSuccess || cudaEventElapsedTime(&ms, t.e0, t.e1) != cudaSuccess) {
      cudaGetLastError();
      st = ROT_ECUDA;
    }
    if (out && n < capacity) {
      out[n].kind = t.kind;
      out[n].ms = ms;
      out[n].work = t.work;
    }
    ++n;
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  rs::g_trace.clear();
  if (count) *count = n;
  return st;
}

int64_t rot_launch_count(void) { return rs::g_launches.load(); }

rot_status rot_measure_fp64_peak(double* gflops, double* ms_out) {
  if (!gflops) return ROT_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROT_ECUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 1024, iters = 4000;
  const int blocks = nsm * 2;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return ROT_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  rs::dfma_probe_kernel<8><<<blocks, threads>>>(buf, 0.9999999, 1e-9, iters);
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) rs::dfma_probe_kernel<8><<<blocks, threads>>>(buf, 0.9999999, 1e-9, iters);
  cudaEventRecord(e1);
  rot_status st = ROT_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    st = ROT_ECUDA;
  rs::count_launches(reps + 1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != ROT_OK) return st;
  const double fmas = (double)blocks * threads * iters * 8 * reps;
  *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
  if (ms_out) *ms_out = ms / reps;
  return ROT_OK;
}


rot_status rot_measure_fp64_mix(int kind, int warps_per_cta, int ctas_per_sm, double* lane_ops_per_s,
                                double* ms_out) {
  if (!lane_ops_per_s || kind < 0 || kind > 5 || warps_per_cta < 1 || warps_per_cta > 32 ||
      ctas_per_sm < 1 || ctas_per_sm > 32 || warps_per_cta * ctas_per_sm > 64)
    return ROT_EINVAL;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rs::cuda_failed(e, "fp64 mix probe: cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return rs::cuda_failed(e, "fp64 mix probe: cudaDeviceGetAttribute");
  constexpr int NP = 4;
  const int threads = warps_per_cta * 32;
  const int blocks = nsm * ctas_per_sm;
  // About 16 ms per launch at 2 FP64 lanes per clock per SM and 2 GHz.
  const double lanes_per_iter = (double)NP * ((kind >= 2 && kind <= 4) ? 4 : 2);
  int iters = (int)(2.0e9 * 0.016 * 2.0 / (warps_per_cta * ctas_per_sm * 32.0 * lanes_per_iter));
  if (iters < 16) iters = 16;
  using K = void (*)(double*, double, double, int);
  const K kernels[6] = {rs::fp64_mix_probe_kernel<0, NP>, rs::fp64_mix_probe_kernel<1, NP>,
                        rs::fp64_mix_probe_kernel<2, NP>, rs::fp64_mix_probe_kernel<3, NP>,
                        rs::fp64_mix_probe_kernel<4, NP>, rs::fp64_mix_probe_kernel<5, NP>};
  double* buf = nullptr;
  e = cudaMalloc(&buf, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rot_status st = ROT_OK;
  float ms = 0.f;
  const int reps = 3;
  const double c = 0.99999999, s = 1.4142135e-4;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = rs::cuda_failed(e, "fp64 mix probe: cudaEventCreate");
  } else {
    kernels[kind]<<<blocks, threads>>>(buf, c, s, iters);
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) kernels[kind]<<<blocks, threads>>>(buf, c, s, iters);
    cudaEventRecord(e1);
    if ((e = cudaGetLastError()) != cudaSuccess) st = rs::cuda_failed(e, "fp64 mix probe: launch");
    else if ((e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
      st = rs::cuda_failed(e, "fp64 mix probe: events");
    rs::count_launches(reps + 1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != ROT_OK) return st;
  const double lane_ops = (double)blocks * threads * iters * lanes_per_iter * reps;
  *lane_ops_per_s = lane_ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms / reps;
  return ROT_OK;
}

}  // extern "C"
