// rs_util.cu -- tracing (CUDA events around the library's main kernels), the
// kernel launch counter, the FP64 throughput probe used as the roofline
// denominator, and the host-buffer entry point.
#include <atomic>
#include <mutex>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>
#include "rs_internal.h"

namespace rs {

static std::atomic<long long> g_launches{0};

static thread_local char g_last_error[256] = "";

rot_status cuda_failed(cudaError_t e, const char* where) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
  cudaGetLastError();
  return ROT_ECUDA;
}

void note_error(const char* what) { snprintf(g_last_error, sizeof g_last_error, "%s", what); }
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

rot_status rot_apply_host(int64_t m, int64_t n, int64_t k, double* A_host, int64_t lda,
                          const double* C_host, int64_t ldc, const double* S_host, int64_t lds,
                          void* stream) {
  if (m < 0 || n < 0 || k < 0 || lda < (m > 1 ? m : 1)) return ROT_EINVAL;
  const int64_t nm1 = n - 1 > 1 ? n - 1 : 1;
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) return ROT_OK;
  if (!A_host || !C_host || !S_host) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t a_bytes = (size_t)m * n * sizeof(double);
  const size_t cs_bytes = (size_t)(n - 1) * k * sizeof(double);
  double *dA = nullptr, *dC = nullptr, *dS = nullptr;
  if (cudaMallocAsync((void**)&dA, a_bytes, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dC, cs_bytes, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dS, cs_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    if (dA) cudaFreeAsync(dA, s);
    if (dC) cudaFreeAsync(dC, s);
    cudaStreamSynchronize(s);
    return ROT_ENOMEM;
  }
  rot_status st = ROT_OK;
  do {
    if (cudaMemcpy2DAsync(dA, m * sizeof(double), A_host, lda * sizeof(double), m * sizeof(double), n,
                          cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(dC, (n - 1) * sizeof(double), C_host, ldc * sizeof(double),
                          (n - 1) * sizeof(double), k, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(dS, (n - 1) * sizeof(double), S_host, lds * sizeof(double),
                          (n - 1) * sizeof(double), k, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = ROT_ECUDA;
      break;
    }
    st = rot_apply(m, n, k, dA, m, dC, n - 1, dS, n - 1, stream);
    if (st != ROT_OK) break;
    if (cudaMemcpy2DAsync(A_host, lda * sizeof(double), dA, m * sizeof(double), m * sizeof(double), n,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      st = ROT_ECUDA;
      break;
    }
  } while (0);
  cudaFreeAsync(dA, s);
  cudaFreeAsync(dC, s);
  cudaFreeAsync(dS, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ROT_OK) st = ROT_ECUDA;
  return st;
}

}  // extern "C"
