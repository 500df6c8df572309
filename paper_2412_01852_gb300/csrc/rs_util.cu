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


}  // extern "C"
