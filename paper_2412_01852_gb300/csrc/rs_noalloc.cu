// rs_noalloc.cu -- rot_apply_noalloc: the FP64 wavefront path with its scratch
// memory in a fixed static device array, for callers that cannot let a
// library allocate device memory.
//
// Who needs this: applications that own all device memory themselves (a
// framework that reserves the GPU's memory up front for its own pool, or a
// plugin running inside such a host) cannot have a library call cudaMalloc:
// the call may fail because the pool already holds the memory, it fragments
// the host's pool, and cudaMalloc/cudaFree can synchronize the device, which
// latency-bound loops cannot afford.  rot_apply takes its scratch from the
// stream-ordered allocator; this entry point takes none.
//
// The scratch lives in g_noalloc_scratch below (kNoAllocScratchBytes, 32 MiB).
// Every GPU that loads this library reserves that array until the process
// exits.  In host code the array's name only stands in for the symbol, so its
// device address is looked up once per device with cudaGetSymbolAddress and
// passed to the kernels.
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>
#include <cuda.h>

#include "rs_wave.cuh"
#include "rs_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;
constexpr int kKMAX = 16;
constexpr int kNBT = 16;
constexpr int kWarps = 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kNoAllocMaxDevices] = {};
bool g_attr_set[kNoAllocMaxDevices] = {};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Device address of the static scratch array on the current device (looked up
// on the first call per device).  Returns nullptr on failure.
void* scratch_for_device(int dev) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" rot_status rot_apply_noalloc(int64_t m, int64_t n, int64_t k, double* A, int64_t lda,
                                        const double* C, int64_t ldc, const double* S, int64_t lds,
                                        void* stream) {
  // Same argument checks and quick returns as rot_apply.
  const int64_t lim = (int64_t(1) << 31) - 1;
  if (m < 0 || n < 0 || k < 0) return ROT_EINVAL;
  if (m > lim || n > lim || k > lim || n + k > lim) return ROT_EINVAL;
  if (lda < (m > 1 ? m : 1)) return ROT_EINVAL;
  const int64_t nm1 = n - 1 > 1 ? n - 1 : 1;
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) return ROT_OK;
  if (!A || !C || !S) return ROT_EINVAL;

  using T = double;
  const rs::WavePlan pl = rs::plan_wave(m, n, k, kKMAX, kNBT, 0, 0, (int)sizeof(T));
  const int64_t W2 = 2 * (int64_t)pl.kpad;
  const size_t cs_bytes = (size_t)pl.cs_rows * W2 * sizeof(T);
  const size_t done_off = round_up(cs_bytes, 256);
  const size_t done_bytes = (size_t)pl.nchains * pl.G * sizeof(int);
  const size_t tick_off = round_up(done_off + done_bytes, 256);
  const size_t total_bytes = tick_off + 256;
  if (total_bytes > kNoAllocScratchBytes) return ROT_EINVAL;  // beyond the static scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROT_ECUDA;
  unsigned char* base = static_cast<unsigned char*>(scratch_for_device(dev));
  if (!base) return ROT_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  auto kfn = rs::wave_kernel<T, kKMAX, kNBT, kWarps>;
  const int smem = kWarps * rs::WaveSmem<T, kKMAX, kNBT>::kWarpBytes;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_attr_set[dev]) {
      if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return ROT_ECUDA;
      g_attr_set[dev] = true;
    }
  }

  // Counters, ticket and status start at zero on every call; the repacked
  // (c, s) rows are fully rewritten where they are read.
  if (cudaMemsetAsync(base + done_off, 0, total_bytes - done_off, s) != cudaSuccess) return ROT_ECUDA;
  T* cs = reinterpret_cast<T*>(base);
  dim3 rb(32, 8);
  dim3 rg((unsigned)ceil_div(n - 1, 32), (unsigned)ceil_div(k, 8));
  rs::repack_cs_kernel<T><<<rg, rb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
  if (cudaGetLastError() != cudaSuccess) return ROT_ECUDA;

  CUtensorMap map;
  if (!rs::encode_tile_map_2d(&map, cs, true, (uint64_t)W2, (uint64_t)pl.cs_rows,
                              (uint64_t)W2 * sizeof(T), 2 * kKMAX, kNBT))
    return ROT_ECUDA;

  rs::WaveProblem P{};
  P.A = A; P.lda = lda; P.m = (int)m; P.n = (int)n; P.k = (int)k;
  P.K = pl.K; P.NB = pl.NB; P.delta = pl.delta; P.nchains = pl.nchains; P.G = pl.G; P.B = pl.B;
  P.cs_row0 = 0;
  rs::set_full_range(P);
  P.done = reinterpret_cast<int*>(base + done_off);
  P.ticket = reinterpret_cast<unsigned long long*>(base + tick_off);
  P.status = reinterpret_cast<int*>(base + tick_off + 64);
  P.total = pl.total;

  int nsm = 0, occ = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem) != cudaSuccess || occ < 1)
    return ROT_ECUDA;
  long long grid = (long long)nsm * occ;
  const long long need = (P.total + kWarps - 1) / kWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kfn<<<(unsigned)grid, kWarps * 32, smem, s>>>(map, P);
  if (cudaGetLastError() != cudaSuccess) return ROT_ECUDA;
  rs::record_status_async(P.status, s);
  if (cudaGetLastError() != cudaSuccess) return ROT_ECUDA;
  rs::count_launches(3);
  return ROT_OK;
}
