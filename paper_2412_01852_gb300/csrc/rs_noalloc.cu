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
// It comes into being with this library's device code on a device: under the
// CUDA runtime's lazy module loading that is the first set-up on the device
// (rot_apply_noalloc_prepare or the first rot_apply_noalloc), and it stays
// until the process exits.  In host code the array's name only stands in for
// the symbol, so its device address is looked up with cudaGetSymbolAddress
// once per device and context, and passed to the kernels.
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

// Set-up done on one device, valid for one CUDA context: a device reset (or a
// released and re-created primary context) reloads the library's device code,
// which may place the array elsewhere, and drops the kernel's attributes.
struct DeviceSetup {
  unsigned long long ctx_id = 0;   // context the set-up belongs to (0: none yet)
  void* scratch = nullptr;         // device address of g_noalloc_scratch there
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kNoAllocMaxDevices];

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Unique id of the calling thread's current CUDA context (driver entry points
// taken through the runtime), or 0 if it cannot be read.
unsigned long long current_context_id() {
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(p);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

using WaveKernel = void (*)(const CUtensorMap, const rs::WaveProblem);
inline WaveKernel noalloc_kernel() { return rs::wave_kernel<double, kKMAX, kNBT, kWarps>; }
inline int noalloc_smem() { return kWarps * rs::WaveSmem<double, kKMAX, kNBT>::kWarpBytes; }

// Set-up on the current device: look up the array's device address (loading
// the library's device code, and with it the array, if that has not happened
// yet) and allow the kernel its shared memory.  Done once per device and
// context; *scratch receives the address.
rot_status noalloc_setup(void** scratch) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    rs::note_error("noalloc: device ordinal beyond the supported 64 devices");
    return ROT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup& d = g_setup[dev];
  const unsigned long long ctx = current_context_id();
  if (d.scratch && ctx != 0 && d.ctx_id == ctx) {
    *scratch = d.scratch;
    return ROT_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: cudaGetSymbolAddress");
  e = cudaFuncSetAttribute(noalloc_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, noalloc_smem());
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: cudaFuncSetAttribute");
  d.ctx_id = current_context_id();   // the context exists now
  d.scratch = p;
  *scratch = p;
  return ROT_OK;
}

}  // namespace

extern "C" rot_status rot_apply_noalloc_prepare(void) {
  void* p = nullptr;
  return noalloc_setup(&p);
}

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
  // p-blocks as rot_apply's wavefront kernel takes them (longer ones while
  // they still give every resident warp a work item)
  const rs::WavePlan pl = rs::plan_wave(m, n, k, kKMAX, kNBT, rs::wave_default_K_f64(m, k, 0), 0, (int)sizeof(T));
  const int64_t W2 = 2 * (int64_t)pl.kpad;
  const size_t cs_bytes = (size_t)pl.cs_rows * W2 * sizeof(T);
  const size_t done_off = round_up(cs_bytes, 256);
  const size_t done_bytes = (size_t)pl.nchains * pl.G * sizeof(int);
  const size_t tick_off = round_up(done_off + done_bytes, 256);
  const size_t total_bytes = tick_off + 256;
  if (total_bytes > kNoAllocScratchBytes) {   // beyond the static scratch
    rs::note_error("noalloc: the problem needs more than the 32 MiB static scratch");
    return ROT_EINVAL;
  }

  void* scratch = nullptr;
  const rot_status su = noalloc_setup(&scratch);
  if (su != ROT_OK) return su;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: device attributes");
  const WaveKernel kfn = noalloc_kernel();
  const int smem = noalloc_smem();
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem);
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: occupancy");
  if (occ < 1) {
    rs::note_error("noalloc: the wavefront kernel does not fit on an SM");
    return ROT_ECUDA;
  }

  // Counters, ticket and status start at zero on every call; the repacked
  // (c, s) rows are fully rewritten where they are read.
  e = cudaMemsetAsync(base + done_off, 0, total_bytes - done_off, s);
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: cudaMemsetAsync");
  T* cs = reinterpret_cast<T*>(base);
  dim3 rb(32, 8);
  dim3 rg((unsigned)ceil_div(n - 1, 32), (unsigned)ceil_div(k, 8));
  rs::repack_cs_kernel<T><<<rg, rb, 0, s>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: repack launch");
  rs::count_launches(1);

  CUtensorMap map;
  if (!rs::encode_tile_map_2d(&map, cs, true, (uint64_t)W2, (uint64_t)pl.cs_rows,
                              (uint64_t)W2 * sizeof(T), 2 * kKMAX, kNBT)) {
    rs::note_error("noalloc: cuTensorMapEncodeTiled failed");
    return ROT_ECUDA;
  }

  rs::WaveProblem P{};
  P.A = A; P.lda = lda; P.m = (int)m; P.n = (int)n; P.k = (int)k;
  P.K = pl.K; P.NB = pl.NB; P.delta = pl.delta; P.nchains = pl.nchains; P.G = pl.G; P.B = pl.B;
  P.cs_row0 = 0;
  rs::set_full_range(P);
  P.done = reinterpret_cast<int*>(base + done_off);
  P.ticket = reinterpret_cast<unsigned long long*>(base + tick_off);
  P.status = reinterpret_cast<int*>(base + tick_off + 64);
  P.total = pl.total;

  long long grid = (long long)nsm * occ;
  const long long need = (P.total + kWarps - 1) / kWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  const int tr = rs::trace_begin(ROT_KERNEL_WAVE_F64, m * (n - 1) * k, s);
  kfn<<<(unsigned)grid, kWarps * 32, smem, s>>>(map, P);
  rs::trace_end(tr, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: wavefront kernel launch");
  rs::record_status_async(P.status, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rs::cuda_failed(e, "noalloc: status launch");
  rs::count_launches(2);
  return ROT_OK;
}
