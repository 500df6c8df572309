// rs_wave_host.cu -- host side of the wavefront kernel: planning, scratch
// memory, the repack of C/S, the TMA tensor map and the launch.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rs_wave.cuh"
#include "rs_wave_f32.cuh"
#include "rs_internal.h"

namespace rs {

// Sticky device status: the first error any launch of this library recorded.
__device__ int g_sticky_status = 0;

__global__ void accumulate_status_kernel(const int* status) {
  const int s = *status;
  if (s != 0) atomicCAS(&g_sticky_status, 0, s);
}

int take_sticky_status() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_sticky_status, sizeof(int)) != cudaSuccess) return -1;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_sticky_status, &zero, sizeof(int)) != cudaSuccess) return -1;
  return v;
}

void record_status_async(const int* status, cudaStream_t stream) {
  accumulate_status_kernel<<<1, 1, 0, stream>>>(status);
}

// ---- cuTensorMapEncodeTiled through the runtime's driver entry point ---------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode_tile_map_2d(CUtensorMap* map, const void* base, bool is_double, uint64_t inner,
                        uint64_t outer, uint64_t row_pitch_bytes, uint32_t box_inner,
                        uint32_t box_outer) {
  auto fn = get_encode();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, is_double ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The same for 16-bit elements (the tensor-core block apply's BF16 operands).
bool encode_tile_map_2d_b16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                            uint64_t row_pitch_bytes, uint32_t box_inner, uint32_t box_outer) {
  auto fn = get_encode();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---- planning -------------------------------------------------------------------
static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

WavePlan plan_wave(int64_t m, int64_t n, int64_t k, int kmax, int nbt, int K_req, int NB_req,
                   int elem_bytes, int rows_per_chain) {
  WavePlan pl{};
  pl.K = (int)std::min<int64_t>(K_req > 0 ? K_req : kmax, std::min<int64_t>(kmax, k));
  // The TMA x coordinate of p-block g is 2*g*K elements and must be a multiple
  // of 16 bytes: for 4-byte elements K must be even once there are two p-blocks.
  if (elem_bytes == 4 && pl.K < k && (pl.K & 1)) pl.K -= 1;
  if (pl.K < 1) pl.K = 1;
  if (elem_bytes == 4 && pl.K < k && (pl.K & 1)) pl.K = 2;
  pl.NB = NB_req > 0 ? NB_req : 32;
  if (pl.NB < nbt) pl.NB = nbt;
  pl.NB = (int)round_up(pl.NB, nbt);
  pl.delta = 1 + (int)ceil_div(pl.K, pl.NB);
  pl.nchains = (int)ceil_div(m, rows_per_chain);
  pl.G = (int)ceil_div(k, pl.K);
  pl.B = (int)ceil_div(n + pl.K - 2, pl.NB);
  pl.total = (long long)pl.nchains * pl.G * pl.B;
  pl.kpad = (int)std::max<int64_t>(round_up(k, 4), kmax);
  pl.cs_rows = (int)std::max<int64_t>(n + k - 2, nbt);
  return pl;
}

// ---- launch -------------------------------------------------------------------
template <typename T, int KMAX, int NBT, int WARPS, int OP>
static cudaError_t launch_wave(const WaveProblem& P, const CUtensorMap& map, cudaStream_t stream,
                               int ctas_per_sm_req) {
  using SM = WaveSmem<T, KMAX, NBT>;
  auto kfn = wave_kernel<T, KMAX, NBT, WARPS, OP>;
  const int smem = WARPS * SM::kWarpBytes;
  const cudaError_t attr_err = smem_opt_in(reinterpret_cast<const void*>(kfn), smem);
  if (attr_err != cudaSuccess) return attr_err;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int per_sm = ctas_per_sm_req > 0 ? std::min(ctas_per_sm_req, occ) : occ;
  long long want = (long long)nsm * per_sm;
  // No more CTAs than there are items for their warps.
  long long need = (P.total + WARPS - 1) / WARPS;
  if (want > need) want = need;
  if (want < 1) want = 1;
  kfn<<<(unsigned)want, WARPS * 32, smem, stream>>>(map, P);
  return cudaGetLastError();
}

template <typename T>
static constexpr int kmax_for() { return 16; }
static constexpr int kNBT = 16;
static constexpr int kWarps = 8;

// Sequences per p-block when the caller leaves the choice to the library:
// the longest of 16, 8 and 4 that still gives every resident warp a work
// item (a 32-row chain in one p-block) at once, the rule the batched launch
// uses.  Measured on GB300 (whole calls, FP64): 8192 x 8192 k = 192 83.3 ms
// at 16 (84.1 at 4); 2048 x 2048 k = 192 9.09 at 16, 6.89 at 4; 512 rows x
// 4096 columns k = 192 13.3 at 16, 7.23 at 4; 4096 x 4096 k = 96 15.0 at 16,
// 11.3 at 4.
template <typename T>
static int default_K(int64_t m, int64_t k, int ctas_per_sm_req) {
  using SM = WaveSmem<T, kmax_for<T>(), kNBT>;
  auto kfn = wave_kernel<T, kmax_for<T>(), kNBT, kWarps, kOpRotate>;
  const int smem = kWarps * SM::kWarpBytes;
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess || smem_opt_in(reinterpret_cast<const void*>(kfn), smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return kmax_for<T>();
  }
  const int per_sm = ctas_per_sm_req > 0 ? std::min(ctas_per_sm_req, occ) : occ;
  const long long warps = (long long)nsm * per_sm * kWarps;
  const long long chains = ceil_div(m, 32);
  for (int K : {16, 8})
    if (chains * ceil_div(k, K) >= warps) return K;
  return 4;
}

int wave_default_K_f64(int64_t m, int64_t k, int ctas_per_sm_req) { return default_K<double>(m, k, ctas_per_sm_req); }

template <typename T>
rot_status wave_apply(int64_t m, int64_t n, int64_t k, T* A, int64_t lda, const T* C, int64_t ldc,
                      const T* S, int64_t lds, cudaStream_t stream, const WaveOptions& opt) {
  constexpr int KMAX = kmax_for<T>();
  const int K_req = opt.K > 0 ? opt.K : default_K<T>(m, k, opt.ctas_per_sm);
  const WavePlan pl = plan_wave(m, n, k, KMAX, kNBT, K_req, opt.NB, (int)sizeof(T), 32);

  // Scratch: [repacked (c,s) | done counters | ticket | status]
  const int64_t W2 = 2 * (int64_t)pl.kpad;
  const size_t cs_bytes = (size_t)pl.cs_rows * W2 * sizeof(T);
  const size_t cs_off = 0;
  const size_t done_off = round_up(cs_bytes, 256);
  const size_t done_bytes = (size_t)pl.nchains * pl.G * sizeof(int);
  const size_t tick_off = round_up(done_off + done_bytes, 256);
  const size_t total_bytes = tick_off + 256;

  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, total_bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  rot_status st = ROT_OK;
  do {
    if (cudaMemsetAsync(base + done_off, 0, total_bytes - done_off, stream) != cudaSuccess) { st = ROT_ECUDA; break; }
    T* cs = reinterpret_cast<T*>(base + cs_off);
    dim3 rb(32, 8);
    dim3 rg((unsigned)ceil_div(n - 1, 32), (unsigned)ceil_div(k, 8));
    repack_cs_kernel<T><<<rg, rb, 0, stream>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) { st = ROT_ECUDA; break; }

    CUtensorMap map;
    if (!encode_tile_map_2d(&map, cs, sizeof(T) == 8, (uint64_t)W2, (uint64_t)pl.cs_rows,
                            (uint64_t)W2 * sizeof(T), 2 * KMAX, kNBT)) { st = ROT_ECUDA; break; }

    WaveProblem P{};
    P.A = A; P.lda = lda; P.m = (int)m; P.n = (int)n; P.k = (int)k;
    P.K = pl.K; P.NB = pl.NB; P.delta = pl.delta; P.nchains = pl.nchains; P.G = pl.G; P.B = pl.B;
    P.cs_row0 = 0;
    set_full_range(P);
    P.chain_stride = opt.chain_stride;
    P.done = reinterpret_cast<int*>(base + done_off);
    P.ticket = reinterpret_cast<unsigned long long*>(base + tick_off);
    P.status = reinterpret_cast<int*>(base + tick_off + 64);
    P.total = pl.total;
    P.arrived = opt.arrived;
    P.arrive_cols = opt.arrive_cols;
    P.last_done = opt.last_done;
    const int tr = trace_begin(opt.reflectors ? ROT_KERNEL_REFLECT_F64
                               : sizeof(T) == 8 ? ROT_KERNEL_WAVE_F64 : ROT_KERNEL_WAVE_F32,
                               (long long)m * (n - 1) * k, stream);
    const int prod = opt.fp64_products ? opt.fp64_products : kDefaultFp64Products;
    cudaError_t le;
    if constexpr (sizeof(T) == 8) {
      if (opt.reflectors) le = launch_wave<T, KMAX, kNBT, kWarps, kOpReflect>(P, map, stream, opt.ctas_per_sm);
      else if (prod == 2) le = launch_wave<T, KMAX, kNBT, kWarps, kOpRotateIntmul>(P, map, stream, opt.ctas_per_sm);
      else le = launch_wave<T, KMAX, kNBT, kWarps, kOpRotate>(P, map, stream, opt.ctas_per_sm);
    } else {
      (void)prod;
      le = launch_wave<T, KMAX, kNBT, kWarps, kOpRotate>(P, map, stream, opt.ctas_per_sm);
    }
    trace_end(tr, stream);
    if (le != cudaSuccess) { st = ROT_ECUDA; break; }
    record_status_async(P.status, stream);
    count_launches(2);
    if (cudaGetLastError() != cudaSuccess) { st = ROT_ECUDA; break; }
  } while (0);
  cudaFreeAsync(scratch, stream);
  return st;
}

// FP32: 64-row chains (2 rows per lane), p-blocks of 8 sequences, 9-wave
// tiles, 6 tiles per item, 2 CTAs of 8 warps per SM.  Measured on GB300
// (A 8192x8192, k = 192): this shape 3.43 ms (4 tiles per item 3.53, 8 tiles
// 3.56); 16-sequence p-blocks with 17-wave tiles 4.51 ms (their unrolled tile
// strains the instruction cache); 12-sequence 3.70 ms; 4 rows per lane
// 3.88 ms.
static constexpr int kF32Kmax = 8;
static constexpr int kF32R = 2;
static constexpr int kF32NBT = kF32Kmax + 1;
static constexpr int kF32MinBlocks = 2;

static cudaError_t launch_wave_f32(const WaveProblem& P, const CUtensorMap& map, cudaStream_t stream,
                                   int ctas_per_sm_req) {
  using SM = WaveSmem<float, kF32Kmax, kF32NBT>;
  auto kfn = wave_f32_kernel<kF32Kmax, kF32R, kWarps, kF32MinBlocks>;
  const int smem = kWarps * SM::kWarpBytes;
  const cudaError_t attr_err = smem_opt_in(reinterpret_cast<const void*>(kfn), smem);
  if (attr_err != cudaSuccess) return attr_err;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int per_sm = ctas_per_sm_req > 0 ? std::min(ctas_per_sm_req, occ) : occ;
  long long want = std::min<long long>((long long)nsm * per_sm, (P.total + kWarps - 1) / kWarps);
  kfn<<<(unsigned)std::max<long long>(want, 1), kWarps * 32, smem, stream>>>(map, P);
  return cudaGetLastError();
}

rot_status wave_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C,
                          int64_t ldc, const float* S, int64_t lds, cudaStream_t stream, const WaveOptions& opt) {
  const WavePlan pl = plan_wave(m, n, k, kF32Kmax, kF32NBT, opt.K, opt.NB > 0 ? opt.NB : 6 * kF32NBT, 4,
                                32 * kF32R);
  const int64_t W2 = 2 * (int64_t)pl.kpad;
  const size_t cs_bytes = (size_t)pl.cs_rows * W2 * sizeof(float);
  const size_t done_off = round_up(cs_bytes, 256);
  const size_t done_bytes = (size_t)pl.nchains * pl.G * sizeof(int);
  const size_t tick_off = round_up(done_off + done_bytes, 256);
  const size_t total_bytes = tick_off + 256;
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, total_bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return ROT_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  rot_status st = ROT_OK;
  do {
    cudaError_t e = cudaMemsetAsync(base + done_off, 0, total_bytes - done_off, stream);
    if (e != cudaSuccess) { st = cuda_failed(e, "rot_apply_f32: memset"); break; }
    float* cs = reinterpret_cast<float*>(base);
    dim3 rb(32, 8);
    dim3 rg((unsigned)ceil_div(n - 1, 32), (unsigned)ceil_div(k, 8));
    repack_cs_kernel<float><<<rg, rb, 0, stream>>>(C, ldc, S, lds, (int)n, (int)k, cs, W2, 0);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_failed(e, "rot_apply_f32: repack"); break; }
    CUtensorMap map;
    if (!encode_tile_map_2d(&map, cs, false, (uint64_t)W2, (uint64_t)pl.cs_rows, (uint64_t)W2 * sizeof(float),
                            2 * kF32Kmax, kF32NBT)) {
      note_error("rot_apply_f32: cuTensorMapEncodeTiled failed");
      st = ROT_ECUDA;
      break;
    }
    WaveProblem P{};
    P.A = A; P.lda = lda; P.m = (int)m; P.n = (int)n; P.k = (int)k;
    P.K = pl.K; P.NB = pl.NB; P.delta = pl.delta; P.nchains = pl.nchains; P.G = pl.G; P.B = pl.B;
    P.cs_row0 = 0;
    set_full_range(P);
    P.chain_stride = opt.chain_stride;
    P.done = reinterpret_cast<int*>(base + done_off);
    P.ticket = reinterpret_cast<unsigned long long*>(base + tick_off);
    P.status = reinterpret_cast<int*>(base + tick_off + 64);
    P.total = pl.total;
    const int tr = trace_begin(ROT_KERNEL_WAVE_F32, (long long)m * (n - 1) * k, stream);
    e = launch_wave_f32(P, map, stream, opt.ctas_per_sm);
    trace_end(tr, stream);
    if (e != cudaSuccess) { st = cuda_failed(e, "rot_apply_f32: kernel launch"); break; }
    record_status_async(P.status, stream);
    count_launches(2);
  } while (0);
  cudaFreeAsync(scratch, stream);
  return st;
}

// Fault-detection self-test: the FP64 wave kernel on a small problem whose
// ticket counter starts past the first wave-block of every chain, so the
// items handed out wait on counters that nothing will advance.  Their bounded
// waits run out after wait_ms, record a timeout in the status word and the
// kernel returns; nothing faults or traps, and the context stays usable.
rot_status selftest_dependency_timeout(int wait_ms, cudaStream_t stream, int* device_status) {
  const int64_t m = 64, n = 256, k = 4;
  const WavePlan pl = plan_wave(m, n, k, 16, kNBT, 0, 0, 8, 32);
  const int64_t W2 = 2 * (int64_t)pl.kpad;
  const size_t a_bytes = (size_t)m * n * sizeof(double);
  const size_t cs_bytes = (size_t)pl.cs_rows * W2 * sizeof(double);
  const size_t cs_off = round_up(a_bytes, 256);
  const size_t done_off = round_up(cs_off + cs_bytes, 256);
  const size_t tick_off = round_up(done_off + (size_t)pl.nchains * pl.G * sizeof(int), 256);
  const size_t total = tick_off + 256;
  unsigned char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, total, stream);
  if (e != cudaSuccess) return cuda_failed(e, "selftest: allocation");
  rot_status st = ROT_OK;
  do {
    e = cudaMemsetAsync(base, 0, total, stream);
    if (e != cudaSuccess) { st = cuda_failed(e, "selftest: memset"); break; }
    // Start the tickets after key 0: every chain's first item (b = 0, g = 0)
    // is never handed out, so its dependants wait in vain.
    const unsigned long long first = (unsigned long long)pl.nchains;
    e = cudaMemcpyAsync(base + tick_off, &first, sizeof first, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) { st = cuda_failed(e, "selftest: ticket"); break; }
    CUtensorMap map;
    if (!encode_tile_map_2d(&map, base + cs_off, true, (uint64_t)W2, (uint64_t)pl.cs_rows,
                            (uint64_t)W2 * sizeof(double), 2 * 16, kNBT)) {
      note_error("selftest: cuTensorMapEncodeTiled failed");
      st = ROT_ECUDA;
      break;
    }
    WaveProblem P{};
    P.A = base; P.lda = m; P.m = (int)m; P.n = (int)n; P.k = (int)k;
    P.K = pl.K; P.NB = pl.NB; P.delta = pl.delta; P.nchains = pl.nchains; P.G = pl.G; P.B = pl.B;
    set_full_range(P);
    P.done = reinterpret_cast<int*>(base + done_off);
    P.ticket = reinterpret_cast<unsigned long long*>(base + tick_off);
    P.status = reinterpret_cast<int*>(base + tick_off + 64);
    P.total = pl.total;
    P.wait_ns = (unsigned long long)wait_ms * 1000000ull;
    e = launch_wave<double, 16, kNBT, kWarps, kOpRotate>(P, map, stream, 1);
    if (e != cudaSuccess) { st = cuda_failed(e, "selftest: launch"); break; }
    int hs = 0;
    e = cudaMemcpyAsync(&hs, P.status, sizeof hs, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { st = cuda_failed(e, "selftest: status"); break; }
    *device_status = hs;
  } while (0);
  cudaFreeAsync(base, stream);
  cudaStreamSynchronize(stream);
  return st;
}

template rot_status wave_apply<double>(int64_t, int64_t, int64_t, double*, int64_t, const double*,
                                       int64_t, const double*, int64_t, cudaStream_t,
                                       const WaveOptions&);


}  // namespace rs
