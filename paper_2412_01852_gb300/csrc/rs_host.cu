// rs_host.cu -- rot_apply on host buffers, with the copies overlapped with
// the rotations.
//
// A is uploaded in column chunks on a copy stream; after each chunk the copy
// stream writes that chunk's arrival flag (a stream memory operation, so no
// SM is needed while the persistent wavefront kernel holds them all).  Work
// items of the first p-block wait for the chunk holding the columns they
// read.  The kernel counts, per wave-block, the chains that finished that
// wave-block of the last p-block; the copy stream waits (stream memory
// operation) until a chunk's columns are final in every chain and copies it
// back while the kernel works on later columns.  After the kernel a small
// kernel sets every count to its final value, so the copy stream never waits
// on a launch that stopped early.  Without stream memory operations the same
// steps run one after another.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "rs_internal.h"

namespace rs {
namespace {

typedef CUresult (*WriteValue32Fn)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
typedef CUresult (*WaitValue32Fn)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);

struct StreamOps {
  WriteValue32Fn write = nullptr;
  WaitValue32Fn wait = nullptr;
};

const StreamOps& stream_ops() {
  static StreamOps ops;
  static std::once_flag once;
  std::call_once(once, [] {
    void* w = nullptr;
    void* v = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &w, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuStreamWaitValue32", &v, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
      ops.write = reinterpret_cast<WriteValue32Fn>(w);
      ops.wait = reinterpret_cast<WaitValue32Fn>(v);
    }
    cudaGetLastError();
  });
  return ops;
}

// Per-device resources of the overlapped path, created on first use: a copy
// stream and a flag buffer from cudaMalloc (stream memory operations act on
// ordinary device allocations).  Calls on one device take turns (the call is
// synchronous anyway).
struct HostPathDevice {
  std::mutex mu;
  cudaStream_t copy = nullptr;
  int* flags = nullptr;
  size_t flag_count = 0;
  bool stream_ops_ok = true;   // cleared if the driver refuses a stream memory operation
};

HostPathDevice& host_path_device(int dev) {
  static std::mutex mu;
  static std::vector<HostPathDevice*> devs;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)devs.size() <= dev) devs.resize(dev + 1, nullptr);
  if (!devs[dev]) devs[dev] = new HostPathDevice;
  return *devs[dev];
}

// One copy stream per device, created on first use.
cudaStream_t copy_stream(int dev) {
  static std::mutex mu;
  static std::vector<cudaStream_t> streams;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

__global__ void fill_kernel(int* p, int count, int value) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) p[i] = value;
}

}  // namespace
}  // namespace rs

extern "C" rot_status rot_apply_host(int64_t m, int64_t n, int64_t k, double* A_host, int64_t lda,
                                     const double* C_host, int64_t ldc, const double* S_host, int64_t lds,
                                     void* stream) {
  if (m < 0 || n < 0 || k < 0 || lda < (m > 1 ? m : 1)) return ROT_EINVAL;
  const int64_t nm1 = n - 1 > 1 ? n - 1 : 1;
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) return ROT_OK;
  if (!A_host || !C_host || !S_host) return ROT_EINVAL;
  if (m > (int64_t(1) << 31) - 1 || n > (int64_t(1) << 31) - 1 || n + k > (int64_t(1) << 31) - 1) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ROT_ECUDA;
  const rs::StreamOps& ops = rs::stream_ops();
  rs::HostPathDevice& hp = rs::host_path_device(dev);
  std::unique_lock<std::mutex> hold(hp.mu);
  cudaStream_t sc = (ops.write && ops.wait && hp.stream_ops_ok) ? rs::copy_stream(dev) : nullptr;

  // The wave kernel's tiling for these sizes (the same call rot_apply makes).
  const rs::WavePlan pl = rs::plan_wave(m, n, k, 16, 16, 0, 0, 8, 32);
  const int kr_last = (int)(k - (int64_t)(pl.G - 1) * pl.K);
  const int nw_last = (int)(n + kr_last - 2);
  const int b_last = (nw_last + pl.NB - 1) / pl.NB;          // wave-blocks of the last p-block with work
  const int nchunks = (int)std::min<int64_t>(16, n);
  const int cols = (int)((n + nchunks - 1) / nchunks);

  const size_t a_bytes = (size_t)m * n * sizeof(double);
  const size_t cs_bytes = (size_t)(n - 1) * k * sizeof(double);
  const size_t flag_count = (size_t)(nchunks + b_last);
  const size_t flag_bytes = flag_count * sizeof(int);
  if (hp.flag_count < flag_count) {
    // The previous call finished (synchronously) with the old buffer.
    if (hp.flags) cudaFree(hp.flags);
    hp.flags = nullptr;
    hp.flag_count = 0;
    if (cudaMalloc((void**)&hp.flags, flag_bytes) != cudaSuccess) { cudaGetLastError(); return ROT_ENOMEM; }
    hp.flag_count = flag_count;
  }
  int* flags = hp.flags;
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
  int* arrived = flags;
  int* last_done = flags + nchunks;
  rot_status st = ROT_OK;
  cudaEvent_t ready = nullptr, copied = nullptr;
  do {
    if (cudaMemsetAsync(flags, 0, flag_bytes, s) != cudaSuccess ||
        cudaMemcpy2DAsync(dC, (n - 1) * sizeof(double), C_host, ldc * sizeof(double), (n - 1) * sizeof(double), k,
                          cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(dS, (n - 1) * sizeof(double), S_host, lds * sizeof(double), (n - 1) * sizeof(double), k,
                          cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = rs::cuda_failed(cudaGetLastError(), "rot_apply_host: setup");
      break;
    }
    if (!sc) {
      // Sequential: upload, rotate, download.
      if (cudaMemcpy2DAsync(dA, m * sizeof(double), A_host, lda * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyHostToDevice, s) != cudaSuccess) { st = ROT_ECUDA; break; }
      st = rs::wave_apply<double>(m, n, k, dA, m, dC, n - 1, dS, n - 1, s, rs::WaveOptions{});
      if (st != ROT_OK) break;
      if (cudaMemcpy2DAsync(A_host, lda * sizeof(double), dA, m * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess) st = ROT_ECUDA;
      break;
    }
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(sc, ready, 0) != cudaSuccess) {
      st = rs::cuda_failed(cudaGetLastError(), "rot_apply_host: events");
      break;
    }
    // Uploads, each followed by its arrival flag.
    CUresult cr = CUDA_SUCCESS;
    for (int i = 0; i < nchunks && st == ROT_OK && cr == CUDA_SUCCESS; ++i) {
      const int64_t c0 = (int64_t)i * cols, c1 = std::min<int64_t>(n, c0 + cols);
      if (c0 < c1 && cudaMemcpy2DAsync(dA + c0 * m, m * sizeof(double), A_host + c0 * lda, lda * sizeof(double),
                                       m * sizeof(double), c1 - c0, cudaMemcpyHostToDevice, sc) != cudaSuccess) {
        st = rs::cuda_failed(cudaGetLastError(), "rot_apply_host: chunked upload");
        break;
      }
      cr = ops.write(sc, (CUdeviceptr)(arrived + i), 1, 0);
    }
    if (st != ROT_OK) break;
    if (cr != CUDA_SUCCESS) {
      // The driver refuses stream memory operations: finish this call and
      // later ones with the copies in sequence.
      char msg[96];
      snprintf(msg, sizeof msg, "rot_apply_host: stream memory operations unavailable (CUresult %d)", (int)cr);
      rs::note_error(msg);
      hp.stream_ops_ok = false;
      if (cudaStreamSynchronize(sc) != cudaSuccess ||
          cudaMemcpy2DAsync(dA, m * sizeof(double), A_host, lda * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyHostToDevice, s) != cudaSuccess) { st = ROT_ECUDA; break; }
      st = rs::wave_apply<double>(m, n, k, dA, m, dC, n - 1, dS, n - 1, s, rs::WaveOptions{});
      if (st != ROT_OK) break;
      if (cudaMemcpy2DAsync(A_host, lda * sizeof(double), dA, m * sizeof(double), m * sizeof(double), n,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess) st = ROT_ECUDA;
      break;
    }
    rs::WaveOptions o;
    o.arrived = arrived;
    o.arrive_cols = cols;
    o.last_done = last_done;
    st = rs::wave_apply<double>(m, n, k, dA, m, dC, n - 1, dS, n - 1, s, o);
    // Whatever happened to the kernel, release the copy stream's waits.
    rs::fill_kernel<<<1, 256, 0, s>>>(last_done, b_last, pl.nchains);
    rs::count_launches(1);
    if (st != ROT_OK) break;
    // Downloads: chunk i once its last column (c1 - 1) is final in every
    // chain, i.e. after wave c1 - 1 + kr_last - 1 of the last p-block.
    for (int i = 0; i < nchunks && st == ROT_OK; ++i) {
      const int64_t c0 = (int64_t)i * cols, c1 = std::min<int64_t>(n, c0 + cols);
      if (c0 >= c1) continue;
      const int wb = (int)std::min<int64_t>(b_last - 1, (c1 - 1 + kr_last - 1) / pl.NB);
      const CUresult wr = ops.wait(sc, (CUdeviceptr)(last_done + wb), (cuuint32_t)pl.nchains,
                                   CU_STREAM_WAIT_VALUE_GEQ);
      if (wr != CUDA_SUCCESS) {
        char msg[96];
        snprintf(msg, sizeof msg, "rot_apply_host: stream wait refused (CUresult %d)", (int)wr);
        rs::note_error(msg);
        st = ROT_ECUDA;
      } else if (cudaMemcpy2DAsync(A_host + c0 * lda, lda * sizeof(double), dA + c0 * m, m * sizeof(double),
                                   m * sizeof(double), c1 - c0, cudaMemcpyDeviceToHost, sc) != cudaSuccess) {
        st = rs::cuda_failed(cudaGetLastError(), "rot_apply_host: chunked download");
      }
    }
    if (st != ROT_OK) break;
  } while (0);
  // The buffers are freed on `s` after the copy stream's work.
  if (sc && copied) {
    if (cudaEventRecord(copied, sc) != cudaSuccess || cudaStreamWaitEvent(s, copied, 0) != cudaSuccess) {
      cudaStreamSynchronize(sc);
      if (st == ROT_OK) st = ROT_ECUDA;
    }
  }
  cudaFreeAsync(dA, s);
  cudaFreeAsync(dC, s);
  cudaFreeAsync(dS, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == ROT_OK) st = ROT_ECUDA;
  if (ready) cudaEventDestroy(ready);
  if (copied) cudaEventDestroy(copied);
  return st;
}
