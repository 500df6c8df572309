// rs_api.cu -- the extern "C" entry points declared in include/rotseq.h:
// argument validation, quick returns, dispatch to the kernels.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#include "rs_internal.h"
#include "rs_device.cuh"

namespace {

constexpr int64_t kLimit = (int64_t(1) << 31) - 1;

rot_status validate(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda, const void* C,
                    int64_t ldc, const void* S, int64_t lds, bool* quick) {
  *quick = false;
  if (m < 0 || n < 0 || k < 0) return ROT_EINVAL;
  if (m > kLimit || n > kLimit || k > kLimit || n + k > kLimit) return ROT_EINVAL;
  if (lda < (m > 1 ? m : 1)) return ROT_EINVAL;
  const int64_t nm1 = n - 1 > 1 ? n - 1 : 1;
  if (ldc < nm1 || lds < nm1) return ROT_EINVAL;
  if (m == 0 || n <= 1 || k == 0) {
    *quick = true;
    return ROT_OK;
  }
  if (!A || !C || !S) return ROT_EINVAL;
  return ROT_OK;
}

}  // namespace

extern "C" {

int rot_version(void) { return 100; }

const char* rot_status_string(rot_status s) {
  switch (s) {
    case ROT_OK: return "ROT_OK";
    case ROT_EINVAL: return "ROT_EINVAL: invalid argument";
    case ROT_ECUDA: return "ROT_ECUDA: CUDA error";
    case ROT_ENOMEM: return "ROT_ENOMEM: out of device memory";
    case ROT_ETIMEOUT: return "ROT_ETIMEOUT: a bounded wait ran out";
    case ROT_EBUSY: return "ROT_EBUSY: resource busy";
    case ROT_EUNSUPPORTED: return "ROT_EUNSUPPORTED: not supported on this device";
  }
  return "ROT_?: unknown status";
}

rot_status rot_apply(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                     int64_t ldc, const double* S, int64_t lds, void* stream) {
  bool quick;
  rot_status v = validate(m, n, k, A, lda, C, ldc, S, lds, &quick);
  if (v != ROT_OK || quick) return v;
  return rs::apply_f64(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream));
}

rot_status rot_apply_f32(int64_t m, int64_t n, int64_t k, float* A, int64_t lda, const float* C,
                         int64_t ldc, const float* S, int64_t lds, void* stream) {
  bool quick;
  rot_status v = validate(m, n, k, A, lda, C, ldc, S, lds, &quick);
  if (v != ROT_OK || quick) return v;
  // 16 to 55 sequences: the warp chain, eight warps per 32-row strip (k mod 8
  // on the column stream after it; measured at 8192 x 8192: k = 32 0.81 ms
  // against 1.36 for stream passes of 8, k = 48 1.03 against 1.82 for the
  // lane pipeline).  Otherwise the column stream up to 41 sequences, the
  // lane pipeline beyond (where each applies), the wavefront kernel
  // otherwise.  With at most 4096 rows the stream has few warps (one per
  // 32 rows) and the pipeline takes over from 20 sequences (measured: 4096 x
  // 4096, k = 32: 0.48 ms against 0.77; 2048 x 2048, k = 24: about 0.33
  // against 0.39).
  if (rs::chain_f32_fits(m, n, k, A, lda))
    return rs::chain_apply_f32(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream));
  const int64_t stream_max = m <= 4096 ? 19 : 41;
  if (k <= stream_max && rs::stream_fits<float>(m, n, k, A, lda))
    return rs::stream_apply<float>(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream));
  if (rs::pipe_f32_fits(m, n, k))
    return rs::pipe_apply_f32(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream));
  if (rs::stream_fits<float>(m, n, k, A, lda))
    return rs::stream_apply<float>(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream));
  return rs::wave_apply_f32(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream),
                            rs::WaveOptions{});
}

rot_status rot_apply_tuned(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* C,
                           int64_t ldc, const double* S, int64_t lds, const rot_tuning* tuning, void* stream) {
  bool quick;
  rot_status v = validate(m, n, k, A, lda, C, ldc, S, lds, &quick);
  if (v != ROT_OK || quick) return v;
  rs::WaveOptions o{};
  if (tuning) {
    if (tuning->K < 0 || tuning->K > 16 || tuning->NB < 0 || tuning->NB > 4096 || tuning->ctas_per_sm < 0 ||
        tuning->fp64_products < 0 || tuning->fp64_products > 2)
      return ROT_EINVAL;
    o.K = tuning->K;
    o.NB = tuning->NB;
    o.ctas_per_sm = tuning->ctas_per_sm;
    o.fp64_products = tuning->fp64_products;
  }
  return rs::wave_apply<double>(m, n, k, A, lda, C, ldc, S, lds, static_cast<cudaStream_t>(stream), o);
}

rot_status rot_apply_reflectors(int64_t m, int64_t n, int64_t k, double* A, int64_t lda, const double* T,
                               int64_t ldt, const double* V, int64_t ldv, void* stream) {
  bool quick;
  rot_status v = validate(m, n, k, A, lda, T, ldt, V, ldv, &quick);
  if (v != ROT_OK || quick) return v;
  rs::WaveOptions o{};
  o.reflectors = true;
  return rs::wave_apply<double>(m, n, k, A, lda, T, ldt, V, ldv, static_cast<cudaStream_t>(stream), o);
}

rot_status rot_selftest_wait_timeout(int wait_ms, void* stream) {
  if (wait_ms < 1 || wait_ms > 10000) return ROT_EINVAL;
  int dev_status = 0;
  const rot_status st = rs::selftest_dependency_timeout(wait_ms, static_cast<cudaStream_t>(stream), &dev_status);
  if (st != ROT_OK) return st;
  return dev_status == rs::kDevTimeoutDependency ? rot_device_code_status(dev_status) : ROT_ECUDA;
}

rot_status rot_device_status(void) {
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return rs::cuda_failed(e, "rot_device_status: cudaDeviceSynchronize");
  const int s = rs::take_sticky_status();
  if (s < 0) {
    rs::note_error("rot_device_status: reading the sticky device status failed");
    return ROT_ECUDA;
  }
  return rot_device_code_status(s);
}

rot_status rot_device_code_status(int code) {
  switch (code) {
    case rs::kDevOk: return ROT_OK;
    case rs::kDevTimeoutDependency:
      rs::note_error("device: a wait on another work item's progress ran out");
      return ROT_ETIMEOUT;
    case rs::kDevTimeoutTma:
      rs::note_error("device: a wait on a (c,s) tile copy ran out");
      return ROT_ETIMEOUT;
    case rs::kDevBadItem:
      rs::note_error("device: a work item decoded outside the problem (internal error)");
      return ROT_ECUDA;
    case rs::kDevCancelled:
      rs::note_error("device: the launch was cancelled by the host");
      return ROT_ECUDA;
    default: {
      char buf[96];
      snprintf(buf, sizeof buf, "device: unknown status code %d", code);
      rs::note_error(buf);
      return ROT_ECUDA;
    }
  }
}

}  // extern "C"
