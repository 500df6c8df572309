// rs_tune.cu -- autotuner for the batched wavefront launch.
//
// The tiling choices (sequences per item K, waves per item NB, resident CTAs
// per SM) trade pipeline fill and drain against per-item overhead, and the
// best point depends on the mix of shapes in a batch.  The autotuner times a
// small grid of candidates on scratch copies of the batch and caches the
// winner under a signature of the batch's shapes and the device.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "rs_internal.h"

namespace rs {
namespace {

std::mutex g_mu;
std::map<std::string, rot_tuning> g_cache;
bool g_file_loaded = false;

int log2_bucket(double x) { return x <= 1 ? 0 : (int)std::lround(std::log2(x)); }

// Shape signature: device, number of problems with work, and log2 buckets of
// total rotation-rows, largest n, mean m and mean k.
std::string signature(int count, const rot_problem* probs) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  double rows = 0, msum = 0, ksum = 0, nmax = 0;
  int used = 0;
  for (int i = 0; i < count; ++i) {
    const rot_problem& q = probs[i];
    if (q.m <= 0 || q.n <= 1 || q.k <= 0) continue;
    ++used;
    rows += (double)q.m * (q.n - 1) * q.k;
    msum += (double)q.m;
    ksum += (double)q.k;
    nmax = std::max(nmax, (double)q.n);
  }
  char buf[160];
  snprintf(buf, sizeof buf, "sm%d:c%d:w%d:n%d:m%d:k%d", nsm, used, log2_bucket(rows), log2_bucket(nmax),
           log2_bucket(used ? msum / used : 0), log2_bucket(used ? ksum / used : 0));
  return buf;
}

void load_file_locked() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = std::getenv("ROTSEQ_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[160];
  rot_tuning t;
  t.fp64_products = 0;
  while (std::fscanf(f, "%159s %d %d %d", key, &t.K, &t.NB, &t.ctas_per_sm) == 4) g_cache[key] = t;
  std::fclose(f);
}

void store_locked(const std::string& key, const rot_tuning& t) {
  g_cache[key] = t;
  const char* path = std::getenv("ROTSEQ_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d\n", key.c_str(), t.K, t.NB, t.ctas_per_sm);
  std::fclose(f);
}

}  // namespace

void tuning_lookup(int count, const rot_problem* problems, rot_tuning* out) {
  *out = rot_tuning{0, 0, 0, 0};
  if (count <= 0 || !problems) return;
  const std::string key = signature(count, problems);
  std::lock_guard<std::mutex> lk(g_mu);
  load_file_locked();
  auto it = g_cache.find(key);
  if (it != g_cache.end()) *out = it->second;
}

}  // namespace rs

extern "C" rot_status rot_batch_autotune(int count, const rot_problem* problems, void* stream,
                                         rot_tuning* best, float* best_ms) {
  if (!best || count < 0 || (count > 0 && !problems)) return ROT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Scratch copies of every A so the caller's data is left as it is.
  std::vector<rot_problem> copy(problems, problems + count);
  std::vector<void*> bufs;
  rot_status st = ROT_OK;
  for (int i = 0; i < count && st == ROT_OK; ++i) {
    rot_problem& q = copy[i];
    if (q.m <= 0 || q.n <= 1 || q.k <= 0 || !q.A) continue;
    void* d = nullptr;
    const size_t bytes = (size_t)q.lda * (size_t)(q.n - 1) * sizeof(double) + (size_t)q.m * sizeof(double);
    if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); st = ROT_ENOMEM; break; }
    bufs.push_back(d);
    if (cudaMemcpyAsync(d, q.A, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = ROT_ECUDA;
    q.A = static_cast<double*>(d);
  }
  const int Ks[] = {4, 8, 16};
  const int NBs[] = {32, 64, 128};
  const int Cs[] = {1, 2};
  float best_t = -1.f;
  rot_tuning bt{16, 32, 0, 0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == ROT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = ROT_ECUDA;
  for (int K : Ks) {
    for (int NB : NBs) {
      for (int C : Cs) {
        if (st != ROT_OK) break;
        rot_tuning t{K, NB, C, 0};
        rot_batch_plan* plan = nullptr;
        st = rot_batch_plan_create(count, copy.data(), &t, &plan);
        if (st != ROT_OK) break;
        st = rot_batch_plan_execute(plan, stream);  // warm-up
        cudaEventRecord(e0, s);
        const int reps = 2;
        for (int r = 0; r < reps && st == ROT_OK; ++r) st = rot_batch_plan_execute(plan, stream);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          st = ROT_ECUDA;
        rot_status d = rot_batch_plan_destroy(plan);
        if (st == ROT_OK) st = d;
        ms /= reps;
        if (st == ROT_OK && (best_t < 0 || ms < best_t)) {
          best_t = ms;
          bt = t;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  for (void* d : bufs) cudaFree(d);
  if (st != ROT_OK) return st;
  const rot_status dev = rot_device_status();
  if (dev != ROT_OK) return dev;
  *best = bt;
  if (best_ms) *best_ms = best_t;
  {
    std::lock_guard<std::mutex> lk(rs::g_mu);
    rs::load_file_locked();
    rs::store_locked(rs::signature(count, problems), bt);
  }
  return ROT_OK;
}
