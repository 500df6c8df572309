// rs_batch.cu -- many independent FP64 problems in one persistent launch.
//
// A batch plan holds, in one device workspace: the instance descriptors, one
// TMA descriptor per instance, the segment table that orders every instance's
// work items by wavefront key, the dependency counters and the repacked (c,s)
// rows of every instance.  Executing a plan only enqueues kernels (clear the
// counters, repack C/S, the persistent wave kernel, fold the status), so it
// can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>
#include <cuda.h>

#include "rs_batch.h"

namespace rs {

namespace {

constexpr int kKMAX = 16;
constexpr int kNBT = 16;
constexpr int kWarps = 8;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Where one instance's C and S are and where its repacked rows go.
struct RepackDesc {
  const double* C;
  const double* S;
  int64_t ldc, lds;
  double* out;
  int64_t W2;
  int n, k;
  int64_t count;  // (n-1) * k
};

// One launch repacks every instance: blockIdx.y is the instance, blockIdx.x
// strides over its (n-1)*k entries.
__global__ void repack_batch_kernel(const RepackDesc* __restrict__ d, int ninst) {
  const int i = blockIdx.y;
  if (i >= ninst) return;
  const RepackDesc r = d[i];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r.count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % (r.n - 1));
    const int p = (int)(e / (r.n - 1));
    double2 v;
    v.x = r.C[j + (int64_t)p * r.ldc];
    v.y = r.S[j + (int64_t)p * r.lds];
    *reinterpret_cast<double2*>(r.out + (int64_t)(j + p) * r.W2 + 2 * p) = v;
  }
}

int host_pairs_in_key(int kappa, int G, int B, int delta, int* g_lo) {
  int hi = kappa / delta;
  if (hi > G - 1) hi = G - 1;
  int lo = kappa - (B - 1);
  lo = lo <= 0 ? 0 : (lo + delta - 1) / delta;
  *g_lo = lo;
  return hi >= lo ? hi - lo + 1 : 0;
}

}  // namespace

rot_status batch_layout(int count, const rot_problem* probs, const rot_tuning& tu, BatchLayout* L) {
  const int64_t lim = (int64_t(1) << 31) - 1;
  for (int i = 0; i < count; ++i) {
    const rot_problem& q = probs[i];
    if (q.m < 0 || q.n < 0 || q.k < 0) return ROT_EINVAL;
    if (q.m > lim || q.n > lim || q.k > lim || q.n + q.k > lim) return ROT_EINVAL;
    if (q.lda < std::max<int64_t>(1, q.m)) return ROT_EINVAL;
    const int64_t nm1 = std::max<int64_t>(1, q.n - 1);
    if (q.ldc < nm1 || q.lds < nm1) return ROT_EINVAL;
    if (q.m == 0 || q.n <= 1 || q.k == 0) continue;  // quick return: nothing to do
    if (!q.A || !q.C || !q.S) return ROT_EINVAL;
    L->idx.push_back(i);
  }
  const int ni = (int)L->idx.size();
  if (ni > 65535) return ROT_EINVAL;  // one grid row per instance in the repack launch
  L->wp.resize(ni);
  L->cs_off.resize(ni);
  L->done_off.resize(ni);
  int max_key = 0;
  for (int t = 0; t < ni; ++t) {
    const rot_problem& q = probs[L->idx[t]];
    const WavePlan pl = plan_wave(q.m, q.n, q.k, kKMAX, kNBT, tu.K, tu.NB, 8);
    L->wp[t] = pl;
    L->done_off[t] = L->done_ints;
    L->done_ints += (size_t)pl.nchains * pl.G;
    L->cs_off[t] = L->cs_bytes;
    L->cs_bytes += round_up((int64_t)pl.cs_rows * 2 * pl.kpad * 8, 256);
    L->rotation_rows += q.m * (q.n - 1) * q.k;
    max_key = std::max(max_key, (pl.B - 1) + pl.delta * (pl.G - 1));
  }
  // Segment table: keys in increasing order, instances in order within a key.
  for (int kappa = 0; kappa <= max_key && ni > 0; ++kappa) {
    long long in_key = 0;
    for (int t = 0; t < ni; ++t) {
      int glo;
      const WavePlan& pl = L->wp[t];
      const int pairs = host_pairs_in_key(kappa, pl.G, pl.B, pl.delta, &glo);
      if (pairs <= 0) continue;
      L->seg.push_back(WaveSegment{L->tickets, t, kappa});
      L->tickets += (long long)pairs * pl.nchains;
      in_key += (long long)pairs * pl.nchains;
    }
    L->key_items_max = std::max(L->key_items_max, in_key);
  }
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = round_up(off, align);
    const size_t o = off;
    off += bytes;
    return o;
  };
  L->o_inst = take(sizeof(WaveInstance) * std::max(ni, 1), 256);
  L->o_tmap = take(sizeof(CUtensorMap) * std::max(ni, 1), 128);
  L->o_seg = take(sizeof(WaveSegment) * std::max<size_t>(L->seg.size(), 1), 256);
  L->o_rep = take(sizeof(RepackDesc) * std::max(ni, 1), 256);
  L->cnt_bytes = round_up(L->done_ints * sizeof(int), 256) + 256;
  L->o_cnt = take(L->cnt_bytes, 256);
  L->o_cs = take(L->cs_bytes, 1024);
  L->total = std::max<size_t>(off, 1024);
  return ROT_OK;
}

rot_status batch_image(const BatchLayout& L, const rot_problem* probs, unsigned char* base,
                       unsigned char* img, BatchLaunch* B) {
  const int ni = (int)L.idx.size();
  std::memset(img, 0, L.o_cs);
  WaveInstance* hi = reinterpret_cast<WaveInstance*>(img + L.o_inst);
  CUtensorMap* ht = reinterpret_cast<CUtensorMap*>(img + L.o_tmap);
  WaveSegment* hs = reinterpret_cast<WaveSegment*>(img + L.o_seg);
  RepackDesc* hr = reinterpret_cast<RepackDesc*>(img + L.o_rep);
  int* d_done = reinterpret_cast<int*>(base + L.o_cnt);
  int64_t max_count = 1;
  for (int t = 0; t < ni; ++t) {
    const rot_problem& q = probs[L.idx[t]];
    const WavePlan& pl = L.wp[t];
    double* cs = reinterpret_cast<double*>(base + L.o_cs + L.cs_off[t]);
    const int64_t W2 = 2 * (int64_t)pl.kpad;
    if (!encode_tile_map_2d(&ht[t], cs, true, (uint64_t)W2, (uint64_t)pl.cs_rows,
                            (uint64_t)W2 * sizeof(double), 2 * kKMAX, kNBT))
      return ROT_ECUDA;
    WaveInstance I{};
    I.A = q.A; I.lda = q.lda; I.m = (int)q.m; I.n = (int)q.n; I.k = (int)q.k;
    I.K = pl.K; I.NB = pl.NB; I.delta = pl.delta; I.nchains = pl.nchains; I.G = pl.G; I.B = pl.B;
    I.cs_row0 = 0;
    set_full_range(I);
    I.done = d_done + L.done_off[t];
    I.tmap = reinterpret_cast<const CUtensorMap*>(base + L.o_tmap) + t;
    hi[t] = I;
    hr[t] = RepackDesc{q.C, q.S, q.ldc, q.lds, cs, W2, (int)q.n, (int)q.k, (q.n - 1) * q.k};
    max_count = std::max<int64_t>(max_count, hr[t].count);
  }
  for (size_t i = 0; i < L.seg.size(); ++i) hs[i] = L.seg[i];

  B->count = ni;
  B->base = base;
  B->bytes = L.total;
  B->d_inst = reinterpret_cast<WaveInstance*>(base + L.o_inst);
  B->d_seg = reinterpret_cast<WaveSegment*>(base + L.o_seg);
  B->d_rep = base + L.o_rep;
  B->d_counters = base + L.o_cnt;
  B->counters_bytes = L.cnt_bytes;
  B->launch.ticket = reinterpret_cast<unsigned long long*>(base + L.o_cnt +
                                                           round_up(L.done_ints * sizeof(int), 256));
  B->launch.status = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(B->launch.ticket) + 64);
  B->launch.total = L.tickets;
  B->nseg = (int)L.seg.size();
  B->total = L.tickets;
  B->rotation_rows = L.rotation_rows;
  B->key_items_max = L.key_items_max;
  B->repack_grid_x = (int)std::min<int64_t>(ceil_div(max_count, 256), 1024);
  return ROT_OK;
}

// The two instantiations of the batched kernel: FP64 products on the FP64
// pipe or on the integer pipe (bit-identical results).
static auto batched_fn(bool intmul) {
  return intmul ? wave_batched_kernel<double, kKMAX, kNBT, kWarps, kOpRotateIntmul>
                : wave_batched_kernel<double, kKMAX, kNBT, kWarps, kOpRotate>;
}

rot_status batch_prepare(BatchLaunch* B) {
  const bool intmul = B->tuning.fp64_products == 2 ||
                      (B->tuning.fp64_products == 0 && kDefaultFp64Products == 2);
  B->intmul = intmul;
  auto kfn = batched_fn(intmul);
  const int smem = kWarps * WaveSmem<double, kKMAX, kNBT>::kWarpBytes;
  cudaError_t e = cudaGetDevice(&B->device);
  if (e != cudaSuccess) return cuda_failed(e, "batch_prepare: cudaGetDevice");
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_failed(e, "batch_prepare: cudaFuncSetAttribute");
  int nsm = 0, occ = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem);
  if (e != cudaSuccess) return cuda_failed(e, "batch_prepare: occupancy");
  if (occ < 1) return cuda_failed(cudaErrorInvalidConfiguration, "batch_prepare: occupancy 0");
  const int per_sm = B->tuning.ctas_per_sm > 0 ? std::min(B->tuning.ctas_per_sm, occ) : occ;
  long long grid = (long long)nsm * per_sm;
  // Warps beyond ~1.5 per item of the busiest key would only wait on
  // dependencies; leave their SMs to other launches.  (0: not known, no cap.)
  if (B->key_items_max > 0) {
    const long long useful = (3 * B->key_items_max + 1) / 2;
    grid = std::min<long long>(grid, (useful + kWarps - 1) / kWarps);
  }
  grid = std::min<long long>(grid, (B->total + kWarps - 1) / kWarps);
  B->grid = (int)std::max<long long>(grid, 1);
  B->smem = smem;
  return ROT_OK;
}

rot_status batch_resident_warps(long long* warps) {
  auto kfn = batched_fn(kDefaultFp64Products == 2);
  const int smem = kWarps * WaveSmem<double, kKMAX, kNBT>::kWarpBytes;
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_failed(e, "batch_resident_warps: cudaGetDevice");
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_failed(e, "batch_resident_warps: cudaFuncSetAttribute");
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kWarps * 32, smem);
  if (e != cudaSuccess) return cuda_failed(e, "batch_resident_warps: occupancy");
  *warps = (long long)nsm * std::max(occ, 1) * kWarps;
  return ROT_OK;
}

int batch_pick_K(int count, const rot_problem* probs, long long warps) {
  for (int K : {16, 8}) {
    long long items = 0;
    for (int i = 0; i < count; ++i) {
      const rot_problem& q = probs[i];
      if (q.m <= 0 || q.n <= 1 || q.k <= 0) continue;
      items += ceil_div(q.m, 32) * ceil_div(q.k, K);
    }
    if (items >= warps) return K;
  }
  return 4;
}

rot_status batch_launch_kernel(const BatchLaunch& B, cudaStream_t s, int trace_kind, long long work) {
  auto kfn = batched_fn(B.intmul);
  const int tr = trace_begin(trace_kind, work, s);
  kfn<<<(unsigned)B.grid, kWarps * 32, B.smem, s>>>(B.d_inst, B.d_seg, B.nseg, B.launch);
  trace_end(tr, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_failed(e, "wave_batched_kernel launch");
  record_status_async(B.launch.status, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_failed(e, "status kernel launch");
  count_launches(2);
  return ROT_OK;
}

rot_status batch_enqueue(const BatchLaunch& B, cudaStream_t s) {
  if (B.count == 0) return ROT_OK;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != B.device) return ROT_EINVAL;
  if (cudaMemsetAsync(B.d_counters, 0, B.counters_bytes, s) != cudaSuccess) return ROT_ECUDA;
  dim3 rg(B.repack_grid_x, B.count);
  repack_batch_kernel<<<rg, 256, 0, s>>>(static_cast<const RepackDesc*>(B.d_rep), B.count);
  if (cudaGetLastError() != cudaSuccess) return ROT_ECUDA;
  const rot_status st = batch_launch_kernel(B, s, ROT_KERNEL_WAVE_BATCHED, B.rotation_rows);
  if (st != ROT_OK) return st;
  count_launches(1);
  return ROT_OK;
}

}  // namespace rs

struct rot_batch_plan_s {
  rs::BatchLaunch p;   // p.base is the plan's own workspace
};

extern "C" {

rot_status rot_batch_plan_create(int count, const rot_problem* problems, const rot_tuning* tuning,
                                 rot_batch_plan** out) {
  if (!out || count < 0 || (count > 0 && !problems)) return ROT_EINVAL;
  *out = nullptr;
  // Validate everything before touching the device.
  {
    rs::BatchLayout probe;
    rot_status v = rs::batch_layout(count, problems, rot_tuning{0, 0, 0}, &probe);
    if (v != ROT_OK) return v;
  }
  rot_tuning tu{};
  if (tuning) tu = *tuning;
  else rs::tuning_lookup(count, problems, &tu);
  if (tu.K < 0 || tu.K > 16 || tu.NB < 0 || tu.NB > 4096 || tu.ctas_per_sm < 0 || tu.fp64_products < 0 ||
      tu.fp64_products > 2)
    return ROT_EINVAL;
  rs::BatchLayout L;
  rot_status st = rs::batch_layout(count, problems, tu, &L);
  if (st != ROT_OK) return st;
  auto* h = new (std::nothrow) rot_batch_plan_s;
  if (!h) return ROT_ENOMEM;
  h->p.tuning = tu;
  if (cudaGetDevice(&h->p.device) != cudaSuccess) { delete h; return ROT_ECUDA; }
  if (!L.idx.empty()) {
    void* ws = nullptr;
    if (cudaMalloc(&ws, L.total) != cudaSuccess) { cudaGetLastError(); delete h; return ROT_ENOMEM; }
    std::vector<unsigned char> img(L.o_cs);
    st = rs::batch_image(L, problems, static_cast<unsigned char*>(ws), img.data(), &h->p);
    if (st == ROT_OK && cudaMemcpy(ws, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      st = ROT_ECUDA;
    if (st == ROT_OK) st = rs::batch_prepare(&h->p);
    if (st != ROT_OK) { cudaFree(ws); delete h; return st; }
  }
  h->p.bytes = L.total;
  *out = h;
  return ROT_OK;
}

rot_status rot_batch_plan_execute(rot_batch_plan* plan, void* stream) {
  if (!plan) return ROT_EINVAL;
  return rs::batch_enqueue(plan->p, static_cast<cudaStream_t>(stream));
}

rot_status rot_batch_plan_info(const rot_batch_plan* plan, rot_batch_info* info) {
  if (!plan || !info) return ROT_EINVAL;
  info->problems = plan->p.count;
  info->work_items = plan->p.total;
  info->rotation_rows = plan->p.rotation_rows;
  info->workspace_bytes = plan->p.bytes;
  info->tuning = plan->p.tuning;
  return ROT_OK;
}

rot_status rot_batch_plan_destroy(rot_batch_plan* plan) {
  if (!plan) return ROT_OK;
  rot_status st = ROT_OK;
  if (plan->p.base) {
    // The plan's workspace may still be in use by queued work.
    if (cudaDeviceSynchronize() != cudaSuccess) st = ROT_ECUDA;
    if (cudaFree(plan->p.base) != cudaSuccess) st = ROT_ECUDA;
  }
  delete plan;
  return st;
}

rot_status rot_batched_workspace_size(int count, const rot_problem* problems, size_t* bytes) {
  if (!bytes || count < 0 || (count > 0 && !problems)) return ROT_EINVAL;
  *bytes = 0;
  rot_tuning tu{};
  rs::tuning_lookup(count, problems, &tu);
  rs::BatchLayout L;
  rot_status st = rs::batch_layout(count, problems, tu, &L);
  if (st != ROT_OK) return st;
  *bytes = L.idx.empty() ? 0 : L.total;
  return ROT_OK;
}

rot_status rot_apply_batched_ws(int count, const rot_problem* problems, void* workspace, size_t workspace_bytes,
                                void* stream) {
  if (count < 0 || (count > 0 && !problems)) return ROT_EINVAL;
  rot_tuning tu{};
  rs::tuning_lookup(count, problems, &tu);
  rs::BatchLayout L;
  rot_status st = rs::batch_layout(count, problems, tu, &L);
  if (st != ROT_OK) return st;
  if (L.idx.empty()) return ROT_OK;
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return ROT_EINVAL;
  unsigned char* base = static_cast<unsigned char*>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rs::BatchLaunch B;
  B.tuning = tu;
  if (cudaGetDevice(&B.device) != cudaSuccess) return ROT_ECUDA;
  std::vector<unsigned char> img(L.o_cs);
  st = rs::batch_image(L, problems, base, img.data(), &B);
  if (st != ROT_OK) return st;
  // From pageable memory the copy is staged before the call returns, so the
  // host image may go out of scope; the kernels that read it follow in order.
  if (cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return rs::cuda_failed(cudaGetLastError(), "rot_apply_batched_ws: descriptor upload");
  st = rs::batch_prepare(&B);
  if (st != ROT_OK) return st;
  return rs::batch_enqueue(B, s);
}

rot_status rot_apply_batched(int count, const rot_problem* problems, void* stream) {
  rot_batch_plan* plan = nullptr;
  rot_status st = rot_batch_plan_create(count, problems, nullptr, &plan);
  if (st != ROT_OK) return st;
  st = rot_batch_plan_execute(plan, stream);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && st == ROT_OK) st = ROT_ECUDA;
  rot_status d = rot_batch_plan_destroy(plan);
  return st != ROT_OK ? st : d;
}

}  // extern "C"
