// rs_server.cu -- continuous-batching server for rotation-sequence requests.
//
// Clients register matrices that stay resident on the device and submit
// requests (a matrix handle plus the k sequences of rotations, C and S, from
// host memory).  A scheduler thread admits pending requests while request
// slots and workspace memory (an arena carved once out of the HBM budget) are
// free, batches everything it admits in one scheduling step into a single
// launch of the batched wavefront kernel, and issues that launch on a free
// stream.  Requests that arrive while earlier launches run are admitted as
// slots and memory free up and go out on another stream, so their work
// overlaps on the device.  Requests on the same matrix keep their submission
// order (a matrix is never in two launches at once).  Completion is reported
// by a host callback queued behind each launch (cudaLaunchHostFunc), which
// also stamps the completion time used for latency statistics.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>

#include "rs_batch.h"

namespace rs {

struct Server;

namespace {

using Clock = std::chrono::steady_clock;
inline double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, cap) in 256-byte units of one device buffer.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(std::max<size_t>(bytes, 256));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(std::max<size_t>(bytes, 256));
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }

 private:
  size_t cap_, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Matrix {
  int64_t m, n, lda;
  double* A;
  bool busy = false;
  bool wide = false;   // its launches can fill much of the GPU (see Server::wide_rows)
};

struct Request {
  uint64_t ticket = 0;
  int handle = 0;
  int64_t k = 0;
  std::vector<double> cs;   // C then S, each (n-1) x k compact
  double t_submit = 0, t_done = 0;
  int status = ROT_OK;
  bool done = false;
  int64_t rotation_rows = 0;
};

struct Launch;

struct Slot {
  cudaStream_t stream = nullptr;
  unsigned char* staging = nullptr;   // pinned
  size_t staging_bytes = 0;
  bool busy = false;
};

struct Launch {
  Server* srv = nullptr;
  int slot = -1;
  size_t arena_off = 0, arena_bytes = 0;
  std::vector<std::shared_ptr<Request>> reqs;
  volatile int* status_host = nullptr;  // pinned copy of the launch's device status
  bool wide = false;                    // a launch over wide matrices
};

}  // namespace

struct Server {
  rot_server_config cfg{};
  int device = 0;
  unsigned char* arena_base = nullptr;
  std::unique_ptr<Arena> arena;
  std::vector<Slot> slots;
  std::vector<Matrix> mats;

  std::mutex mu;
  std::condition_variable cv_sched;   // wakes the scheduler
  std::condition_variable cv_done;    // wakes waiters
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> live;  // submitted, not yet waited on
  std::vector<Launch*> finished;      // completed launches, released by the scheduler
  uint64_t next_ticket = 1;
  long long warps = 1;                // resident warps of the batched kernel on this device
  // Launch classes.  A matrix with at least wide_rows rows is "wide": its
  // launch can keep most SMs busy for milliseconds.  Launches never mix the
  // classes (a request completes with its whole launch, so a small request
  // in a wide launch would wait for the large ones); at most one wide launch
  // is in flight, and it runs one CTA per SM (enough to keep the FP64 pipe
  // busy), so the other CTA slot of every SM stays open for narrow launches
  // arriving meanwhile.
  int64_t wide_rows = 2048;           // rows from which a matrix is wide (rot_server_config)
  bool wide_inflight = false;
  int inflight = 0;                   // requests admitted and not completed
  bool stop = false;
  std::thread thread;

  // statistics
  std::vector<double> latencies;
  int64_t completed = 0, rejected = 0, launches = 0, batched_requests = 0;
  int64_t rotation_rows = 0;
  double t_first = -1, t_last = 0;
};

namespace {

void CUDART_CB on_launch_done(void* p) {
  Launch* L = static_cast<Launch*>(p);
  Server* S = L->srv;
  const double t = now_s();
  const int st = *L->status_host;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& r : L->reqs) {
      r->t_done = t;
      r->status = st == kDevOk ? ROT_OK
                  : (st == kDevTimeoutDependency || st == kDevTimeoutTma) ? ROT_ETIMEOUT : ROT_ECUDA;
      r->done = true;
      S->latencies.push_back(t - r->t_submit);
      S->completed += 1;
      S->rotation_rows += r->rotation_rows;
      S->t_last = t;
      S->inflight -= 1;
      S->mats[r->handle].busy = false;
    }
    if (L->wide) S->wide_inflight = false;
    S->finished.push_back(L);
  }
  S->cv_done.notify_all();
  S->cv_sched.notify_one();
}

// Release what completed launches held (called by the scheduler, lock held).
void reap_locked(Server* S) {
  for (Launch* L : S->finished) {
    S->arena->release(L->arena_off, L->arena_bytes);
    S->slots[L->slot].busy = false;
    delete L;
  }
  S->finished.clear();
}

// Requests on one matrix that go out together as one problem.  Their
// sequences are concatenated in submission order: Algorithm 2 applies every
// rotation of sequence p before any of sequence p+1, so applying request r1
// and then r2 is the same computation, in the same order for every element,
// as one request holding r1's sequences followed by r2's.
struct Group {
  int handle = -1;
  int64_t k = 0;
  std::vector<std::shared_ptr<Request>> reqs;
};

// Device bytes a launch over these groups needs (layout + compact C/S).
bool size_launch(Server* S, const std::vector<Group>& gs, BatchLayout* L, std::vector<rot_problem>* probs,
                 size_t* cs_region, size_t* total) {
  probs->clear();
  size_t cs = 0;
  for (const Group& g : gs) {
    const Matrix& M = S->mats[g.handle];
    rot_problem q{};
    q.m = M.m; q.n = M.n; q.k = g.k; q.A = M.A; q.lda = M.lda;
    q.C = reinterpret_cast<const double*>(0x100);  // placeholders until the arena offset is known
    q.S = reinterpret_cast<const double*>(0x100);
    q.ldc = std::max<int64_t>(1, M.n - 1);
    q.lds = q.ldc;
    probs->push_back(q);
    cs += align256(2 * (size_t)(M.n - 1) * (size_t)g.k * sizeof(double));
  }
  // A launch with few work items per key uses short p-blocks, so that even a
  // lone large request keeps the whole GPU busy (its latency is the tail).
  rot_tuning tu{};
  // A wide launch runs one CTA per SM: half the resident warps.
  const bool wide = !gs.empty() && S->mats[gs[0].handle].wide;
  tu.K = batch_pick_K((int)probs->size(), probs->data(), wide ? S->warps / 2 : S->warps);
  *L = BatchLayout{};
  if (batch_layout((int)probs->size(), probs->data(), tu, L) != ROT_OK) return false;
  *cs_region = align256(L->total);
  *total = *cs_region + cs;
  return true;
}

void scheduler(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    reap_locked(S);
    if (S->stop && S->pending.empty() && S->inflight == 0) break;
    // ---- form one launch from the pending queue, in submission order -------
    // Every matrix that is not busy contributes the longest run of its
    // pending requests that fits (slots, batch size, fused length); a matrix
    // is never in two launches at once, so its requests keep their order.
    int free_slot = -1;
    for (size_t i = 0; i < S->slots.size(); ++i)
      if (!S->slots[i].busy) { free_slot = (int)i; break; }
    std::vector<Group> groups;
    int nreq = 0;
    int launch_wide = -1;   // class of the launch being formed (-1: not yet known)
    if (free_slot >= 0 && !S->pending.empty()) {
      std::vector<int> gidx(S->mats.size(), -1);
      std::vector<char> blocked(S->mats.size(), 0);
      for (auto it = S->pending.begin(); it != S->pending.end();) {
        auto& r = *it;
        const int h = r->handle;
        bool can = !blocked[h] && !S->mats[h].busy && S->inflight + nreq < S->cfg.max_inflight &&
                   nreq < S->cfg.max_batch;
        // The launch takes the class of its first request; a wide launch only
        // while no other wide launch runs.
        if (can && launch_wide < 0 && S->mats[h].wide && S->wide_inflight) can = false;
        if (can && launch_wide >= 0 && (int)S->mats[h].wide != launch_wide) can = false;
        if (can && launch_wide < 0) launch_wide = S->mats[h].wide ? 1 : 0;
        if (can && gidx[h] >= 0 && S->cfg.max_fused_k > 0 && groups[gidx[h]].k + r->k > S->cfg.max_fused_k)
          can = false;
        if (!can) {
          blocked[h] = 1;   // later requests on this matrix keep their order
          ++it;
          continue;
        }
        if (gidx[h] < 0) {
          gidx[h] = (int)groups.size();
          groups.push_back(Group{});
          groups.back().handle = h;
        }
        groups[gidx[h]].k += r->k;
        groups[gidx[h]].reqs.push_back(r);
        ++nreq;
        it = S->pending.erase(it);
      }
    }
    if (groups.empty()) {
      if (S->stop && S->pending.empty() && S->inflight == 0) break;
      S->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    // ---- fit the launch in the arena, returning requests if memory is short -
    // The last request of the last group goes back first, so a group shrinks
    // to the run of its matrix's requests that fits.
    BatchLayout L;
    std::vector<rot_problem> probs;
    size_t cs_region = 0, total = 0, off = 0;
    while (!groups.empty()) {
      if (size_launch(S, groups, &L, &probs, &cs_region, &total) && S->arena->alloc(total, &off)) break;
      Group& g = groups.back();
      S->pending.push_front(g.reqs.back());  // back to the queue
      g.k -= g.reqs.back()->k;
      g.reqs.pop_back();
      --nreq;
      if (g.reqs.empty()) groups.pop_back();
    }
    // Restore submission order in the queue (ticket order).
    std::sort(S->pending.begin(), S->pending.end(),
              [](const std::shared_ptr<Request>& a, const std::shared_ptr<Request>& b) {
                return a->ticket < b->ticket;
              });
    if (groups.empty()) {                   // nothing fits now: wait for memory
      S->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    std::vector<std::shared_ptr<Request>> all;
    for (auto& g : groups) {
      S->mats[g.handle].busy = true;
      all.insert(all.end(), g.reqs.begin(), g.reqs.end());
    }
    S->inflight += nreq;
    const bool wide = launch_wide == 1;
    if (wide) S->wide_inflight = true;
    Slot& slot = S->slots[free_slot];
    slot.busy = true;
    S->launches += 1;
    S->batched_requests += nreq;
    lk.unlock();

    // ---- build and enqueue the launch (no lock held) ------------------------
    unsigned char* base = S->arena_base + off;
    size_t coff = cs_region;
    std::vector<size_t> cs_at;
    for (size_t i = 0; i < groups.size(); ++i) {
      const size_t nm1k = (size_t)(probs[i].n - 1) * probs[i].k;
      probs[i].C = reinterpret_cast<const double*>(base + coff);
      probs[i].S = reinterpret_cast<const double*>(base + coff) + nm1k;
      cs_at.push_back(coff);
      coff += align256(2 * nm1k * sizeof(double));
    }
    const size_t stage_need = total + 256;
    rot_status st = ROT_OK;
    if (slot.staging_bytes < stage_need) {
      if (slot.staging) cudaFreeHost(slot.staging);
      slot.staging = nullptr;
      slot.staging_bytes = 0;
      if (cudaHostAlloc(&slot.staging, stage_need, cudaHostAllocDefault) != cudaSuccess) st = ROT_ENOMEM;
      else slot.staging_bytes = stage_need;
    }
    auto* launch = new Launch;
    launch->srv = S;
    launch->slot = free_slot;
    launch->arena_off = off;
    launch->arena_bytes = total;
    launch->reqs = all;
    launch->wide = wide;
    BatchLaunch B;
    if (st == ROT_OK) {
      launch->status_host = reinterpret_cast<volatile int*>(slot.staging + total);
      *launch->status_host = 0;
      st = batch_image(L, probs.data(), base, slot.staging, &B);
    }
    if (st == ROT_OK) {
      // Stage each group's C (then S) as the concatenation of its requests'.
      for (size_t i = 0; i < groups.size(); ++i) {
        const size_t nm1 = (size_t)(probs[i].n - 1);
        double* c_dst = reinterpret_cast<double*>(slot.staging + cs_at[i]);
        double* s_dst = c_dst + nm1 * (size_t)probs[i].k;
        for (auto& r : groups[i].reqs) {
          const size_t part = nm1 * (size_t)r->k;
          std::memcpy(c_dst, r->cs.data(), part * sizeof(double));
          std::memcpy(s_dst, r->cs.data() + part, part * sizeof(double));
          c_dst += part;
          s_dst += part;
          std::vector<double>().swap(r->cs);  // staged: the host copy is no longer needed
        }
      }
      B.device = S->device;
      if (wide) B.tuning.ctas_per_sm = 1;
      st = batch_prepare(&B);
    }
    cudaStream_t s = slot.stream;
    if (st == ROT_OK &&
        (cudaMemcpyAsync(base, slot.staging, L.o_cs, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(base + cs_region, slot.staging + cs_region, total - cs_region,
                         cudaMemcpyHostToDevice, s) != cudaSuccess))
      st = ROT_ECUDA;
    if (st == ROT_OK) st = batch_enqueue(B, s);
    if (st == ROT_OK &&
        cudaMemcpyAsync((void*)launch->status_host, B.launch.status, sizeof(int), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
      st = ROT_ECUDA;
    if (st == ROT_OK && cudaLaunchHostFunc(s, on_launch_done, launch) != cudaSuccess) st = ROT_ECUDA;
    if (st != ROT_OK) cudaStreamSynchronize(s);  // nothing of this launch may still be running
    lk.lock();
    if (st != ROT_OK) {
      // The launch could not be issued: finish its requests with the error.
      const double t = now_s();
      for (auto& r : all) {
        r->status = st;
        r->done = true;
        r->t_done = t;
        S->inflight -= 1;
        S->mats[r->handle].busy = false;
      }
      S->arena->release(off, total);
      slot.busy = false;
      if (wide) S->wide_inflight = false;
      delete launch;
      S->cv_done.notify_all();
    }
  }
}

}  // namespace
}  // namespace rs

struct rot_server_s {
  rs::Server s;
};

extern "C" {

rot_status rot_server_create(const rot_server_config* cfg, rot_server** out) {
  if (!out || !cfg) return ROT_EINVAL;
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->streams < 1 || cfg->streams > 64 ||
      cfg->max_batch < 1 || cfg->max_fused_k < 0)
    return ROT_EINVAL;
  auto* h = new (std::nothrow) rot_server_s;
  if (!h) return ROT_ENOMEM;
  rs::Server& S = h->s;
  S.cfg = *cfg;
  S.wide_rows = cfg->wide_rows > 0 ? cfg->wide_rows : cfg->wide_rows < 0 ? INT64_MAX : 2048;
  if (cudaGetDevice(&S.device) != cudaSuccess) { delete h; return ROT_ECUDA; }
  void* a = nullptr;
  if (cudaMalloc(&a, cfg->hbm_budget_bytes) != cudaSuccess) { cudaGetLastError(); delete h; return ROT_ENOMEM; }
  S.arena_base = static_cast<unsigned char*>(a);
  S.arena.reset(new rs::Arena(cfg->hbm_budget_bytes));
  if (rs::batch_resident_warps(&S.warps) != ROT_OK) {
    cudaFree(a);
    delete h;
    return ROT_ECUDA;
  }
  S.slots.resize(cfg->streams);
  for (auto& sl : S.slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& t : S.slots) if (t.stream) cudaStreamDestroy(t.stream);
      cudaFree(a);
      delete h;
      return ROT_ECUDA;
    }
  }
  S.thread = std::thread(rs::scheduler, &S);
  *out = h;
  return ROT_OK;
}

rot_status rot_server_register(rot_server* srv, int64_t m, int64_t n, double* A, int64_t lda, int* handle) {
  if (!srv || !handle || m < 1 || n < 2 || !A || lda < m) return ROT_EINVAL;
  if (m > (int64_t(1) << 31) - 1 || n > (int64_t(1) << 31) - 1) return ROT_EINVAL;
  std::lock_guard<std::mutex> lk(srv->s.mu);
  rs::Matrix M;
  M.m = m; M.n = n; M.lda = lda; M.A = A;
  M.wide = m >= srv->s.wide_rows;
  srv->s.mats.push_back(M);
  *handle = (int)srv->s.mats.size() - 1;
  return ROT_OK;
}

rot_status rot_server_submit(rot_server* srv, int handle, int64_t k, const double* C_host, int64_t ldc,
                             const double* S_host, int64_t lds, uint64_t* ticket) {
  if (!srv || !ticket || k < 1 || !C_host || !S_host) return ROT_EINVAL;
  rs::Server& S = srv->s;
  int64_t n = 0, m = 0;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (handle < 0 || handle >= (int)S.mats.size() || S.stop) return ROT_EINVAL;
    n = S.mats[handle].n;
    m = S.mats[handle].m;
  }
  if (ldc < n - 1 || lds < n - 1 || n + k > (int64_t(1) << 31) - 1) return ROT_EINVAL;
  auto r = std::make_shared<rs::Request>();
  r->handle = handle;
  r->k = k;
  r->rotation_rows = m * (n - 1) * k;
  const size_t nm1 = (size_t)(n - 1);
  r->cs.resize(2 * nm1 * (size_t)k);
  for (int64_t p = 0; p < k; ++p) {
    std::memcpy(&r->cs[p * nm1], C_host + p * ldc, nm1 * sizeof(double));
    std::memcpy(&r->cs[nm1 * k + p * nm1], S_host + p * lds, nm1 * sizeof(double));
  }
  // A request that cannot fit in the whole budget is refused now.
  {
    rs::BatchLayout L;
    std::vector<rot_problem> probs;
    size_t csr = 0, total = 0;
    std::vector<rs::Group> one(1);
    one[0].handle = handle;
    one[0].k = k;
    one[0].reqs.push_back(r);
    std::lock_guard<std::mutex> lk(S.mu);
    if (!rs::size_launch(&S, one, &L, &probs, &csr, &total) || total > S.arena->capacity()) {
      S.rejected += 1;
      return ROT_ENOMEM;
    }
    r->t_submit = rs::now_s();
    if (S.t_first < 0) S.t_first = r->t_submit;
    r->ticket = S.next_ticket++;
    *ticket = r->ticket;
    S.live[r->ticket] = r;
    S.pending.push_back(r);
  }
  S.cv_sched.notify_one();
  return ROT_OK;
}

rot_status rot_server_wait(rot_server* srv, uint64_t ticket, int timeout_ms) {
  return rot_server_wait_latency(srv, ticket, timeout_ms, nullptr);
}

rot_status rot_server_wait_latency(rot_server* srv, uint64_t ticket, int timeout_ms, double* latency_ms) {
  if (!srv) return ROT_EINVAL;
  rs::Server& S = srv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.live.find(ticket);
  if (it == S.live.end()) return ROT_EINVAL;
  std::shared_ptr<rs::Request> r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) S.cv_done.wait(lk, pred);
  else if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return ROT_ETIMEOUT;
  S.live.erase(ticket);
  if (latency_ms) *latency_ms = 1e3 * (r->t_done - r->t_submit);
  return (rot_status)r->status;
}

rot_status rot_server_stats(rot_server* srv, rot_server_stats_t* out, int reset) {
  if (!srv || !out) return ROT_EINVAL;
  rs::Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  std::vector<double> lat = S.latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(lat.size() - 1, std::ceil(q * lat.size()) - 1);
    return lat[i];
  };
  *out = rot_server_stats_t{};
  out->completed = S.completed;
  out->rejected = S.rejected;
  out->pending = (int64_t)S.pending.size();
  out->inflight = S.inflight;
  out->launches = S.launches;
  out->mean_batch = S.launches ? (double)S.batched_requests / S.launches : 0.0;
  out->p50_ms = 1e3 * pct(0.50);
  out->p99_ms = 1e3 * pct(0.99);
  out->max_ms = lat.empty() ? 0.0 : 1e3 * lat.back();
  out->rotation_rows = S.rotation_rows;
  out->busy_s = (S.t_first >= 0 && S.t_last > S.t_first) ? S.t_last - S.t_first : 0.0;
  out->rotation_rows_per_s = out->busy_s > 0 ? S.rotation_rows / out->busy_s : 0.0;
  out->arena_used_bytes = S.arena->used();
  if (reset) {
    S.latencies.clear();
    S.completed = S.rejected = S.launches = S.batched_requests = S.rotation_rows = 0;
    S.t_first = -1;
    S.t_last = 0;
  }
  return ROT_OK;
}

rot_status rot_server_destroy(rot_server* srv) {
  if (!srv) return ROT_OK;
  rs::Server& S = srv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.cv_sched.notify_one();
  if (S.thread.joinable()) S.thread.join();   // drains pending and in-flight requests
  rot_status st = ROT_OK;
  for (auto& sl : S.slots) {
    if (sl.stream) {
      if (cudaStreamSynchronize(sl.stream) != cudaSuccess) st = ROT_ECUDA;
      cudaStreamDestroy(sl.stream);
    }
    if (sl.staging) cudaFreeHost(sl.staging);
  }
  {
    std::lock_guard<std::mutex> lk(S.mu);
    rs::reap_locked(&S);
  }
  if (S.arena_base) cudaFree(S.arena_base);
  delete srv;
  return st;
}

}  // extern "C"
