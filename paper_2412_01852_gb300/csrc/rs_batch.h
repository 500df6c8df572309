// rs_batch.h -- the pieces of a batched wavefront launch, shared by batch
// plans (rs_batch.cu) and the serving scheduler (rs_server.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "rs_internal.h"
#include "rs_wave.cuh"

namespace rs {

// Host-side layout of one batched launch: which problems have work, their
// tiling, the segment table and the offsets of every part of its workspace.
struct BatchLayout {
  std::vector<int> idx;               // problems with work
  std::vector<WavePlan> wp;           // their tilings
  std::vector<size_t> cs_off, done_off;
  std::vector<WaveSegment> seg;
  size_t done_ints = 0, cs_bytes = 0;
  size_t o_inst = 0, o_tmap = 0, o_seg = 0, o_rep = 0, o_cnt = 0, o_cs = 0, total = 0;
  size_t cnt_bytes = 0;
  long long tickets = 0, rotation_rows = 0;
  long long key_items_max = 0;        // most work items sharing one wavefront key
};

// Everything needed to enqueue one batched launch whose workspace is at `base`.
struct BatchLaunch {
  int device = 0;
  int count = 0;                      // problems with work
  rot_tuning tuning{};
  unsigned char* base = nullptr;      // device workspace
  size_t bytes = 0;
  WaveInstance* d_inst = nullptr;
  WaveSegment* d_seg = nullptr;
  void* d_rep = nullptr;
  unsigned char* d_counters = nullptr;
  size_t counters_bytes = 0;
  WaveLaunch launch{};
  int nseg = 0;
  long long total = 0;
  int repack_grid_x = 1;
  long long rotation_rows = 0;
  long long key_items_max = 0;        // bounds how many warps can have work at once (0: unknown)
  int grid = 1;
  int smem = 0;
  bool intmul = false;  // FP64 products on the integer pipe
};

// Validate the problems and lay out a launch (no device calls).
rot_status batch_layout(int count, const rot_problem* probs, const rot_tuning& tu, BatchLayout* L);

// Fill the host image (L.o_cs bytes: descriptors, TMA descriptors, segments)
// of a launch whose workspace will live at device address `dev_base`, and the
// launch record.  No device calls; the caller copies img to dev_base.
rot_status batch_image(const BatchLayout& L, const rot_problem* probs, unsigned char* dev_base,
                       unsigned char* img, BatchLaunch* B);

// Launch geometry on the current device (occupancy; not during stream capture).
// The grid is the smaller of a full persistent grid and what the launch's
// parallelism can use (about one warp per work item of its busiest key), so a
// small launch leaves SMs free for launches running beside it.
rot_status batch_prepare(BatchLaunch* B);

// Warps of the batched kernel that fit on the current device at once.
rot_status batch_resident_warps(long long* warps);

// Sequences per p-block for a launch over these problems: the largest of
// 16, 8, 4 whose p-blocks give at least `warps` work items per key summed over
// the problems (smaller p-blocks mean more items that can run at once), else 4.
int batch_pick_K(int count, const rot_problem* probs, long long warps);

// Launch the persistent batched kernel and the status fold for a prepared
// launch (the only place the batched kernel is launched).
rot_status batch_launch_kernel(const BatchLaunch& B, cudaStream_t s, int trace_kind, long long work);

// Enqueue: clear counters, repack C/S, the persistent kernel, fold the status.
rot_status batch_enqueue(const BatchLaunch& B, cudaStream_t s);

}  // namespace rs
