#!/usr/bin/env python3
"""Benchmark of the plain FP64 rotation-sequence path on GB300.

Workload (default "plain-8192"): A is 8192 x 8192 with i.i.d. N(0,1) entries,
column-major; C, S are 8191 x 192 from angles uniform in [0, 2*pi); seed 2.
One step = one rot_apply over the whole instance (all 192 sequences of 8191
rotations applied to all 8192 rows), in place.  A is 512 MiB, larger than the
129 MB L2, so consecutive steps do not hit in L2.

Metric: rotation-row updates per second (one rotation applied to one row is 6
flops), whole job over all ranks.  Under torchrun every rank runs its own
independent instance (seed 2 + rank): weak scaling, no collective on the data
path.  Prints ONE JSON line on rank 0.

--impl reference times the CPU oracle (plain Algorithm 2 in C, one thread) on
bounded row samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_01852_gb300 import workloads as wl  # noqa: E402

METRIC = "rotation-row updates/s (6 flop each) vs FP64 peak; serving p50/p99 latency"
# The oracle is run on blocks of this many rows (rows are independent, so any
# block of rows is a faithful sample of the workload).
ORACLE_BLOCK = 16
# FP64 fused multiply-adds per SM per clock: the nominal 1.25 TFLOP/s of GB300
# divided by (152 SMs x 2 flops x 2.07 GHz) is 1.99, i.e. 2 lanes/clk/SM.
FP64_FMA_PER_SM_CLK = 2
UNIT = "rot-rows/s"

# DRAM traffic of one wave-kernel launch on this workload, from the ncu capture
# summarised in profiles/ (dram__bytes_read.sum + dram__bytes_write.sum),
# together with a hash of the kernel sources it was taken on.  If the kernel
# sources change, the number no longer applies and traffic is reported as null.
# Captured on plain-8192x4096 (0.5084e9 B per launch) and scaled by the
# rotation-rows of plain-8192 (x2.00024): consecutive p-blocks follow each other
# closely enough that A's columns are still in L2 for the next p-block, so the
# kernel reads and writes A about once and its traffic grows with n.
NCU_TRAFFIC = {"bytes": 1.0170e9, "kernel_src_sha": "0d949a02ccb03b30"}

# The same for the single-p-block column stream at k = 1 (FP32, 8192 x 8192),
# captured on the full workload (the kernel takes 0.1 ms).
NCU_TRAFFIC_STREAM = {"bytes": 4.7453e8, "kernel_src_sha": "ac9bbfd104fcad37"}


def stream_src_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("rs_stream.cuh", "rs_device.cuh"):         # the kernel, its tiling and its launch shape
        with open(os.path.join(ROOT, "paper_2412_01852_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x20: "sync_boost", 0x40: "sw_thermal_slowdown",
               0x80: "hw_thermal_slowdown", 0x100: "hw_power_brake_slowdown"}


def kernel_src_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("rs_wave.cuh", "rs_device.cuh", "rs_wave_host.cu"):
        with open(os.path.join(ROOT, "paper_2412_01852_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + SMI_FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 5:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                mask = int(parts[4], 16)
            except ValueError:
                continue
            for bit, name in REASON_BITS.items():
                if mask & bit and name != "gpu_idle":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def nominal_sm_clock_ghz(dev):
    """Maximum SM clock of the device in GHz (CUDA attribute, in kHz)."""
    try:
        from cuda.bindings import runtime as cr
        err, khz = cr.cudaDeviceGetAttribute(cr.cudaDeviceAttr.cudaDevAttrClockRate, dev.index)
        if int(err) == 0 and khz > 0:
            return khz / 1e6
    except Exception:
        pass
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev.index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        return float(out.splitlines()[0]) / 1e3
    except Exception:
        return 2.07


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base_seed, rank):
    """Each rank applies its own independent instance (weak scaling, no data exchange)."""
    return base_seed + rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, steps, units_per_step, seconds):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return world_size * steps * units_per_step / seconds


def host_cores():
    """Host CPU cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rows_threaded(A, C, S, row_blocks, threads, deadline=None):
    """The oracle as it stands, run on row blocks by `threads` host threads at
    once (rows are independent, and the C oracle releases the interpreter
    while it runs).  Returns the number of rows done before the deadline."""
    import threading
    import oracle
    lock = threading.Lock()
    todo = list(row_blocks)
    done = [0]

    def worker():
        while True:
            with lock:
                if not todo or (deadline is not None and time.perf_counter() > deadline):
                    return
                r0, r1 = todo.pop(0)
            oracle.rot_sequence(A[r0:r1], C, S)
            with lock:
                done[0] += r1 - r0

    ts = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return done[0]


def cpu_baseline_leg(cfg, seconds):
    """The oracle as it stands, on row blocks of the same instance, on all host cores."""
    import oracle
    oracle.build()
    m, n, k, seed = cfg["m"], cfg["n"], cfg["k"], cfg["seed"]
    A = wl.matrix(m, n, seed)
    C, S = wl.rotations(n, k, seed)
    cores = host_cores()
    blocks = [(r, min(r + ORACLE_BLOCK, m)) for r in range(0, m, ORACLE_BLOCK)]
    t0 = time.perf_counter()
    rows = oracle_rows_threaded(A, C, S, blocks, cores, deadline=t0 + seconds)
    el = time.perf_counter() - t0
    return {"value": rows * (n - 1) * k / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of the %d rows of the %dx%d, k=%d instance (%d x %d x %d rotation-rows), in "
                      "blocks of %d rows taken by %d host threads at once; plain Algorithm 2 in C, %.1f s"
                      % (rows, m, m, n, k, rows, n - 1, k, ORACLE_BLOCK, cores, el)}


def cpu_parallel_leg(cfg, seconds):
    """The multi-core CPU baseline (row blocks over OpenMP threads, wave order
    inside a block), bit-exact with the oracle, on the same instance."""
    import oracle
    oracle.build()
    m, n, k, seed = cfg["m"], cfg["n"], cfg["k"], cfg["seed"]
    A = np.asfortranarray(wl.matrix(m, n, seed))
    C, S = wl.rotations(n, k, seed)
    chunk = 1024
    rows, used = 0, 1
    t0 = time.perf_counter()
    while rows < m and time.perf_counter() - t0 < seconds:
        r1 = min(rows + chunk, m)
        blk = np.asfortranarray(A[rows:r1])
        _, used = oracle.rot_sequence_parallel(blk, C, S, mb=32, kb=32, inplace=True)
        rows = r1
    el = time.perf_counter() - t0
    return {"value": rows * (n - 1) * k / el, "unit": UNIT, "cores": used,
            "kind": "openmp row blocks, wave order (bit-exact with the oracle)",
            "openmp": oracle.parallel_uses_openmp(),
            "sample": "%d of the %d rows of the %dx%d, k=%d instance in chunks of %d rows; 32-row blocks "
                      "over %d threads, 32 sequences per pass, %.1f s" % (rows, m, m, n, k, chunk, used, el)}


def run_reference(args, cfg):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    m, n, k, seed = cfg["m"], cfg["n"], cfg["k"], cfg["seed"]
    A = wl.matrix(m, n, seed)
    C, S = wl.rotations(n, k, seed)
    rows = min(args.ref_rows, m) if args.ref_rows > 0 else m
    cores = host_cores()

    def one_step(r0):
        blocks = [(b, min(b + ORACLE_BLOCK, r0 + rows)) for b in range(r0, r0 + rows, ORACLE_BLOCK)]
        done = oracle_rows_threaded(A, C, S, blocks, cores)
        assert done == rows

    for i in range(args.warmup):
        one_step(0)
    times = []
    for i in range(args.steps):
        r0 = (i * rows) % (m - rows + 1)
        t0 = time.perf_counter()
        one_step(r0)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    work = args.steps * rows * (n - 1) * k
    value = work / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(cfg, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d rows per step of the %dx%d, k=%d instance, in blocks of %d rows taken "
                                   "by %d host threads at once; plain Algorithm 2 in C"
                                   % (rows, m, n, k, ORACLE_BLOCK, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(cfg, ws):
    return {"workload": "%s: A %dx%d N(0,1) column-major, C/S %dx%d from uniform angles, seed %d"
                        % (cfg["name"], cfg["m"], cfg["n"], cfg["n"] - 1, cfg["k"], cfg["seed"]),
            "m": cfg["m"], "n": cfg["n"], "k": cfg["k"],
            "parallelism": "independent instance per rank" if ws > 1 else "single GPU",
            "l2": "inputs larger than L2 (A is %d MiB)" % (cfg["m"] * cfg["n"] * 8 >> 20)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain-8192")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="rows of the instance per reference step (0: all of them)")
    ap.add_argument("--variant", default="plain",
                    choices=["plain", "f32", "gemm-f16", "gemm-bf16", "gemm-dmma", "gemm-f16-q32",
                             "gemm-bf16-q32", "batched", "serving", "reflectors", "left", "small-k", "k-sweep"],
                    help="plain (default) is the measured line; the others measure the other "
                         "paths of the library on the same GPU")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--variants", default="f32,gemm-bf16,batched,serving",
                    help="other paths measured after the plain line and reported in its 'variants' "
                         "object ('none' to skip)")
    ap.add_argument("--variant-steps", type=int, default=5)
    ap.add_argument("--variant-serve-requests", type=int, default=2000,
                    help="requests per offered-load level in the embedded serving measurement")
    ap.add_argument("--serve-batch", type=int, default=64, help="requests per launch in the serving variant")
    ap.add_argument("--serve-streams", type=int, default=8, help="server streams in the serving variant")
    ap.add_argument("--serve-wide-rows", type=int, default=0,
                    help="server's wide-matrix threshold in rows (0: the library default, 2048)")
    ap.add_argument("--serve-fuse-k", type=int, default=192,
                    help="most sequences fused per matrix per launch in the serving variant (0 = no limit)")
    args = ap.parse_args()
    cfg = dict(wl.WORKLOADS[args.workload])
    cfg["name"] = args.workload

    if args.impl == "reference":
        run_reference(args, cfg)
        return
    if args.variant != "plain":
        run_variant(args)
        return

    import torch
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import api, build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()

    def barrier():
        if dist is not None:
            dist.barrier()

    m, n, k = cfg["m"], cfg["n"], cfg["k"]
    seed = rank_seed(cfg["seed"], rank)
    A, C, S = wl.problem(m, n, k, seed)
    W = wl.rotation_rows(m, n, k)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
    Cd = torch.from_numpy(np.ascontiguousarray(C.T)).to(dev).t()
    Sd = torch.from_numpy(np.ascontiguousarray(S.T)).to(dev).t()
    stream = torch.cuda.current_stream()

    peak_gflops, _ = api.measure_fp64_peak()
    # The rotation's own FP64 instruction mix (2 DMUL + 2 DFMA per rotation-row),
    # registers only, at the wave kernel's launch shape (2 CTAs x 8 warps per SM)
    # and at full occupancy: the best of these is the measured rotation ceiling.
    mix = {}
    for kind in ("rotation", "rotation_smem", "rotation_fma_smem", "dfma", "dmul", "dfma_smem"):
        for wpc, cps in ((8, 2), (32, 2)):
            r, _ = api.measure_fp64_mix(kind, wpc, cps)
            mix["%s_%dw" % (kind, wpc * cps)] = r

    for _ in range(args.warmup):
        rs.rot_apply(Ad, Cd, Sd)
    torch.cuda.synchronize()
    rs.rot_device_status()

    # ---- device-timed region ------------------------------------------------------
    barrier()
    torch.cuda.synchronize()
    api.trace_start()
    l0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            rs.rot_apply(Ad, Cd, Sd)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = api.launch_count() - l0
    recs = api.trace_stop()
    rs.rot_device_status()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = job_throughput(ws, args.steps, W, ms * 1e-3)

    wave = [r for r in recs if r[0] == "wave_f64"]
    kms = sum(r[1] for r in wave) / max(len(wave), 1)
    achieved_tflops = 6.0 * W / (kms * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    max_clk_ghz = nominal_sm_clock_ghz(dev)
    peak_tflops = props.multi_processor_count * FP64_FMA_PER_SM_CLK * 2 * max_clk_ghz / 1e3
    traffic = NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["kernel_src_sha"] == kernel_src_sha() else None
    rot_probe_tflops = max(v for kname, v in mix.items() if kname.startswith("rotation")) * 6 / 4 / 1e12

    # ---- end to end through the host-buffer entry point ---------------------------
    Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
    Ah.numpy()[:] = A.T
    Ch = torch.empty((k, n - 1), dtype=torch.float64, pin_memory=True)
    Ch.numpy()[:] = C.T
    Sh = torch.empty((k, n - 1), dtype=torch.float64, pin_memory=True)
    Sh.numpy()[:] = S.T
    A_host, C_host, S_host = Ah.numpy().T, Ch.numpy().T, Sh.numpy().T
    api.rot_apply_host(A_host, C_host, S_host)  # warm-up
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        api.rot_apply_host(A_host, C_host, S_host)
    el = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": job_throughput(ws, args.e2e_steps, W, el), "unit": UNIT,
           "h2d_bytes_per_step": int(A.nbytes + C.nbytes + S.nbytes), "d2h_bytes_per_step": int(A.nbytes),
           "steps": args.e2e_steps}

    cpu = (cpu_baseline_leg(cfg, args.cpu_seconds)
           if (rank == 0 and ws == 1 and args.cpu_seconds > 0) else None)
    cpu_par = (cpu_parallel_leg(cfg, args.cpu_seconds)
               if (rank == 0 and ws == 1 and args.cpu_seconds > 0) else None)

    # ---- the other forms of the path on the same GPU (after the timed region) ------
    variants = None
    if rank == 0 and ws == 1 and args.variants not in ("", "none"):
        variants = {}
        for name in args.variants.split(","):
            va = argparse.Namespace(**vars(args))
            va.variant = name
            va.steps = args.variant_steps
            va.warmup = 3
            va.serve_requests = args.variant_serve_requests
            t_v = time.perf_counter()
            v = variant_line(va)
            for key in ("metric", "unit", "n_gpus", "higher_is_better", "data", "variant"):
                v.pop(key, None)
            v["wall_s"] = time.perf_counter() - t_v
            variants[name] = v

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(cfg, ws),
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops,
                         "traffic": traffic, "kernel": "wave_kernel<double>",
                         "kernel_ms": kms,
                         "peak_source": "nominal FP64 FMA rate: %d SMs x %d DFMA/clk x 2 flops x "
                                        "%.3f GHz max SM clock" % (props.multi_processor_count,
                                                                   FP64_FMA_PER_SM_CLK, max_clk_ghz),
                         "dfma_probe_tflops": peak_gflops / 1e3,
                         "frac_of_dfma_probe": achieved_tflops / (peak_gflops / 1e3) if peak_gflops else None,
                         "rotation_ceiling_frac": 0.75,
                         "fp64_pipe_lanes_per_s_probes": mix,
                         "rotation_probe_tflops": rot_probe_tflops,
                         "frac_of_rotation_probe": achieved_tflops / rot_probe_tflops,
                         "rotation_probe": "best FP64 rate of the rotation's own instruction mix (4 FP64 "
                                           "instructions per rotation-row: the products as DMUL or as DFMA with "
                                           "a -0 addend, bit-identical), registers only, (c,s) in registers or "
                                           "read from shared memory, 16 or 64 warps per SM; 6 flops per 4 "
                                           "lane-ops"},
            "cpu_baseline": cpu,
            "cpu_parallel": cpu_par,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if variants is not None:
            line["variants"] = variants
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------
# Other paths of the library, measured on the same GPU (``--variant``).  Each prints one
# JSON line with the same metric and unit as the plain line.
# ---------------------------------------------------------------------------------------

FP32_FMA_PER_SM_CLK = 128


def _dev_colmajor(torch, a, dev, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a.T)).to(dev).t()
    return t if dtype is None else t.to(dtype)


def _orth_drift(torch, apply_fn, n, dtype, dev):
    """max |Q^T Q - I| for Q = the variant applied to the n x n identity (the
    precision workload's orthogonality check), Q^T Q formed in FP64."""
    Q = torch.eye(n, dtype=dtype, device=dev).t().contiguous().t()
    apply_fn(Q)
    torch.cuda.synchronize()
    Qd = Q.double()
    M = Qd.t() @ Qd
    M.diagonal().sub_(1.0)
    drift = float(M.abs().max())
    del Q, Qd, M
    torch.cuda.empty_cache()
    return drift


def _row_rel(torch, out, ref):
    d = torch.linalg.norm((out.double() - ref), dim=1)
    return float((d / torch.linalg.norm(ref, dim=1)).max())


def _timed_steps(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _measured_peaks():
    """The measured peaks of this machine's GPUs, if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def run_variant(args):
    print(json.dumps(variant_line(args)), flush=True)


def variant_line(args):
    """Measure one of the library's other paths; returns its JSON line (a dict)."""
    import torch
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import api, build
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    clk = nominal_sm_clock_ghz(dev)
    fp64_peak = props.multi_processor_count * FP64_FMA_PER_SM_CLK * 2 * clk / 1e3
    fp32_peak = props.multi_processor_count * FP32_FMA_PER_SM_CLK * 2 * clk / 1e3
    line = {"metric": METRIC, "unit": UNIT, "variant": args.variant, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic"}

    if args.variant == "f32" or args.variant.startswith("gemm-"):
        cfg = wl.WORKLOADS["precision-8192"]
        m, n, k = cfg["m"], cfg["n"], cfg["k"]
        A, C, S = wl.problem(m, n, k, cfg["seed"])
        W = wl.rotation_rows(m, n, k)
        A64 = _dev_colmajor(torch, A, dev)
        C64 = _dev_colmajor(torch, C, dev)
        S64 = _dev_colmajor(torch, S, dev)
        ref = rs.colmajor(A64)
        rs.rot_apply(ref, C64, S64)                     # the FP64 path's result, for the error
        if args.variant == "f32":
            A32, C32, S32 = rs.colmajor(A64.float()), rs.colmajor(C64.float()), rs.colmajor(S64.float())
            once = rs.colmajor(A32)
            rs.rot_apply_f32(once, C32, S32)
            err = _row_rel(torch, once, ref)
            fn = lambda: rs.rot_apply_f32(A32, C32, S32)
            drift = _orth_drift(torch, lambda Q: rs.rot_apply_f32(Q, C32, S32), n, torch.float32, dev)
            drift_bound = 8 * k * 2.0 ** -24
            kind, peak, dtype = "wave_f32", fp32_peak, "f32"
            cfg_line = {"workload": "precision-8192 FP32: A 8192x8192, C/S 8191x192 rounded to FP32", "m": m,
                        "n": n, "k": k}
        else:
            mode = args.variant[len("gemm-"):]          # dmma, f16, bf16, f16-q32, bf16-q32
            base = mode.split("-")[0]
            nb, kb = cfg["nb"], cfg["kb"]
            once = rs.colmajor(A64)
            api.rot_apply_gemm(once, C64, S64, nb=nb, kb=kb, mode=mode)
            err = _row_rel(torch, once, ref)
            work = rs.colmajor(A64)
            fn = lambda: api.rot_apply_gemm(work, C64, S64, nb=nb, kb=kb, mode=mode)
            drift = _orth_drift(torch, lambda Q: api.rot_apply_gemm(Q, C64, S64, nb=nb, kb=kb, mode=mode), n,
                                torch.float64, dev)
            P = -(-k // kb)
            drift_bound = {"dmma": 32 * P ** 0.5 * 2.0 ** -53, "f16": P * 2.0 ** -20,
                           "bf16": 1.5 * P * 2.0 ** -17}[base]
            kind, peak, dtype = "form_blocks", fp64_peak, {"f16": "f16x2", "bf16": "bf16x2", "dmma": "f64"}[base]
            cfg_line = {"workload": "precision-8192 accumulated blocks: A 8192x8192, k=192, nb=%d, kb=%d, %s"
                                    % (nb, kb, mode), "m": m, "n": n, "k": k, "nb": nb, "kb": kb, "mode": mode}
        torch.cuda.synchronize()
        rs.rot_device_status()
        api.trace_start()
        ms = _timed_steps(torch, fn, args.steps, args.warmup, stream)
        recs = api.trace_stop()
        rs.rot_device_status()
        by, work_by = {}, {}
        for r in recs:
            by.setdefault(r[0], []).append(r[1])
            work_by.setdefault(r[0], []).append(r[2])
        kernels = {kname: sum(v) / len(v) for kname, v in by.items()}
        steps_traced = max(len(v) for v in by.values())
        per_step = {kname: sum(v) / steps_traced for kname, v in by.items()}
        line.update({"value": args.steps * W / (ms * 1e-3), "ms_per_step": ms / args.steps, "dtype": dtype,
                     "config": cfg_line, "max_row_rel_err_vs_fp64_path": err,
                     "row_rel_err_bound": drift_bound,
                     "orthogonality_identity": {"max_abs_QtQ_minus_I": drift, "bound": drift_bound,
                                                "input": "I_%d" % n},
                     "kernel_ms_per_step": per_step})
        if args.variant == "f32":
            # k = 192 runs as one pass of the lane pipeline; other shapes may
            # add the wavefront kernel or the column stream.
            kms = sum(per_step.get(kn, 0.0) for kn in ("pipe_f32", "wave_f32"))
            kname = "+".join(kn for kn in ("pipe_f32_kernel", "wave_f32_kernel") if per_step.get(kn[:-7], 0.0) > 0)
            line["roofline"] = {"bound": "alu", "achieved": 6.0 * W / (kms * 1e-3) / 1e12, "peak": peak,
                                "unit": "TFLOP/s", "kernel": kname, "kernel_ms": kms,
                                "peak_source": "nominal FP32 FMA rate: SMs x 128 x 2 x max SM clock"}
            line["roofline"]["frac"] = line["roofline"]["achieved"] / peak
        else:
            kms = kernels.get("form_blocks", 0.0)
            nblk = api.form_blocks_count(n, k, cfg["nb"], cfg["kb"])
            # Rotation-row updates the formation kernel executed, as its launch
            # reports them (waves where a block's rows are still zero are
            # skipped in FP64; the FP32 pipeline also runs its (1,0) stages).
            fw = work_by.get("form_blocks", [0])
            form_rows = sum(fw) / len(fw)
            q32 = cfg_line["mode"].endswith("-q32")
            fpeak = fp32_peak if q32 else fp64_peak
            line["roofline"] = {"bound": "alu",
                                "kernel": "form32_kernel (block formation, FP32 lane pipeline)" if q32 else
                                          "wave_batched_kernel (block formation, FP64)",
                                "achieved": 6.0 * form_rows / (kms * 1e-3) / 1e12, "peak": fpeak,
                                "unit": "TFLOP/s", "kernel_ms": kms, "executed_rotation_rows": form_rows,
                                "share_of_step": kms / (ms / args.steps),
                                "rotation_ceiling_frac": 0.75,
                                "peak_source": "nominal %s FMA rate: SMs x %d x 2 x max SM clock"
                                               % (("FP32", FP32_FMA_PER_SM_CLK) if q32 else
                                                  ("FP64", FP64_FMA_PER_SM_CLK)),
                                "note": "achieved counts the rotation-row updates the kernel executed "
                                        "(6 flops each), as its trace record reports them"}
            line["roofline"]["frac"] = line["roofline"]["achieved"] / fpeak
            # The block apply on its own: 2*L^2 flops per row and block per product.
            akms = kernels.get("gemm_apply", 0.0)
            L = cfg["nb"] + cfg["kb"]
            mode = cfg_line["mode"].split("-")[0]
            products = 1 if mode == "dmma" else 3
            aflops = products * 2.0 * m * L * L * nblk
            if akms > 0:
                ap = {"kernel": "block apply (%s)" % ("mma.sync DMMA" if mode == "dmma" else "tcgen05 split " + mode),
                      "kernel_ms": akms, "achieved": aflops / (akms * 1e-3) / 1e12, "unit": "TFLOP/s"}
                if mode == "dmma":
                    ap.update({"bound": "tensor", "peak": None,
                               "note": "FP64 MMA shares the FP64 pipe; its measured rate is about 1.05 TFLOP/s"})
                else:
                    peaks = _measured_peaks()
                    bf = peaks.get("bf16_tflops")
                    ap.update({"bound": "tensor", "peak": bf,
                               "peak_source": "measured bf16 dense burst (FP16 has the same dense rate)"})
                    if bf:
                        ap["frac"] = ap["achieved"] / bf
                    # The kernel's own ceiling: per 64-row tile and block it
                    # issues a fixed number of M = 64, N = Lp/2 products over
                    # two accumulators, whose issue rate is measured here.
                    Lp = (L + 31) // 32 * 32
                    nk, kb = Lp // 16, cfg["kb"]
                    kz = min(nk, -(-(Lp // 2 + kb) // 16))      # chunks with half 0 nonzero
                    per_block = 6 * nk - 3 * (nk - kz) if mode == "bf16" else 3 * kz + 3 * nk
                    ns = api.measure_tc_issue(64, Lp // 2, 2, 3000)
                    floor_ms = nblk * per_block * ns * 1e-6
                    ap.update({"mma_issue_ns": ns, "mmas_per_tile_block": per_block,
                               "issue_floor_ms": floor_ms, "frac_of_issue_floor": floor_ms / akms})
                line["apply_roofline"] = ap
        return line

    if args.variant == "reflectors":
        cfg = wl.WORKLOADS["plain-8192"]
        m, n, k = cfg["m"], cfg["n"], cfg["k"]
        A = wl.matrix(m, n, cfg["seed"])
        T, V = wl.reflectors(n, k, cfg["seed"])
        W = wl.rotation_rows(m, n, k)
        Ad, Td, Vd = (_dev_colmajor(torch, X, dev) for X in (A, T, V))
        api.trace_start()
        ms = _timed_steps(torch, lambda: api.rot_apply_reflectors(Ad, Td, Vd), args.steps, args.warmup, stream)
        recs = api.trace_stop()
        rs.rot_device_status()
        kms = [r[1] for r in recs if r[0] == "reflect_f64"]
        kms = sum(kms) / len(kms)
        line.update({"value": args.steps * W / (ms * 1e-3), "ms_per_step": ms / args.steps, "dtype": "f64",
                     "config": {"workload": "reflectors: A 8192x8192 N(0,1), 2x2 reflectors (tau, nu) "
                                            "8191x192, nu = tan(phi), phi uniform in [-pi/4, pi/4]",
                                "m": m, "n": n, "k": k},
                     "roofline": {"bound": "alu", "kernel": "wave_kernel<double, reflect>", "kernel_ms": kms,
                                  "achieved": 6.0 * W / (kms * 1e-3) / 1e12, "peak": fp64_peak,
                                  "unit": "TFLOP/s"}})
        line["roofline"]["frac"] = line["roofline"]["achieved"] / fp64_peak
        return line

    if args.variant == "k-sweep":
        # Whole calls of rot_apply (FP64) and rot_apply_f32 over k, on four
        # shapes (FP64 on seven), to show how the dispatch (column stream,
        # lane pipeline in passes, wavefront kernel) behaves between the fixed
        # k of the other variants.  Median of four calls per k, each after an L2
        # flush (a 256 MiB write), CUDA events around the call.
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)

        def call_ms(fn, reps=4):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts))

        shapes = {}
        # FP64 also on 4864 x 8192 (152 strips of 32 rows, one per SM),
        # 1024 x 8192 and 16384 x 2048 (512 strips), around the split
        # stream's strip thresholds.
        for (m, n, precs) in ((8192, 8192, ("f32", "f64")), (4096, 4096, ("f32", "f64")),
                              (2048, 2048, ("f32", "f64")), (8192, 512, ("f32", "f64")), (4864, 8192, ("f64",)),
                              (1024, 8192, ("f64",)), (16384, 2048, ("f64",))):
            A = wl.matrix(m, n, 6)
            per = {}
            for prec in precs:
                Ad = _dev_colmajor(torch, A.astype(np.float32) if prec == "f32" else A, dev)
                ks = (list(range(1, 65)) + [65, 80, 86, 95, 96, 100, 128, 150, 160, 191, 192] if prec == "f32"
                      else list(range(1, 41)) + [48, 64, 80, 96, 128, 160, 192])
                row = {}
                for kk in ks:
                    C, S = wl.rotations(n, kk, 6)
                    if prec == "f32":
                        Cd, Sd = (_dev_colmajor(torch, X.astype(np.float32), dev) for X in (C, S))
                        fn = lambda: rs.rot_apply_f32(Ad, Cd, Sd)
                    else:
                        Cd, Sd = (_dev_colmajor(torch, X, dev) for X in (C, S))
                        fn = lambda: rs.rot_apply(Ad, Cd, Sd)
                    row[str(kk)] = call_ms(fn)
                per[prec] = row
            shapes["%dx%d" % (m, n)] = per
        line.update({"value": None, "ms_per_step": None, "dtype": "f32/f64",
                     "config": {"workload": "k sweep: A N(0,1) m x n column-major, uniform angles, seed 6",
                                "shapes": list(shapes)},
                     "ms_per_call": shapes})
        return line

    if args.variant == "small-k":
        # Few sequences: one HBM pass over A carries little arithmetic, so FP32
        # is bound by HBM; FP64 (0.375 flop/B at k = 1 against a machine balance
        # near 0.19) stays bound by the FP64 pipe.  L2 is flushed (a 256 MiB
        # write) before every timed run, which is timed alone.
        cfg = wl.WORKLOADS["plain-8192"]
        m, n = cfg["m"], cfg["n"]
        A = wl.matrix(m, n, cfg["seed"])
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
        peaks = _measured_peaks()
        hbm = peaks.get("hbm_gbs")

        def timed_alone(fn, reps):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts))

        rows = []
        A32 = _dev_colmajor(torch, A.astype(np.float32), dev)
        A64 = _dev_colmajor(torch, A, dev)
        # k > 8: the wavefront kernel (several p-blocks), for the crossover
        for prec, kk in (("f32", 1), ("f32", 2), ("f32", 4), ("f32", 8), ("f32", 16), ("f32", 32), ("f32", 64),
                         ("f64", 1), ("f64", 2), ("f64", 8), ("f64", 16), ("f64", 32)):
            C, S = wl.rotations(n, kk, cfg["seed"])
            if prec == "f32":
                Cd, Sd = (_dev_colmajor(torch, X.astype(np.float32), dev) for X in (C, S))
                fn = lambda: rs.rot_apply_f32(A32, Cd, Sd)
                esz, fpeak = 4, fp32_peak
            else:
                Cd, Sd = (_dev_colmajor(torch, X, dev) for X in (C, S))
                fn = lambda: rs.rot_apply(A64, Cd, Sd)
                esz, fpeak = 8, fp64_peak
            reps = max(args.steps, 10)
            api.trace_start()
            ms = timed_alone(fn, reps)
            recs = api.trace_stop()
            kern = [r[1] for r in recs if r[0] in (("wave_f32", "pipe_f32") if prec == "f32" else ("wave_f64", "pipe_f64"))]
            kms = sum(kern) / (3 + reps) if kern else ms       # every launch of a call (warm-up included)
            Wk = wl.rotation_rows(m, n, kk)
            # FP32: the column stream makes one pass over A per 8 sequences and
            # one per binary digit of the rest (up to k = 48), the lane
            # pipeline one per 192 (plus the k mod 32 left over, on the
            # stream).  FP64: one pass (the stream for k <= 2, the lane
            # pipeline for 3 <= k <= 32, the wavefront kernel beyond).
            def stream_passes(r):
                return r // 8 + bin(r % 8).count("1")
            if prec == "f32":
                passes = stream_passes(kk) if kk <= 48 else -(-(kk // 32) // 6) + stream_passes(kk % 32)
            else:
                passes = 1
            nbytes = passes * 2 * m * n * esz + 2 * (n - 1) * kk * esz   # A read and written per pass, C and S read
            # ms: the whole call (scratch, repack, kernel, status); kernel_ms: the
            # rotation kernel alone (CUDA events around its launch), which the
            # roofline fractions use.
            row = {"precision": prec, "k": kk, "passes": passes, "ms": ms, "kernel_ms": kms,
                   "rot_rows_per_s": Wk / (ms * 1e-3),
                   "tflops": 6.0 * Wk / (kms * 1e-3) / 1e12,
                   "frac_of_nominal_flops": 6.0 * Wk / (kms * 1e-3) / 1e12 / fpeak,
                   "hbm_gbs": nbytes / (kms * 1e-3) / 1e9, "bytes": nbytes}
            if hbm:
                row["frac_of_measured_hbm"] = row["hbm_gbs"] / hbm
            rows.append(row)
        # The same HBM-bound cases on the packed layout (32-row strips, each a
        # contiguous 32 x n panel): same kernels, same bits, contiguous runs.
        P32 = api.pack(A32)
        P64 = api.pack(A64)
        packed_rows = []
        for prec, kk in (("f32", 1), ("f32", 2), ("f32", 4), ("f32", 8), ("f32", 16), ("f64", 1), ("f64", 2)):
            C, S = wl.rotations(n, kk, cfg["seed"])
            if prec == "f32":
                Cd, Sd = (_dev_colmajor(torch, X.astype(np.float32), dev) for X in (C, S))
                fn = lambda: api.rot_apply_packed(P32, m, n, Cd, Sd)
                esz = 4
            else:
                Cd, Sd = (_dev_colmajor(torch, X, dev) for X in (C, S))
                fn = lambda: api.rot_apply_packed(P64, m, n, Cd, Sd)
                esz = 8
            reps = max(args.steps, 10)
            api.trace_start()
            ms = timed_alone(fn, reps)
            recs = api.trace_stop()
            kern = [r[1] for r in recs if r[0] in ("wave_f32", "wave_f64")]
            kms = sum(kern) / (3 + reps) if kern else ms
            passes = -(-kk // 8)
            nbytes = passes * 2 * m * n * esz + 2 * (n - 1) * kk * esz
            col = next(r for r in rows if r["precision"] == prec and r["k"] == kk)
            row = {"precision": prec, "k": kk, "layout": "packed", "ms": ms, "kernel_ms": kms,
                   "hbm_gbs": nbytes / (kms * 1e-3) / 1e9, "column_major_kernel_ms": col["kernel_ms"],
                   "speedup_vs_column_major": col["kernel_ms"] / kms}
            if hbm:
                row["frac_of_measured_hbm"] = row["hbm_gbs"] / hbm
            packed_rows.append(row)
        del P32, P64
        rs.rot_device_status()
        first = rows[0]
        line.update({"value": first["rot_rows_per_s"], "ms_per_step": first["ms"], "dtype": "f32",
                     "config": {"workload": "small k: A 8192x8192 N(0,1) (FP32 and FP64), C/S 8191xk from uniform "
                                            "angles, k in {1,2,4,8,16,32,64} (FP32) and {1,2,8,16,32} (FP64), "
                                            "seed 2",
                                "m": m, "n": n, "l2": "flushed before every timed run (256 MiB write)"},
                     "per_k": rows,
                     "packed_layout": packed_rows,
                     "roofline": {"bound": "hbm", "kernel": "stream_kernel<float, 1> at k = 1",
                                  "kernel_ms": first["kernel_ms"],
                                  "achieved": first["hbm_gbs"], "peak": hbm, "unit": "GB/s",
                                  "frac": first.get("frac_of_measured_hbm"),
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)",
                                  "algorithmic_bytes": first["bytes"],
                                  "traffic": NCU_TRAFFIC_STREAM["bytes"]
                                  if NCU_TRAFFIC_STREAM["kernel_src_sha"] == stream_src_sha() else None}})
        return line

    if args.variant == "left":
        # Rotations mixing the rows of A (C, S are (m-1) x k): A is transposed in
        # 32x32 shared-memory tiles, the column kernel runs, and it is
        # transposed back.  The step time includes both transposes.
        cfg = wl.WORKLOADS["plain-8192"]
        m, n, k = cfg["m"], cfg["n"], cfg["k"]
        A = wl.matrix(m, n, cfg["seed"])
        C, S = wl.rotations(m, k, cfg["seed"])
        W = wl.rotation_rows(n, m, k)                   # n columns, each rotated through m rows
        Ad, Cd, Sd = (_dev_colmajor(torch, X, dev) for X in (A, C, S))
        api.trace_start()
        ms = _timed_steps(torch, lambda: api.rot_apply_left(Ad, Cd, Sd), args.steps, args.warmup, stream)
        recs = api.trace_stop()
        rs.rot_device_status()
        kms = [r[1] for r in recs if r[0] == "wave_f64"]
        kms = sum(kms) / len(kms)
        line.update({"value": args.steps * W / (ms * 1e-3), "ms_per_step": ms / args.steps, "dtype": "f64",
                     "config": {"workload": "left application: A 8192x8192 N(0,1), C/S 8191x192 from uniform "
                                            "angles acting on rows, seed 2", "m": m, "n": n, "k": k},
                     "kernel_ms_per_step": {"wave_f64": kms, "transposes": ms / args.steps - kms},
                     "roofline": {"bound": "alu", "kernel": "wave_kernel<double> (on the transpose)",
                                  "kernel_ms": kms, "achieved": 6.0 * W / (kms * 1e-3) / 1e12,
                                  "peak": fp64_peak, "unit": "TFLOP/s"}})
        line["roofline"]["frac"] = line["roofline"]["achieved"] / fp64_peak
        return line

    if args.variant == "batched":
        shapes = wl.batch_shapes(512, seed=4)
        probs = []
        for i, (m, n, k) in enumerate(shapes):
            A, C, S = wl.problem(m, n, k, seed=40000 + i)
            probs.append((_dev_colmajor(torch, A, dev), _dev_colmajor(torch, C, dev), _dev_colmajor(torch, S, dev)))
        W = sum(wl.rotation_rows(m, n, k) for (m, n, k) in shapes)
        best, tune_ms = api.batch_autotune(probs)
        plan = api.BatchPlan(probs)
        s2 = torch.cuda.Stream()
        with torch.cuda.stream(s2):
            plan.execute()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s2):
            plan.execute()
        api.trace_start()
        ms = _timed_steps(torch, g.replay, args.steps, args.warmup, stream)
        recs = api.trace_stop()
        rs.rot_device_status()
        # the plain path on the same GPU, same instances one launch each, for comparison
        def one_by_one():
            for (Ad, Cd, Sd) in probs:
                rs.rot_apply(Ad, Cd, Sd)
        ms_single = _timed_steps(torch, one_by_one, 2, 1, stream)
        line.update({"value": args.steps * W / (ms * 1e-3), "ms_per_step": ms / args.steps, "dtype": "f64",
                     "config": {"workload": "batched: 512 instances, m log-uniform [64,4096], n log-uniform "
                                            "[32,2048], k uniform [1,96], seed 4", "instances": 512,
                                "rotation_rows_per_step": W, "tuning": best, "graph": True},
                     "one_launch_per_instance": {"value": 2 * W / (ms_single * 1e-3), "ms_per_step": ms_single / 2},
                     "roofline": {"bound": "alu", "kernel": "wave_batched_kernel", "peak": fp64_peak,
                                  "unit": "TFLOP/s"}})
        kms = [r[1] for r in recs if r[0] == "wave_batched"]
        if kms:
            line["roofline"]["kernel_ms"] = sum(kms) / len(kms)
        else:  # launches replayed from a graph are not traced: use the step time
            line["roofline"]["kernel_ms"] = ms / args.steps
        line["roofline"]["achieved"] = 6.0 * W / (line["roofline"]["kernel_ms"] * 1e-3) / 1e12
        line["roofline"]["frac"] = line["roofline"]["achieved"] / fp64_peak
        plan.close()
        return line

    if args.variant == "serving":
        sizes = wl.SERVING_SIZES
        per_size = 4
        mats, handles = [], {}
        srv = api.Server(hbm_budget_bytes=4 << 30, max_inflight=256, streams=args.serve_streams,
                         max_batch=args.serve_batch, max_fused_k=args.serve_fuse_k,
                         wide_rows=args.serve_wide_rows)
        for s_i, nsz in enumerate(sizes):
            for j in range(per_size):
                Ad = _dev_colmajor(torch, wl.matrix(nsz, nsz, seed=7000 + 10 * s_i + j), dev)
                mats.append(Ad)
                handles.setdefault(nsz, []).append(srv.register(Ad))
        pool = {nsz: [wl.rotations(nsz, 64, seed=8000 + 10 * s_i + j) for j in range(4)]
                for s_i, nsz in enumerate(sizes)}
        rng = np.random.default_rng(5)

        def submit(req):
            C, S = pool[req.n][int(rng.integers(0, 4))]
            h = handles[req.n][int(rng.integers(0, per_size))]
            return srv.submit(h, C[:, :req.k], S[:, :req.k]), wl.rotation_rows(req.n, req.n, req.k)

        # capacity: a burst of requests, all submitted at once
        burst = wl.serving_trace(min(args.serve_requests, 4000), 1e9, seed=5)
        srv.stats(reset=True)
        t0 = time.perf_counter()
        tk = [submit(r)[0] for r in burst]
        for t in tk:
            srv.wait(t)
        el = time.perf_counter() - t0
        cap_rps = len(burst) / el
        st_burst = srv.stats(reset=True)
        # each size class alone on the idle server: one request at a time
        alone = {}
        for nsz in sizes:
            row = {}
            for kk in (33, 64):
                lat = []
                for i in range(5):
                    C, S = pool[nsz][i % 4]
                    t = srv.submit(handles[nsz][i % per_size], C[:, :kk], S[:, :kk])
                    lat.append(srv.wait_latency(t))
                row["k%d_ms" % kk] = float(np.median(lat))
            alone[str(nsz)] = row
        srv.stats(reset=True)

        def pct(xs, q):
            xs = sorted(xs)
            return xs[min(len(xs) - 1, max(0, int(np.ceil(q * len(xs))) - 1))] if xs else None

        levels = []
        for frac in (0.25, 0.5, 0.9):
            trace = wl.serving_trace(args.serve_requests, frac * cap_rps, seed=5 + int(frac * 100))
            t0 = time.perf_counter()
            tk = []
            for r in trace:
                d = t0 + r.arrival_s - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tk.append((submit(r)[0], r.n))
            by_n = {}
            for t, nsz in tk:
                by_n.setdefault(nsz, []).append(srv.wait_latency(t))
            st = srv.stats(reset=True)
            per_class = {str(nsz): {"requests": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99),
                                    "max_ms": max(v)} for nsz, v in sorted(by_n.items())}
            levels.append({"offered_load": frac, "offered_rps": frac * cap_rps, "requests": len(trace),
                           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                           "throughput_rot_rows_per_s": st["rotation_rows_per_s"],
                           "achieved_rps": st["completed"] / st["busy_s"] if st["busy_s"] > 0 else 0,
                           "mean_batch": st["mean_batch"], "launches": st["launches"],
                           "per_size": per_class})
        srv.close()
        rs.rot_device_status()
        line.update({"value": st_burst["rotation_rows_per_s"], "dtype": "f64",
                     "ms_per_step": None,
                     "config": {"workload": "serving: Poisson arrivals, square A with n in {128..4096} "
                                            "weights 1/n, k uniform [2,64], seed 5; %d resident matrices"
                                            % len(mats), "requests_per_level": args.serve_requests,
                                "server": {"hbm_budget_bytes": 4 << 30, "max_inflight": 256,
                                           "streams": args.serve_streams, "max_batch": args.serve_batch,
                                           "max_fused_k": args.serve_fuse_k,
                                           "wide_rows": args.serve_wide_rows or 2048}},
                     "capacity": {"requests_per_s": cap_rps, "p50_ms": st_burst["p50_ms"],
                                  "p99_ms": st_burst["p99_ms"], "mean_batch": st_burst["mean_batch"]},
                     "alone_latency_idle_gpu": alone,
                     "loads": levels})
        return line


if __name__ == "__main__":
    main()
