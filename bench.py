#!/usr/bin/env python
"""Ray / cubic-fiber closest-hit throughput on the 1080p hair-patch frame.

One step = one intersect_closest pass (persistent FP32 kernel, replayed from a
CUDA graph) over every candidate (ray, segment) pair of the frame: 100,000
fibers x 8 cubic segments, 1920 x 1080 pinhole rays, candidates from the
uniform-grid cull (mean ~12 per ray).  Inputs are resident in HBM; the L2 is
flushed (256 MB write) between timed steps and each step is timed with CUDA
events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own full frame (weak
scaling, no collective on the data path); the reported time is the maximum
over ranks.  ``--impl reference`` times the FP64 oracle on the host cores on a
bounded sample of the same frame.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G ray–segment intersections/s at depth d (FP32 vs oracle tol) and % FP32 FMA peak"
UNIT = "G intersections/s"
WORKLOAD = "hair_patch_1080p"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--depth", type=int, default=None)
    p.add_argument("--kernel", default="persistent", choices=["persistent", "naive"])
    p.add_argument("--fast", type=int, default=None, help="1: approximate rcp/sqrt, 0: IEEE")
    p.add_argument("--no-graph", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--tune", action="store_true", help="re-run the launch autotuner")
    p.add_argument("--out", default=None, help="also append the JSON line to this file")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist, device):
    """The largest of the ranks' x (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, pairs_per_rank, seconds):
    """Whole-job throughput in G pairs/s: every rank tests its own frame of
    pairs_per_rank pairs (weak scaling) in at most `seconds`."""
    return world * pairs_per_rank / seconds / 1e9


def emit(obj, args):
    line = json.dumps(obj)
    print(line, flush=True)
    if args.out:
        with open(args.out, "a") as f:
            f.write(line + "\n")


# ----------------------------------------------------------------- clocks

class NvmlClocks:
    """SM clock and clock-event reasons of one GPU, sampled from a thread
    about every `period` seconds between start() and stop() through NVML's
    read-only queries (libnvidia-ml via ctypes; nothing is set).  A timed
    region of a few milliseconds still gets several samples."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device, period=0.0005):
        import ctypes
        self.ok = False
        self.samples = []
        self.period = period
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            got = False
            try:
                import torch
                uuid = "GPU-" + str(torch.cuda.get_device_properties(torch_device).uuid)
                got = nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0
            except Exception:
                got = False
            if not got:
                vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
                idx = int(vis.split(",")[torch_device]) if vis and vis.split(",")[0].isdigit() else torch_device
                got = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) == 0
            if not got:
                return
            reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self._nv, self._h, self._reasons, self._ct = nv, h, reasons, ctypes
            mx = ctypes.c_uint(0)
            self.max_mhz = float(mx.value) if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 else None
            self.ok = True
        except Exception:
            self.ok = False

    def _sample(self):
        ct = self._ct
        mhz, rs = ct.c_uint(0), ct.c_ulonglong(0)
        if self._nv.nvmlDeviceGetClockInfo(self._h, 1, ct.byref(mhz)) == 0 and \
                self._reasons(self._h, ct.byref(rs)) == 0:
            self.samples.append((time.perf_counter(), float(mhz.value), int(rs.value)))

    def start(self):
        import threading
        if not self.ok:
            return self
        self._stop = threading.Event()

        def loop():
            while not self._stop.is_set():
                self._sample()
                time.sleep(self.period)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        return self

    def stop(self, ms_per_step=None):
        if not self.ok:
            return None
        self._stop.set()
        self._thread.join()
        self._sample()  # at least one sample at the end of the region
        self._nv.nvmlShutdown()
        self.ok = False
        if not self.samples:
            return None
        sm = np.array([x[1] for x in self.samples])
        seen = 0
        for x in self.samples:
            seen |= x[2]
        out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz, "samples": len(self.samples),
               "sm_mhz_min": float(sm.min()), "sm_mhz_max_seen": float(sm.max()),
               "reasons": sorted(v for k, v in self.REASONS.items() if seen & k), "source": "nvml"}
        if ms_per_step is not None:
            # time x clock: thousands of SM cycles per step at the median clock
            out["kcycles_per_step_at_median"] = ms_per_step * out["sm_mhz"]
        return out


class ClockSampler:
    """nvidia-smi sampling (100 ms period): the fallback where NVML cannot be
    loaded."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "fiberx_bench_clocks_%d.csv" % os.getpid())
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
               "-lms", "100"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, ms_per_step=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[2][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)),
               "samples": len(rows), "reasons": sorted(reasons), "source": "nvidia-smi"}
        if ms_per_step is not None:
            out["kcycles_per_step_at_median"] = ms_per_step * out["sm_mhz"]
        return out


def clock_sampler(local):
    """NVML sampling where it loads, else nvidia-smi's."""
    c = NvmlClocks(local)
    return c.start() if c.ok else ClockSampler(local)


# ------------------------------------------------------------- workload

def load_workload(rank=0):
    from paper_1811_03374_gb300 import inputs as I
    t0 = time.time()
    case = I.hair_patch()
    case["gen_seconds"] = time.time() - t0
    return case


# DRAM traffic per launch of the timed persistent kernel, from the committed
# ncu summaries, by variant: (key in profiles/traffic.json, its sources)
TRAFFIC = {1: ("k_lane_hair", ("trace.cuh", "lane_kernels.cu")),
           4: ("k_scan_hair", ("trace.cuh", "scan_kernels.cu"))}


def source_hash(files):
    """Hash of a kernel's sources (traffic figures taken on another version
    of it do not apply)."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1811_03374_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled(variant, field="dram_bytes_per_launch"):
    """A per-launch figure of the committed ncu summary (DRAM bytes, warp
    instructions), if it was taken on the current source of the variant's
    kernel."""
    if variant not in TRAFFIC:
        return None
    key, files = TRAFFIC[variant]
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        e = json.load(open(path)).get(key)
        if e and e.get("source_hash") == source_hash(files):
            return e.get(field)
    except Exception:
        pass
    return None


# ------------------------------------------------------------ CPU oracle

def oracle_rate(case, depth, seconds, seed=7, nthreads=0):
    """Times the FP64 oracle on a seeded ray sample sized to ~`seconds`
    (nthreads 0: all host cores)."""
    import oracle as O
    from paper_1811_03374_gb300 import inputs as I
    g = np.random.default_rng(seed)
    n = case["rays"].shape[0]
    pieces = O.presplit(case["cps"])
    frac = 0.002
    while True:
        idx = np.sort(g.choice(n, max(1, int(frac * n)), replace=False))
        sub = I.subsample_rays(case, idx)
        t0 = time.perf_counter()
        O.closest(sub, depth, pieces, nthreads=nthreads)
        dt = time.perf_counter() - t0
        pairs = len(sub["seg_idx"])
        if dt >= 0.5 * seconds or frac >= 1.0:
            break
        frac = min(1.0, frac * max(2.0, 0.8 * seconds / max(dt, 1e-3)))
    reps = 1
    while dt * reps < 0.5 * seconds:  # the whole frame is cheap: repeat it
        t0 = time.perf_counter()
        O.closest(sub, depth, pieces, nthreads=nthreads)
        dt_r = time.perf_counter() - t0
        dt = (dt * reps + dt_r) / (reps + 1)
        reps += 1
    return dict(value=pairs / dt / 1e9, pairs=pairs, rays=len(idx), seconds=dt * reps, frac=len(idx) / n,
                cores=nthreads or O.num_threads(), reps=reps)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    case = load_workload()
    # the depth the GPU arm runs: the tuned one cached for this workload
    from paper_1811_03374_gb300 import tune as T
    depth = args.depth if args.depth is not None else T.cached_depth(
        int(case["cps"].shape[0]), int(case["rays"].shape[0]), len(case["seg_idx"]))
    # size one step to ~ (a few minutes / steps)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    probe = oracle_rate(case, depth, per_step)
    from paper_1811_03374_gb300 import inputs as I
    g = np.random.default_rng(11)
    n = case["rays"].shape[0]
    pieces = O.presplit(case["cps"])
    times, pairs = [], 0
    for step in range(args.warmup + args.steps):
        idx = np.sort(g.choice(n, max(1, int(probe["frac"] * n)), replace=False))
        sub = I.subsample_rays(case, idx)
        t0 = time.perf_counter()
        O.closest(sub, depth, pieces)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pairs += len(sub["seg_idx"])
    value = pairs / sum(times) / 1e9
    sample = "%.3f%% of the frame's rays per step (seeded), all their candidates" % (100 * probe["frac"])
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": WORKLOAD, "depth": depth, "oracle": "FP64 C, OpenMP over rays"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": probe["cores"], "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}},
         args)


# --------------------------------------------------------------- GPU run

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_1811_03374_gb300 import fiberx as F
    from paper_1811_03374_gb300 import flops as FL
    from paper_1811_03374_gb300 import tune as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    case = load_workload(rank)
    n_ray, n_pair = case["rays"].shape[0], len(case["seg_idx"])
    t_up = time.perf_counter()
    fib = F.Fibers(case["cps"])  # host FP64 validation and pre-split, one copy per array (untimed)
    upload_s = time.perf_counter() - t_up
    info = fib.info()
    rays = torch.from_numpy(case["rays"]).to(dev)
    row_ptr = torch.from_numpy(case["row_ptr"]).to(dev)
    seg_idx = torch.from_numpy(case["seg_idx"]).to(dev)

    cfg = T.tuned_config(fib, rays, row_ptr, seg_idx, retune=args.tune, cps=case["cps"])
    depth = args.depth if args.depth is not None else cfg["depth"]
    fast = cfg["fast"] if args.fast is None else bool(args.fast)
    flags = (F.FX_FAST_MATH if fast else 0) | (F.FX_KERNEL_NAIVE if args.kernel == "naive" else 0)
    tu = torch.empty((n_ray, 2), dtype=torch.float32, device=dev)
    seg = torch.empty(n_ray, dtype=torch.int32, device=dev)
    leaf = torch.empty(n_ray, dtype=torch.int32, device=dev)
    out = (tu, seg, leaf)

    def step():
        F.intersect_closest(fib, rays, row_ptr, seg_idx, depth, flags, out=out)

    # counters (untimed) for the algorithmic work of one launch, taken on the
    # lane kernel: it performs every root test as a node step (the scan
    # variant tests most roots inside its warp-wide scans, where they are
    # not counted as nodes); descents, backtracks, hits and pair tests are
    # the same on both.  The naive kernel is timed against the same work (it
    # prunes nothing across candidates and so performs much more).
    fib.set_launch(cfg["block"], cfg["blocks_per_sm"], cfg["chunk"], F.FX_VARIANT_LANE)
    fib.counters(reset=True)
    F.intersect_closest(fib, rays, row_ptr, seg_idx, depth, (flags & ~F.FX_KERNEL_NAIVE) | F.FX_COUNT, out=out)
    counters = fib.counters(reset=True)
    fib.set_launch(cfg["block"], cfg["blocks_per_sm"], cfg["chunk"], cfg.get("variant", 0))
    n_ray_cand = int(np.count_nonzero(np.diff(case["row_ptr"])))
    n_piece_touched = int(len(np.unique(case["seg_idx"])))
    work = FL.alg_flops(counters, n_ray_cand)
    mwork = FL.method_flops(counters, n_ray_cand)
    ework = FL.estimate_flops(counters, n_ray_cand)
    abytes = FL.alg_bytes(n_ray, n_pair, n_piece_touched)

    graph = None
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            step()  # warm the allocator / lazy loading outside capture
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            step()
        run = graph.replay
    else:
        run = step
    # kernels of ours per step: the naive path's pair kernel and resolve; the
    # two-phase and scan variants' two kernels; one persistent kernel
    # otherwise
    two = fib.get_launch()["variant"] in (F.FX_VARIANT_FILTER, F.FX_VARIANT_SCAN)
    launches_per_step = 2 if args.kernel == "naive" or two else 1

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            run()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = clock_sampler(local) if rank == 0 else None
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i & 7))
            starts[i].record(stream)
            run()
            ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    clk = clocks.stop(float(np.mean(ms))) if clocks else None
    ms_step = max_over_ranks(float(np.mean(ms)), dist, dev)
    if dist:
        dist.barrier()
    value = job_value(world, n_pair, ms_step * 1e-3)

    # ---- end to end through the host-buffer entry (pinned buffers)
    e2e = None
    if not args.no_e2e:
        h_rays = torch.from_numpy(case["rays"]).pin_memory()
        h_rp = torch.from_numpy(case["row_ptr"]).pin_memory()
        h_si = torch.from_numpy(case["seg_idx"]).pin_memory()
        # the step's result is (t, u, seg) per ray; the leaf is not copied back
        h_out = (torch.empty((n_ray, 2), dtype=torch.float32).pin_memory(),
                 torch.empty(n_ray, dtype=torch.int32).pin_memory(), None)
        n_e2e = max(3, min(args.steps, 50))
        for _ in range(2):
            F.intersect_closest_host(fib, h_rays, h_rp, h_si, depth, flags, out=h_out, stream=stream)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            F.intersect_closest_host(fib, h_rays, h_rp, h_si, depth, flags, out=h_out, stream=stream)
        dt = max_over_ranks((time.perf_counter() - t0) / n_e2e, dist, dev)
        # bytes the library copied in the last step (rays of candidate-free
        # blocks of rows are not copied; see intersect_closest_host)
        h2d, d2h = F.host_bytes(fib)
        e2e = {"value": job_value(world, n_pair, dt), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "input_bytes_per_step": int(h_rays.numel() * 4 + h_rp.numel() * 4 + h_si.numel() * 4),
               "ms_per_step": dt * 1e3, "steps": n_e2e}

    status = fib.status()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    sm = info["sm_count"]
    peak = FL.fp32_peak_tflops(sm, 2070.0)
    fma_tflops, _ = F.fma_peak()  # measured FP32 FMA throughput, the cross-check of `peak`
    achieved = work / (ms_step * 1e-3) / 1e12
    variant = fib.get_launch()["variant"]
    traffic = profiled(variant) if args.kernel == "persistent" else None
    winst = profiled(variant, "warp_inst_per_launch") if args.kernel == "persistent" else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_note": "FP32 FMA: %d SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock)" % sm,
                "fma_microbenchmark_tflops": fma_tflops,
                "alg_flops_per_launch": work,
                # context: the paper's algorithm on the same frame (no bound
                # test; every candidate set up and its root tested), at this time
                "method_flops_per_launch": mwork,
                "frac_method_equivalent": mwork / (ms_step * 1e-3) / 1e12 / peak,
                # the same with per-unit estimates from App. C's operation counts
                "estimate_flops_per_launch": ework,
                "frac_per_unit_estimate": ework / (ms_step * 1e-3) / 1e12 / peak,
                "hbm_gbs_algorithmic": abytes / (ms_step * 1e-3) / 1e9,
                "alg_bytes_per_launch": abytes}
    if winst:
        # what binds the kernel: instruction issue, one warp instruction per
        # cycle on each of an SM's 4 schedulers (the ncu count per launch
        # over the live time)
        issue_peak = sm * 4 * 2070.0e6 / 1e9
        issue = winst / (ms_step * 1e-3) / 1e9
        roofline["issue"] = {"warp_inst_per_launch": winst, "achieved": issue, "peak": issue_peak,
                             "unit": "G warp instructions/s", "frac": issue / issue_peak}
    if clk:
        roofline["frac_at_sampled_clock"] = achieved / FL.fp32_peak_tflops(sm, clk["sm_mhz"])

    cpu = None
    if not args.no_cpu_baseline and world == 1:  # rank 0 at N = 1 only
        r = oracle_rate(case, depth, args.cpu_seconds)
        r1 = oracle_rate(case, depth, max(2.0, args.cpu_seconds / 4), seed=8, nthreads=1)
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": "%d seeded rays (%.2f%% of the frame) with their %d candidate pairs, "
                         "FP64 oracle, OpenMP over rays, %d repetition(s), %.1f s" % (
                             r["rays"], 100 * r["frac"], r["pairs"], r["reps"], r["seconds"]),
               "single_core": {"value": r1["value"], "unit": UNIT, "cores": 1,
                               "sample": "%d seeded rays with their %d candidate pairs, %.1f s" % (
                                   r1["rays"], r1["pairs"], r1["seconds"])}}

    emit({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
          "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
          "config": {"workload": WORKLOAD, "fibers": 100000, "segments": int(case["cps"].shape[0]),
                     "pieces": info["n_piece"], "rays": n_ray, "pairs": n_pair,
                     "pairs_per_ray_mean": n_pair / n_ray,
                     "pairs_per_ray_max": int(np.diff(case["row_ptr"]).max()), "depth": depth,
                     "kernel": args.kernel, "math": "fast" if fast else "ieee",
                     "launch": fib.get_launch(), "cuda_graph": graph is not None,
                     "l2": "flushed between timed steps (256 MB write)",
                     "parallelism": "replica per GPU" if world > 1 else "single GPU",
                     "counters": counters, "device_status": status, "timed_wall_s": wall,
                     "fiber_upload_ms": upload_s * 1e3},
          "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
          "gpu_launches": launches_per_step * args.steps, "clocks": clk}, args)
    fib.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
