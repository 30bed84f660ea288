"""Runs a few closest-hit launches on one workload, for timing and profiling.

    python -m paper_1811_03374_gb300.profile_run --workload hair --depth 10 \\
        --variant warp --fast 1 --launches 3

Workloads: hair (the 1080p hair-patch frame), tiny (16 fibers x 16,384
rays), sweep-<class> (1M segments, one ray each).  Prints the mean launch
time measured with CUDA events after one untimed launch.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def load(name):
    from paper_1811_03374_gb300 import inputs as I
    if name == "hair":
        return I.hair_patch()
    if name == "tiny":
        return I.tiny_case()
    if name.startswith("sweep-"):
        return I.sweep_case(name.split("-", 1)[1], 1_000_000)
    raise SystemExit("unknown workload %s" % name)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="hair")
    p.add_argument("--depth", type=int, default=10)
    p.add_argument("--variant", default="auto", choices=["auto", "lane", "warp", "filter", "scan"])
    p.add_argument("--kernel", default="persistent", choices=["persistent", "naive"])
    p.add_argument("--fast", type=int, default=1)
    p.add_argument("--block", type=int, default=128)
    p.add_argument("--chunk", type=int, default=32)
    p.add_argument("--launches", type=int, default=3)
    a = p.parse_args()

    import torch
    from paper_1811_03374_gb300 import fiberx as F
    case = load(a.workload)
    dev = torch.device("cuda")
    fib = F.Fibers(case["cps"])
    fib.set_launch(a.block, 0, a.chunk, {"auto": 0, "lane": 1, "warp": 2, "filter": 3, "scan": 4}[a.variant])
    rays = torch.from_numpy(case["rays"]).to(dev)
    rp = torch.from_numpy(case["row_ptr"]).to(dev)
    si = torch.from_numpy(case["seg_idx"]).to(dev)
    flags = (F.FX_FAST_MATH if a.fast else 0) | (F.FX_KERNEL_NAIVE if a.kernel == "naive" else 0)
    out = F.intersect_closest(fib, rays, rp, si, a.depth, flags)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(a.launches):
        F.intersect_closest(fib, rays, rp, si, a.depth, flags, out=out)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / max(1, a.launches)
    print(json.dumps({"workload": a.workload, "pairs": int(len(case["seg_idx"])), "ms_per_launch": ms,
                      "gpairs_s": len(case["seg_idx"]) / ms / 1e6, "status": fib.status(),
                      "launch": fib.get_launch()}))
    fib.close()


if __name__ == "__main__":
    main()
