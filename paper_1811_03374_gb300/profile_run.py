"""Runs closest-hit launches on one workload, for timing and profiling.

    python -m paper_1811_03374_gb300.profile_run --workload hair --depth 10 \\
        --variant warp --fast 1 --launches 3

Workloads: hair (the 1080p hair-patch frame), tiny (16 fibers x 16,384
rays), sweep-<class> (1M segments, one ray each, aimed at the segment's
box), aimed-hair (1M rays aimed inside segments of 2000 hair fibers, the
differentiation workload), single-<class> (one segment of the class against
2^20 rays aimed at its box: the shape of the paper's Fig. 1).  Prints the
mean launch time measured with CUDA events after one untimed launch.

    --depths 2-22      one JSON line per depth in the range
    --backward 1       also times the adjoint (intersect_backward) of the
                       loss sum_i w_i t_i, w ~ N(0, 1), after each forward,
                       and reports the backward / forward time ratio
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
    if name == "aimed-hair":
        return I.aimed_hair_case(1_000_000)
    if name.startswith("single-"):
        return I.single_fiber_case(name.split("-", 1)[1], 1 << 20)
    raise SystemExit("unknown workload %s" % name)


def depth_list(spec):
    if "-" in spec:
        a, b = spec.split("-")
        return list(range(int(a), int(b) + 1))
    return [int(x) for x in spec.split(",")]


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="hair")
    p.add_argument("--depth", type=int, default=10)
    p.add_argument("--depths", default=None, help="a range a-b or a list a,b,c of depths")
    p.add_argument("--variant", default="auto", choices=["auto", "lane", "warp", "filter", "scan", "ray"])
    p.add_argument("--kernel", default="persistent", choices=["persistent", "naive"])
    p.add_argument("--fast", type=int, default=1)
    p.add_argument("--block", type=int, default=128)
    p.add_argument("--chunk", type=int, default=32)
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--backward", type=int, default=0)
    a = p.parse_args()

    import torch
    from paper_1811_03374_gb300 import fiberx as F
    from paper_1811_03374_gb300 import inputs as I
    case = load(a.workload)
    dev = torch.device("cuda")
    fib = F.Fibers(case["cps"])
    fib.set_launch(a.block, 0, a.chunk, {"auto": 0, "lane": 1, "warp": 2, "filter": 3, "scan": 4, "ray": 5}[a.variant])
    rays = torch.from_numpy(case["rays"]).to(dev)
    rp = torch.from_numpy(case["row_ptr"]).to(dev)
    si = torch.from_numpy(case["seg_idx"]).to(dev)
    flags = (F.FX_FAST_MATH if a.fast else 0) | (F.FX_KERNEL_NAIVE if a.kernel == "naive" else 0)
    n_pair = len(case["seg_idx"])
    w = torch.from_numpy(I.hit_weights(rays.shape[0])).to(dev)
    grad = torch.zeros((fib.n_seg, 4, 4), dtype=torch.float32, device=dev)
    for depth in (depth_list(a.depths) if a.depths else [a.depth]):
        out = F.intersect_closest(fib, rays, rp, si, depth, flags)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(a.launches):
            F.intersect_closest(fib, rays, rp, si, depth, flags, out=out)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / max(1, a.launches)
        rec = {"workload": a.workload, "depth": depth, "pairs": int(n_pair), "ms_per_launch": ms,
               "gpairs_s": n_pair / ms / 1e6, "hits": int((out[1] >= 0).sum().item()), "status": fib.status(),
               "launch": fib.get_launch()}
        if a.backward:
            tu, seg = out[0], out[1]
            gt = torch.where(seg >= 0, w, torch.zeros_like(w))
            F.intersect_backward(fib, rays, tu, seg, gt, grad_cps=grad)
            torch.cuda.synchronize()
            s.record()
            for _ in range(a.launches):
                F.intersect_backward(fib, rays, tu, seg, gt, grad_cps=grad)
            e.record()
            torch.cuda.synchronize()
            ms_b = s.elapsed_time(e) / max(1, a.launches)
            rec.update(backward_ms=ms_b, backward_over_forward=ms_b / ms)
        print(json.dumps(rec), flush=True)
    fib.close()


if __name__ == "__main__":
    main()
