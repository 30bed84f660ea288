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
    --counts 1         per-ray pruning-test counts (intersect_counts, Fig. 8)
                       with oriented cylinders and with ray-frame boxes: mean,
                       99th percentile and maximum per depth; for image-<class>
                       (one fiber seen by a 512 x 512 camera) --pgm DIR also
                       writes the per-pixel counts as log-scaled PGM images
"""
import argparse
import json
import os
import sys

import numpy as np

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
    if name.startswith("image-"):
        return I.single_fiber_image_case(name.split("-", 1)[1], 512)
    raise SystemExit("unknown workload %s" % name)


def write_pgm(path, counts, case):
    """Per-pixel counts as an 8-bit PGM: log2(1 + count), 255 at 2^16."""
    res = case["res"]
    img = np.zeros(res * res)
    img[case["pixel"]] = np.log2(1.0 + counts.astype(np.float64))
    img = np.clip(img * (255.0 / 16.0), 0, 255).astype(np.uint8).reshape(res, res)
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (res, res))
        f.write(img.tobytes())


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
    p.add_argument("--counts", type=int, default=0)
    p.add_argument("--pgm", default=None)
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
    if a.counts:
        for depth in (depth_list(a.depths) if a.depths else [a.depth]):
            rec = {"workload": a.workload, "depth": depth, "rays": int(rays.shape[0])}
            for mode in ("cylinder", "box"):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                n = F.intersect_counts(fib, rays, rp, si, depth, boxes=mode == "box", flags=flags)
                e.record()
                torch.cuda.synchronize()
                n = n.cpu().numpy()
                rec[mode] = {"mean": float(n.mean()), "p99": float(np.percentile(n, 99)), "max": int(n.max()),
                             "total": int(n.sum()), "ms": s.elapsed_time(e)}
                if a.pgm and "pixel" in case:
                    write_pgm(os.path.join(a.pgm, "%s_d%02d_%s.pgm" % (a.workload, depth, mode)), n, case)
            print(json.dumps(rec), flush=True)
        fib.close()
        return
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
