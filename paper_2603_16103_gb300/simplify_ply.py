"""Simplify a Gaussian-splat PLY file on the GPU (Algorithm 1 end to end).

    python -m paper_2603_16103_gb300.simplify_ply in.ply out.ply --ratio 0.1

Reads the splats on the host, runs the whole loop through ngs_simplify_host
(pre-filter, then kNN graph, edge costs, disjoint pairs and merge until
N_tgt = max(ceil(r N0), 1) splats remain or no pair is left) and writes the
result.  Prints one JSON line with the counts and the timings.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import torch

from . import binding as B
from .ply import read_ply, write_ply
from .synth import Scene


def target_count(n0: int, ratio: float) -> int:
    """N_tgt = max(ceil(r N0), 1) (Algorithm 1)."""
    return max(int(math.ceil(ratio * n0)), 1)


def simplify_file(src: str, dst: str, ratio: float, **params) -> dict:
    t0 = time.perf_counter()
    scene = read_ply(src)
    t1 = time.perf_counter()
    target = target_count(scene.n, ratio)
    host = B.DeviceSplats.from_numpy(scene, device="cpu", pin=True)
    passes = 0
    with B.Context(**params) as ctx:
        if scene.n:
            passes = ctx.simplify_host(host, target)["passes"]
        torch.cuda.synchronize()
    t2 = time.perf_counter()
    write_ply(dst, Scene(*host.numpy()))
    t3 = time.perf_counter()
    return {"n_input": scene.n, "target": target, "n_output": host.n, "passes": passes,
            "read_s": t1 - t0, "simplify_s": t2 - t1, "write_s": t3 - t2}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("src")
    ap.add_argument("dst")
    ap.add_argument("--ratio", type=float, required=True, help="keep ratio r in (0, 1]")
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--tau", type=float, default=0.005, help="opacity pre-filter threshold")
    ap.add_argument("--no-prefilter", action="store_true")
    ap.add_argument("--mc-samples", type=int, default=1)
    ap.add_argument("--cost-mode", type=int, default=0, choices=[0, 1, 2, 3])
    ap.add_argument("--lambda-geo", type=float, default=1.0)
    ap.add_argument("--lambda-app", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if not 0 < args.ratio <= 1:
        ap.error("--ratio must be in (0, 1]")
    res = simplify_file(args.src, args.dst, args.ratio, k=args.k, tau=args.tau,
                        prefilter=0 if args.no_prefilter else 1, mc_samples=args.mc_samples,
                        cost_mode=args.cost_mode, lambda_geo=args.lambda_geo,
                        lambda_app=args.lambda_app, seed=args.seed)
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
