"""Command line: one vector-OMT solve on seeded synthetic colour-image densities.

    python -m paper_1712_10279_gb300 --n 2048 --k 3 --iters 20 --engine stream

Prints the result record as one JSON line.  The densities come from
``synthetic.color_image_pair`` (Gaussian-filtered noise plus rectangles); the
channel graph is the complete graph on k nodes.  Useful for profiling one
engine on one size.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1712_10279_gb300")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--engine", default="auto", choices=["auto", "stream", "resident"])
    ap.add_argument("--halo", type=int, default=0)
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--repeat", type=int, default=1, help="solves in a row (the first warms up)")
    args = ap.parse_args(argv)

    import torch
    from . import solve
    from . import synthetic as S

    r0, r1 = S.color_image_pair(args.n, args.k, seed=args.seed)
    dev = torch.device("cuda", 0)
    d0 = torch.from_numpy(r0.astype(np.float32)).to(dev)
    d1 = torch.from_numpy(r1.astype(np.float32)).to(dev)
    edges = S.complete_graph(args.k)
    res = None
    for _ in range(max(1, args.repeat)):
        sol = solve(d0, d1, edges, args.alpha, max_iters=args.iters, check_every=args.check_every,
                    tol_gap=args.tol, tol_res=args.tol, engine=args.engine, halo=args.halo)
        res = sol.result
    torch.cuda.synchronize()
    print(json.dumps(dict(n=args.n, k=args.k, alpha=args.alpha, **res)), flush=True)


if __name__ == "__main__":
    main()
