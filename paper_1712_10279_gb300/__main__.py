"""Command line: one vector-OMT solve on seeded synthetic densities.

    python -m paper_1712_10279_gb300 --n 2048 --k 3 --iters 20 --engine stream
    python -m paper_1712_10279_gb300 --dim 3 --n 128 --k 3 --iters 100
    python -m paper_1712_10279_gb300 --dim 3 --matrix --n 64 --k 3 --iters 100
    python -m paper_1712_10279_gb300 --batch 512 --path grouped --iters 5000

Prints the result record as one JSON line, with the last solve's time in
milliseconds (CUDA events).  2-D densities come from
``synthetic.color_image_pair`` (Gaussian-filtered noise plus rectangles), 3-D
ones from ``synthetic.blob_pair3``; the channel graph is the complete graph on
k nodes.  --matrix solves matrix OMT instead (k x k tensor fields from
``synthetic.tensor_field_pair(3)``, N = 3 random L).  --batch B solves the first
B of ``synthetic.batched_instances(512)`` (mixed n, k, graphs) in one batched
call along --path (auto, queue or grouped).  Useful for profiling one engine on one size.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1712_10279_gb300")
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--matrix", action="store_true", help="matrix OMT (k x k tensor fields, N = 3)")
    ap.add_argument("--batch", type=int, default=0, help="batched solve of this many mixed problems")
    ap.add_argument("--path", default="auto", choices=["auto", "queue", "grouped"], help="batched path")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--tau", type=float, default=None, help="dual step (default: Table 1 / Table 3 value)")
    ap.add_argument("--norms", default="default", choices=["default", "nuclear"],
                    help="matrix OMT: nuclear = ||U||_{1,nuc} ||W||_{1,nuc}")
    ap.add_argument("--engine", default="auto", choices=["auto", "stream", "resident"])
    ap.add_argument("--halo", type=int, default=0, help="2-D resident engine: halo; 3-D: z planes per block")
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--repeat", type=int, default=1, help="solves in a row (the first warms up)")
    args = ap.parse_args(argv)

    import torch
    from . import Batch, momt_solve, momt_solve3d, solve, solve3d
    from . import synthetic as S

    if args.batch > 0:
        inst = S.batched_instances(512, seed=1004)[:args.batch]
        probs = [dict(n=q["n"], k=q["k"], edges=q["edges"], alpha=args.alpha) for q in inst]
        bt = Batch(probs, [q["rho0"] for q in inst], [q["rho1"] for q in inst], device=0)
        ms = 0.0
        for _ in range(max(1, args.repeat)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bt.solve(max_iters=args.iters, check_every=args.check_every, tol_gap=args.tol, tol_res=args.tol,
                     path=args.path)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        rs = bt.results
        print(json.dumps(dict(batch=args.batch, path=args.path, ms=ms, iters=sum(r["iters"] for r in rs),
                              gp_it=sum(q["n"] ** 2 * r["iters"] for q, r in zip(inst, rs)),
                              max_blocks=max(r["blocks"] for r in rs))), flush=True)
        return

    if args.matrix:
        gen = S.tensor_field_pair3 if args.dim == 3 else S.tensor_field_pair
        r0, r1 = gen(args.n, args.k, seed=args.seed)
        L = S.random_L(args.k, 3, seed=args.seed)
    elif args.dim == 3:
        r0, r1 = S.blob_pair3(args.n, args.k, seed=args.seed)
    else:
        r0, r1 = S.color_image_pair(args.n, args.k, seed=args.seed)
    dev = torch.device("cuda", 0)
    d0 = torch.from_numpy(r0.astype(np.float32)).to(dev)
    d1 = torch.from_numpy(r1.astype(np.float32)).to(dev)
    edges = S.complete_graph(args.k)
    res, ms = None, 0.0
    kw = dict(max_iters=args.iters, check_every=args.check_every, tol_gap=args.tol, tol_res=args.tol, tau=args.tau)
    mkw = dict(u_norm=3, w_norm=2) if args.norms == "nuclear" else {}
    for _ in range(max(1, args.repeat)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.matrix and args.dim == 3:
            sol = momt_solve3d(d0, d1, L, args.alpha, zc=args.halo, **kw)
        elif args.matrix:
            sol = momt_solve(d0, d1, L, args.alpha, engine=args.engine, halo=args.halo, **mkw, **kw)
        elif args.dim == 3:
            sol = solve3d(d0, d1, edges, args.alpha, zc=args.halo, **kw)
        else:
            sol = solve(d0, d1, edges, args.alpha, engine=args.engine, halo=args.halo, **kw)
        e1.record()
        e1.synchronize()
        res, ms = sol.result, e0.elapsed_time(e1)
    print(json.dumps(dict(dim=args.dim, matrix=args.matrix, n=args.n, k=args.k, alpha=args.alpha, ms=ms, **res)),
          flush=True)


if __name__ == "__main__":
    main()
