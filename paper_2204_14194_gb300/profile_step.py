"""Run a few steps of the headline workload through the C ABI, for profilers.

One step = what bench.py times: the table is dropped and rebuilt (Alg. 2),
then the 4096 blocks of 32 x 32 (16 x 16 loss area, DCT u WHT, K = 2048,
I = 100) go through se_extrapolate_strided.  No timing, no L2 flush; every
kernel launch of a step belongs to the method.

    python -m paper_2204_14194_gb300.profile_step [--steps 2] [--products auto|dense|transform] [--prec bf16x6|fp64]

With --masked M (16, 32 or 64) it runs instead the M x M third of the mixed
workload with per-block masks (K = 2MN, DCT u WHT, I from 50 to 500, the
lazy columns of eq. 16), --blocks blocks, one batch call per step with CUDA
graphs off so that every round's kernels are launched one by one.
"""
import argparse

import torch

from . import binding as B
from . import workloads as W


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--products", default="auto", choices=["auto", "dense", "transform"])
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "bf16", "fp64"])
    ap.add_argument("--blocks", type=int, default=4096)
    ap.add_argument("--masked", type=int, default=0, choices=[0, 16, 32, 64])
    args = ap.parse_args()
    if args.masked:
        return masked(args)
    wl = W.config2(args.blocks)
    ctx = B.Context(0)
    plan = ctx.plan(wl.M, wl.N, wl.basis, wl.K, wl.rho_hat, wl.gamma, wl.iterations, prec=args.prec,
                    products=args.products)
    s = torch.from_numpy(wl.samples).cuda()
    o = torch.empty_like(s)
    u = torch.empty((wl.B, wl.iterations), dtype=torch.int32, device="cuda")
    c = torch.empty((wl.B, wl.iterations), dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        plan.reset_tables()
        plan.extrapolate_strided(s, o, u, c)
    ctx.sync()
    print(f"{args.steps} steps of {wl.B} blocks done ({args.prec}, products={args.products})")
    plan.close()
    ctx.close()
    return 0


def masked(args) -> int:
    M = args.masked
    g = [x for x in W.config4(3 * args.blocks) if x.M == M][0]
    ctx = B.Context(0)
    ctx.set_graphs(False)
    I = int(g.iters_per_block.max())
    plan = ctx.plan(M, M, "dct_wht", g.K, g.rho_hat, g.gamma, I, prec=args.prec)
    s = torch.from_numpy(g.samples).cuda()
    m = torch.from_numpy(g.support).cuda()
    o = torch.empty_like(s)
    descs = [{"samples": s[b], "support": m[b], "out": o[b], "iterations": int(g.iters_per_block[b])}
             for b in range(g.B)]
    for _ in range(args.steps):
        plan.extrapolate_batch(descs)
    ctx.sync()
    print(f"{args.steps} steps of {g.B} masked {M}x{M} blocks done ({args.prec}, I up to {I})")
    plan.close()
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
