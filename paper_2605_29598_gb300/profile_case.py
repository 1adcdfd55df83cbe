"""Run a few launches of one operator on a named workload, for profilers.

    python -m paper_2605_29598_gb300.profile_case --op vmult --reps 3
    python -m paper_2605_29598_gb300.profile_case --op explicit --cells 30 30 20
    python -m paper_2605_29598_gb300.profile_case --op precond --cells 30 30 20
    python -m paper_2605_29598_gb300.profile_case --op vmult --cells 30 30 20 \
        --precision fp64 mixed pairs --schedule 0 1 0

Builds the mesh and state of the hill workload (optionally with fewer
cells), prepares one set of implicit coefficients from the state and runs
`reps` applies of the chosen operator per precision named (no timing; pair
it with ncu -k).  --schedule sets the fused vmult schedule of FP64, FP32 and
FP32 pairs (1: neighbour node lines, 0: trace array, 2: one thread per
x-line) instead of the mesh default, --tile the cells per block of schedule 2.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["vmult", "explicit", "rhs", "recover", "precond"], default="vmult")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cells", type=int, nargs=3, default=[60, 60, 20])
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--refine", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "mixed", "pairs"], nargs="+", default=["fp64"])
    ap.add_argument("--schedule", type=int, nargs=3, default=None)
    ap.add_argument("--tile", type=int, default=None, help="cells-per-block multiplier of schedule 2")
    args = ap.parse_args()

    import torch

    from . import build as B
    from . import dgimex as D
    from . import inputs as I

    B.build()
    torch.cuda.set_device(0)
    nx, ny, nz = args.cells
    case = I.hill3d_case(nx=nx, ny=ny, nz=nz, r=args.degree, refine=args.refine)
    ctx = D.Context(0)
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    xyz = mesh.node_coords().cpu().numpy().T
    q = torch.tensor(I.stratified_state(xyz, **case["state_params"]), dtype=torch.float64,
                     device="cuda").contiguous()
    rho = q[0].contiguous()
    u = (q[1:4] / q[0]).contiguous()
    p = (0.4 * (q[4] - 0.5 * (q[1:4] * u).sum(0))).contiguous()
    cf = D.Mesh.coeffs(rho, p, u, 0.29289321881345254 * case["dt"])
    x = (p * (1 + 1e-3 * torch.randn_like(p))).contiguous()
    y = torch.empty_like(x)
    if args.schedule is not None:
        mesh.set_fused_stage(*args.schedule)
    if args.tile is not None:
        for prec in args.precision:
            mesh.set_vmult_tile(prec, args.tile)
    for prec in args.precision:
        phys = D.make_phys(f=case["f"], precision=prec)
        run(args, mesh, phys, q, cf, x, y)
    torch.cuda.synchronize()
    print(f"{args.op}: {args.reps} applies per precision ({' '.join(args.precision)}) on {mesh.n_elem} cells, "
          f"{mesh.N} nodes")


def run(args, mesh, phys, q, cf, x, y):
    for _ in range(args.reps):
        if args.op == "vmult":
            mesh.apply_implicit(phys, cf, x, y)
        elif args.op == "explicit":
            mesh.apply_explicit(phys, q)
        elif args.op == "precond":
            mesh.precond_apply(phys, cf, x, y)        # vertical-line setup + one solve
        elif args.op == "rhs":
            mesh.schur_rhs(phys, cf, q[1:4].contiguous(), q[4].contiguous(), y)
        else:
            mesh.recover_velocity(phys, cf, q[1:4].contiguous(), x)


if __name__ == "__main__":
    main()
