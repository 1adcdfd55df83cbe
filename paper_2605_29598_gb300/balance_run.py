"""Long-run geostrophic balance of the planetary-scale inertia-gravity wave.

Steps the 60 000 km x 10 km channel (300 x 20 cells, degree 4, dt = 10 s)
with the device-driven ARK2 step and prints the geostrophic imbalance E_geo
(domain mean of |(1/rho) dp/dx - f v|, the scheme's own discrete pressure
gradient and Coriolis term) every ``--every`` hours, with the largest
vertical velocity and the solver counters.

    python -m paper_2605_29598_gb300.balance_run --hours 96 --every 6
    python -m paper_2605_29598_gb300.balance_run --lambda-min 1 --precond   # stable, fast

--lambda-min floors the Rusanov coefficient of the non-stiff fluxes (not in
the paper; without it a checkerboard of vertical momentum grows at rest);
--precond runs the Schur GMRES with the vertical-line preconditioner.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--hours", type=float, default=96.0)
    ap.add_argument("--every", type=float, default=6.0)
    ap.add_argument("--dt", type=float, default=None, help="time step in s (default: the case's 10 s)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--host-loop", action="store_true", help="host-driven steps instead of the graph")
    ap.add_argument("--json", default=None, help="also write the table as JSON lines here")
    ap.add_argument("--lambda-min", type=float, default=0.0,
                    help="floor (m/s) of the non-stiff Rusanov coefficient (0: the paper's |u.n|)")
    ap.add_argument("--precond", action="store_true",
                    help="vertical-line preconditioner for the Schur GMRES")
    args = ap.parse_args(argv)

    import torch

    from . import build, dgimex as D, inputs as I

    build.build()
    case = I.planetary_igw_case()
    ctx = D.Context(0)
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    xyz = mesh.node_coords().cpu().numpy().T
    q = torch.tensor(I.isothermal_state(xyz, **case["state_params"]), dtype=torch.float64,
                     device="cuda").contiguous()
    phys = D.make_phys(f=case["f"], variant="R2", precision=args.precision, lambda_min=args.lambda_min)
    opts = dict(picard_rtol=1e-10, picard_maxit=10, gmres_rtol=1e-10, gmres_restart=30,
                gmres_maxit=1000, graph=not args.host_loop,
                gmres_inner_rtol=1e-4 if args.precision == "mixed" else 0.0,
                gmres_precond=args.precond)
    dt = case["dt"] if args.dt is None else args.dt
    steps_per_report = max(1, int(round(args.every * 3600.0 / dt)))
    n_reports = max(1, int(round(args.hours / args.every)))
    rows = []
    out = open(args.json, "w") if args.json else None

    def report(t_h, its, wall):
        e = mesh.geostrophic_error(phys, q)
        w = (q[3] / q[0]).abs().max().item()
        row = {"hours": round(t_h, 3), "dt": dt, "lambda_min": args.lambda_min, "E_geo": e, "max_abs_w": w,
               "gmres_iters": its, "wall_s": round(wall, 2)}
        rows.append(row)
        print(json.dumps(row), flush=True)
        if out:
            out.write(json.dumps(row) + "\n")

    report(0.0, 0, 0.0)
    t0 = time.time()
    for k in range(n_reports):
        its = 0
        try:
            for _ in range(steps_per_report):
                its += mesh.step(phys, q, dt, **opts).gmres_iters_total
        except D.DGError as err:   # e.g. a non-finite state: report and stop
            row = {"hours_reached_before": round(k * steps_per_report * dt / 3600.0, 3), "dt": dt,
                   "error": str(err)[:160]}
            rows.append(row)
            print(json.dumps(row), flush=True)
            break
        torch.cuda.synchronize()
        report((k + 1) * steps_per_report * dt / 3600.0, its, time.time() - t0)
    if out:
        out.close()
    return rows


if __name__ == "__main__":
    main()
