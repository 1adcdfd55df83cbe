"""Throughput benchmark of the IMEX-DG hot path on GB300.

Workload (default): 3D stratified flow over a bell hill, 200 x 200 x 20 km,
60 x 60 x 20 terrain-following hexes, degree 3 (4.608 M nodes x 5 fields,
FP64), N = 0.01 1/s, theta_ref = 293.15 K, inflow 10 m/s, f = 1e-4 1/s,
dt = 4 s, strategy R2, Picard to 1e-10 relative change, GMRES(30) to 1e-10
relative residual.  One step = one full ARK2 IMEX step (3 explicit
operators, 2 implicit stages with their Picard / Schur / GMRES work).

Metric: GDoF-updates/s = 5 * nodes * steps / time / 1e9 (whole job over all
ranks).  Multi-GPU runs are independent replicas (the solve has no data
exchange in this build); the per-rank work is fixed, so scaling is weak.

Printed JSON line: value (device time, inputs resident), e2e (host arrays
copied in and out every step), roofline of the dominant kernel class (CUDA
events around its launches inside the timed region), cpu_baseline (the FP64
oracle on a bounded sample, host cores), clocks sampled during the timed
region, and the number of library kernel launches in the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 FMA throughput (2 flops per FMA): GB300 nominal 1.25 TFLOP/s
FP64_NOMINAL_TFLOPS = 1.25
METRIC = "GDoF-updates/s per IMEX step"

STEP_OPTS = dict(picard_rtol=1e-10, picard_maxit=10, gmres_rtol=1e-10, gmres_restart=30,
                 gmres_maxit=3000)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


# ----------------------------------------------------------------------------
# algorithmic work per launch of each kernel class (FP64 flops, FMA = 2).
# Per-node / per-face-point counts follow the kernels' arithmetic; they are
# derived in the design notes (kernel table).
# ----------------------------------------------------------------------------

def work_model(dim, n, N, S, nF, nnz=None):
    """FP64 flops per launch.  nnz: nonzero metric terms K_ab per node (d^2,
    or 5 in 3D / 3 in 2D on terrain-following meshes, where the kernels skip
    the exact zeros); per pressure component b the number of directions a
    with K_ab != 0 sums to nnz."""
    d = dim
    nnz = d * d if nnz is None else nnz
    return {
        # fused gradient pass: per own face slot the centred value, its n dS
        # products and the penalty jump (d + 4; the plus value read from the
        # trace array), then sum_b sum_{a: K_ab != 0} (x K_ab) contraction +
        # lift of d+1 fields + pointwise
        "volume_grad": S * (d + 4) + N * (nnz + 2 * nnz * n + 2 * 2 * d * (d + 1) + 20),
        # fused divergence pass: per own slot both sides' w.n dS and the
        # centred h rho flux (4d + 4), then h rho K w, d contractions, lift of
        # 1 field, update
        "volume_div": S * (4 * d + 4) + N * (2 * nnz + d + 2 * d * n + 2 * 2 * d + 6),
        # K u, 6 flux fields x d contractions + 3 pressure fields x their
        # nonzero directions, lift of 9 fields
        "volume_explicit": N * (2 * nnz + 9 * d + 2 * (6 * d + nnz) * n + 2 * 2 * d * 9 + 30),
        "face_explicit": nF * 90,
        "face_grad": nF * (2 + d + 3),
        "face_div": nF * (4 * d + 4),
    }


# DRAM bytes per node of one launch, from an ncu capture of the current
# fused FP64 gradient pass (trace-array schedule) on the 30 x 30 x 20 hill
# (profiles/fused_vmult_hill3d_30x30x20_r3.md: 143.1 MB read + 21.2 MB
# written over 1 152 000 nodes), scaled to a launch by the nodes it processes.
NCU_TRAFFIC_B_PER_NODE = {"volume_grad": (143.097856e6 + 21.227776e6) / 1152000}


def bytes_model(dim, n, N, S, nF, nnz=None):
    d = dim
    nnz = d * d if nnz is None else nnz
    return {
        # x, metric, 1/(w det J), 1/rho, w out, y out; per slot: own and plus
        # traces, n dS, penalty coefficient
        "volume_grad": N * 8 * (1 + nnz + 1 + 1 + d + 1) + S * 8 * (2 + d + 1),
        # w, p_lag, metric, 1/(w det J), y in and out; per slot: both sides' w
        # traces and h rho traces, n dS
        "volume_div": N * 8 * (d + 1 + nnz + 1 + 1 + 1) + S * 8 * (2 * d + 2 + d),
        "volume_explicit": N * 8 * (5 + nnz + 1 + 9) + S * 8 * 9,
    }


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------
# the oracle on a bounded sample (host cores)
# ----------------------------------------------------------------------------

SAMPLE = dict(nx=2, ny=2)


def oracle_sample_main(steps, warmup, out_path):
    """Child process: time the FP64 oracle's ARK2 step on a 2 x 2 x 20-cell
    column of the hill workload (same cell size, degree, physics, dt and
    solver settings; hill centred in the sample)."""
    from oracle import dg_oracle as O
    from paper_2605_29598_gb300 import inputs as I
    nx, ny = SAMPLE["nx"], SAMPLE["ny"]
    dx = 200e3 / 60
    mesh = I.box_mesh((nx, ny, 20), (nx * dx, ny * dx, 20e3),
                      hill=dict(h0=400.0, a_c=10e3, xc=nx * dx / 2, yc=ny * dx / 2))
    disc = O.Discretisation(mesh, 3)
    q = I.stratified_state(disc.node_points(), theta_ref=293.15, n_bv=0.01, wind=(10.0, 0, 0))
    ph = O.Phys(f=1e-4)
    opts = O.StepOpts(picard_rtol=STEP_OPTS["picard_rtol"], picard_maxit=STEP_OPTS["picard_maxit"],
                      gmres_rtol=STEP_OPTS["gmres_rtol"], gmres_restart=STEP_OPTS["gmres_restart"],
                      gmres_maxit=STEP_OPTS["gmres_maxit"])
    for _ in range(warmup):
        q = O.imex_ark2_step(disc, ph, q, 4.0, opts)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        q = O.imex_ark2_step(disc, ph, q, 4.0, opts)
        times.append(time.perf_counter() - t0)
    nodes = disc.E * disc.Np
    with open(out_path, "w") as f:
        json.dump({"times": times, "nodes": nodes, "cells": disc.E}, f)


def host_description():
    """CPU model and logical core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle_child_cmd(path, steps, warmup):
    return [sys.executable, os.path.abspath(__file__), "--oracle-child", path,
            "--steps", str(steps), "--warmup", str(warmup)]


def run_oracle_sample(steps, warmup, all_cores=False):
    """The oracle on the column sample with one thread.  all_cores=True also
    runs one copy of the same sample per host core at once (independent
    processes, one thread each) and reports their aggregate throughput."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    subprocess.run(_oracle_child_cmd(path, steps, warmup), check=True, env=env, cwd=ROOT)
    with open(path) as f:
        r = json.load(f)
    os.unlink(path)
    t = sum(r["times"]) / len(r["times"])
    value = 5 * r["nodes"] / t / 1e9
    sample = (f"ARK2 steps of the FP64 oracle on a {SAMPLE['nx']}x{SAMPLE['ny']}x20-cell "
              f"column of the hill workload ({r['cells']} cells, degree 3, {r['nodes']} nodes, "
              f"same dt/physics/solver), mean of {len(r['times'])} step(s)")
    out = {"value": value, "unit": "GDoF-updates/s", "cores": 1, "kind": "oracle",
           "sample": sample, "seconds_per_step": t}
    out.update(host_description())
    if all_cores:
        ncores = os.cpu_count() or 1
        paths, procs = [], []
        for _ in range(ncores):
            fd, pth = tempfile.mkstemp(suffix=".json")
            os.close(fd)
            paths.append(pth)
            procs.append(subprocess.Popen(_oracle_child_cmd(pth, 1, 0), env=env, cwd=ROOT))
        ok = all(pr.wait() == 0 for pr in procs)
        if ok:
            ts = []
            for pth in paths:
                with open(pth) as f:
                    ts.append(sum(json.load(f)["times"]))
            tmax = max(ts)
            out["all_cores"] = {"value": 5 * r["nodes"] * ncores / tmax / 1e9, "unit": "GDoF-updates/s",
                                "cores": ncores, "seconds_per_step_slowest": tmax,
                                "how": "one single-threaded oracle process per core, each stepping "
                                       "its own copy of the column sample once; aggregate nodes / "
                                       "slowest process's step time"}
        for pth in paths:
            os.unlink(pth)
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_ensemble(D, I, ctx, steps, warmup):
    """32 uneven instances: FP64 one instance at a time (one mesh each) vs
    the batched ensemble (instances sharing (dim, degree) merged) in FP64
    and mixed precision, as host-driven steps and as one graph launch (also
    with the vertical-line preconditioner); whole-ensemble steps timed with
    CUDA events."""
    import torch
    cases = I.ensemble_cases()
    stream = torch.cuda.current_stream()
    states = []
    out = {"instances": len(cases), "cells": sum(c["mesh"].n_elem for c in cases)}

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), its

    # one at a time, FP64
    meshes = []
    for c in cases:
        m = D.Mesh(ctx, c["mesh"], c["degree"])
        xyz = m.node_coords().cpu().numpy().T
        q0 = torch.tensor(I.stratified_state(xyz, **c["state_params"]), dtype=torch.float64,
                          device="cuda").contiguous()
        meshes.append(m)
        states.append(q0)
    nodes = sum(m.N for m in meshes)
    out["nodes"] = nodes
    phys = [D.make_phys(f=c["f"]) for c in cases]

    def seq_steps(qs, n):
        its = 0
        for _ in range(n):
            for m, ph, c, q in zip(meshes, phys, cases, qs):
                its += m.step(ph, q, c["dt"], **STEP_OPTS).gmres_iters_total
        return its

    seq_steps([q.clone() for q in states], warmup)
    ms, its = timed(lambda: seq_steps([q.clone() for q in states], steps))
    out["fp64_one_at_a_time"] = {"value": 5.0 * nodes * steps / (ms / 1e3) / 1e9,
                                 "ms_per_step": ms / steps, "gmres_iters": its}
    for m in meshes:
        m.close()
    # batched
    ens = D.Ensemble(ctx, [c["mesh"] for c in cases], [c["degree"] for c in cases],
                     [c["f"] for c in cases])
    out["groups"] = ens.n_groups
    dts = [c["dt"] for c in cases]
    for prec, graph, pc in (("fp64", False, False), ("mixed", False, False), ("mixed", True, False),
                            ("mixed", True, True)):
        ph = D.make_phys(precision=prec)
        opts = dict(STEP_OPTS, gmres_inner_rtol=1e-4) if prec == "mixed" else dict(STEP_OPTS)
        opts["gmres_precond"] = pc

        def ens_steps(n):
            for i, q in enumerate(states):
                ens.set_state(i, q)
            its = 0
            for _ in range(n):
                its += ens.step(ph, dts, graph=graph, **opts).gmres_iters_total
            return its

        ens_steps(warmup)
        ms, its = timed(lambda: ens_steps(steps))
        out["batched_" + prec + ("_one_graph_launch" if graph else "") + ("_vline_precond" if pc else "")] = {
            "value": 5.0 * nodes * steps / (ms / 1e3) / 1e9, "ms_per_step": ms / steps, "gmres_iters": its}
    ens.close()
    out["unit"] = "GDoF-updates/s"
    out["steps"] = steps
    return out


def run_graph_modes(D, I, ctx, case, steps, warmup):
    """Host-driven vs device-driven (one CUDA graph per step) steps of a
    workload, FP64 and mixed, timed with CUDA events."""
    import torch
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    xyz = mesh.node_coords().cpu().numpy().T
    q0 = torch.tensor(I.stratified_state(xyz, **case["state_params"]), dtype=torch.float64,
                      device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    out = {"cells": mesh.stats().n_elem, "nodes": mesh.N, "degree": case["degree"], "dt": case["dt"],
           "steps": steps}
    for prec in ("fp64", "mixed"):
        phys = D.make_phys(f=case["f"], variant="R2", precision=prec)
        opts = dict(STEP_OPTS, gmres_inner_rtol=1e-4) if prec == "mixed" else STEP_OPTS
        res = {}
        for graph in (False, True):
            q = q0.clone()
            for _ in range(warmup):
                mesh.step(phys, q, case["dt"], graph=graph, **opts)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = 0
            for _ in range(steps):
                its += mesh.step(phys, q, case["dt"], graph=graph, **opts).gmres_iters_total
            e1.record(stream)
            torch.cuda.synchronize()
            res["graph" if graph else "host"] = {"ms_per_step": e0.elapsed_time(e1) / steps,
                                                 "gmres_iters": its}
        res["graph_speedup"] = res["host"]["ms_per_step"] / res["graph"]["ms_per_step"]
        out[prec] = res
    mesh.close()
    return out


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); ms itself without a
    process group."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(nodes_per_rank, steps, world, ms_max):
    """Whole-job GDoF-updates/s: every rank advances its own replica of
    nodes_per_rank nodes x 5 fields by `steps` steps; the job takes the
    slowest rank's time."""
    return 5.0 * nodes_per_rank * steps * world / (ms_max / 1e3) / 1e9


def run_per_operator(D, mesh, q, f, a_dt, hbm_gbs, reps=10):
    """Single applies of the boundary's operators on the bench workload, timed
    with CUDA events (3 warm-ups, `reps` timed): GDoF/s over the DoF each
    produces (explicit rates: 5 fields, Schur vmult and preconditioner solves:
    the pressure unknowns), and the fraction of the measured copy bandwidth
    their algorithmic bytes reach (explicit: 5 fields in, 9 rates out, 112
    B/node in FP64; vmult: x, y, rho, p_lag and the face lambda, about 38
    B/node).  Each is a whole entry-point call: the implicit applies also
    prepare their frozen coefficients (1/rho, h rho traces, face lambda; FP32
    copies in the mixed form), the preconditioner call also factors.  All of
    them are bound by the FP64 pipe or by latency, not by HBM."""
    import torch
    N = q.shape[1]
    rho = q[0].contiguous()
    u = (q[1:4] / q[0]).contiguous()
    p = (0.4 * (q[4] - 0.5 * (q[1:4] * u).sum(0))).contiguous()
    cf = D.Mesh.coeffs(rho, p, u, a_dt)
    x = (p * (1 + 1e-3 * torch.randn_like(p))).contiguous()
    y = torch.empty_like(x)
    fns = torch.empty((5, N), dtype=torch.float64, device="cuda")
    fs = torch.empty((4, N), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    rows = [
        ("apply_explicit_fp64", lambda: mesh.apply_explicit(D.make_phys(f=f), q, fns, fs), 5, 112),
        ("apply_implicit_fp64", lambda: mesh.apply_implicit(D.make_phys(f=f), cf, x, y), 1, 38),
        ("apply_implicit_mixed", lambda: mesh.apply_implicit(D.make_phys(f=f, precision="mixed"), cf, x, y), 1, 38),
        ("apply_implicit_pairs", lambda: mesh.apply_implicit(D.make_phys(f=f, precision="pairs"), cf, x, y), 1, 38),
        ("precond_vline_setup_and_solve", lambda: mesh.precond_apply(D.make_phys(f=f), cf, x, y), 1, None),
    ]
    for name, fn, fields, bpn in rows:
        ms = timed(fn)
        r = {"ms": ms, "gdof_per_s": fields * N / (ms / 1e3) / 1e9}
        if bpn:
            gbs = bpn * N / (ms / 1e3) / 1e9
            r.update({"algorithmic_bytes_per_node": bpn, "gb_per_s": gbs, "frac_of_measured_hbm": gbs / hbm_gbs})
        out[name] = r
    # the vmult kernels alone (the calls above also prepare their
    # coefficients): the fused gradient and divergence passes of each
    # precision, CUDA events per launch, and the FP32 pair against the HBM
    # roof at the two-pass algorithmic bytes (43 B/node in FP32: x, y, rho,
    # p_lag, face lambda and the intermediate w written and read once)
    st = mesh.stats()
    for prec, bpn in (("fp64", 86), ("mixed", 43), ("pairs", 86)):
        ph = D.make_phys(f=f, precision=prec)
        for _ in range(3):
            mesh.apply_implicit(ph, cf, x, y)
        torch.cuda.synchronize()
        D.profile_begin(mesh, timed=["volume_grad", "volume_div", "trace"])
        for _ in range(reps):
            mesh.apply_implicit(ph, cf, x, y)
        prof = D.profile_end(mesh)
        g, dv = prof["volume_grad"], prof["volume_div"]
        slot = {"fp64": 0, "mixed": 1, "pairs": 2}[prec]
        sched = st.fused_stage[slot]
        ms = (g[2] + dv[2]) / reps
        names = {0: "trace array (plus two trace passes per vmult, about trace_ms_per_launch each)",
                 1: "neighbour node lines", 2: "one thread per x-line"}
        r = {"grad_ms": g[2] / max(g[1], 1), "div_ms": dv[2] / max(dv[1], 1), "fused_passes_ms": ms,
             "schedule": names.get(sched, str(sched)),
             "trace_ms_per_launch": prof["trace"][2] / max(prof["trace"][1], 1)}
        if sched == 2 and prec != "pairs":
            r["cells_per_block_multiplier"] = (st.tile_fp64 if prec == "fp64" else st.tile_fp32)[1]
        if prec == "mixed":
            gbs = bpn * N / (ms / 1e3) / 1e9
            r.update({"algorithmic_bytes_per_node": bpn, "gb_per_s": gbs, "frac_of_measured_hbm": gbs / hbm_gbs})
        out["vmult_kernels_" + prec] = r
    return out


def run_variant(D, I, ctx, case, steps, warmup, precond=False, state=None, sponge=None):
    """FP64 and mixed steps of another workload (timed with CUDA events);
    precond=True runs the Schur GMRES with the vertical-line preconditioner;
    sponge: keyword arguments of Mesh.set_sponge (damping towards the start
    state)."""
    import torch
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    st = mesh.stats()
    xyz = mesh.node_coords().cpu().numpy().T
    state = state or I.stratified_state
    q0 = torch.tensor(state(xyz, **case["state_params"]), dtype=torch.float64,
                      device="cuda").contiguous()
    out = {"cells": st.n_elem, "nodes": st.n_nodes, "hanging_points": st.n_hang_points,
           "degree": case["degree"], "dt": case["dt"], "gmres_precond": "vline" if precond else "none"}
    if sponge:
        mesh.set_sponge(q0, **sponge)
        out["sponge"] = {k: v for k, v in sponge.items()}
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "mixed"):
        phys = D.make_phys(f=case["f"], variant="R2", precision=prec)
        opts = dict(STEP_OPTS, gmres_inner_rtol=1e-4) if prec == "mixed" else dict(STEP_OPTS)
        opts["gmres_precond"] = precond
        q = q0.clone()
        for _ in range(warmup):
            mesh.step(phys, q, case["dt"], **opts)
        q = q0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for _ in range(steps):
            its += mesh.step(phys, q, case["dt"], **opts).gmres_iters_total
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[prec] = {"value": 5.0 * st.n_nodes * steps / (ms / 1e3) / 1e9, "unit": "GDoF-updates/s",
                     "ms_per_step": ms / steps, "gmres_iters": its, "steps": steps}
    mesh.close()
    return out

def pert_fields(s, gamma=1.4, R=287.0, p_ref=1e5):
    """rho, potential temperature theta, u, v, w of a state (5, N)."""
    u = s[1:4] / s[0]
    p = (gamma - 1.0) * (s[4] - 0.5 * (s[1:4] * u).sum(0))
    theta = p / (R * s[0]) * (p_ref / p) ** ((gamma - 1.0) / gamma)
    return {"rho": s[0], "theta": theta, "u": u[0], "v": u[1], "w": u[2]}


def perturbation_errors(test, ref, bg):
    """Relative L2 error per perturbation field: ||phi(test) - phi(ref)|| /
    ||phi(ref) - phi(bg)||, phi' = phi - phi(bg) about the background bg
    (rho', theta', u' = u - U, v, w)."""
    import torch
    ft, fr, fb = pert_fields(test), pert_fields(ref), pert_fields(bg)
    out = {}
    for k in fr:
        den = torch.linalg.norm(fr[k] - fb[k]).item()
        out[k] = torch.linalg.norm(ft[k] - fr[k]).item() / den if den > 0 else None
    return out


def timed_steps(mesh, phys, q, dt, steps, opts):
    """`steps` ARK2 steps of q in place, bracketed by CUDA events on the
    current stream: (ms, GMRES iterations, FP64 refinement sweeps)."""
    import torch
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its, ref = 0, 0
    for _ in range(steps):
        inf = mesh.step(phys, q, dt, **opts)
        its += inf.gmres_iters_total
        ref += inf.refinements_total
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), its, ref


PRECISION_OPTS = dict(picard_rtol=1e-12, picard_maxit=20, gmres_rtol=1e-12, gmres_restart=30,
                      gmres_maxit=6000)
REFERENCE_OPTS = dict(picard_rtol=1e-13, picard_maxit=30, gmres_rtol=1e-13, gmres_restart=30,
                      gmres_maxit=8000)


def run_precision_pattern(D, mesh, q_bg, f, dt, steps):
    """The precision pattern at tolerances where FP64 itself is accurate to
    well below 1e-6 in the perturbation fields: FP64 and DG_MIXED steps
    (Picard and GMRES / refinement to 1e-12) from the background state,
    timed with CUDA events, and both against an FP64 run at 1e-13 from the
    same start (the FP64 path is parity-tested against the oracle; the
    oracle itself cannot run this mesh)."""
    import torch
    out = {"steps": steps, "start": "background state (t = 0)",
           "tolerances": "Picard 1e-12, GMRES / iterative refinement 1e-12 (FP32 inner 1e-4); "
                         "reference FP64 at 1e-13"}
    q64 = q_bg.clone()
    ph64 = D.make_phys(f=f, variant="R2")
    phmx = D.make_phys(f=f, variant="R2", precision="mixed")
    mesh.step(phmx, q_bg.clone(), dt, **dict(PRECISION_OPTS, gmres_inner_rtol=1e-4))  # FP32 copies
    ms64, it64, _ = timed_steps(mesh, ph64, q64, dt, steps, PRECISION_OPTS)
    qmx = q_bg.clone()
    msmx, itmx, refmx = timed_steps(mesh, phmx, qmx, dt, steps, dict(PRECISION_OPTS, gmres_inner_rtol=1e-4))
    phpr = D.make_phys(f=f, variant="R2", precision="pairs")
    mesh.step(phpr, q_bg.clone(), dt, **PRECISION_OPTS)   # pair geometry once
    qpr = q_bg.clone()
    mspr, itpr, _ = timed_steps(mesh, phpr, qpr, dt, steps, PRECISION_OPTS)
    qref = q_bg.clone()
    timed_steps(mesh, ph64, qref, dt, steps, REFERENCE_OPTS)
    N = q_bg.shape[1]
    out["fp64"] = {"value": 5.0 * N * steps / (ms64 / 1e3) / 1e9, "ms_per_step": ms64 / steps,
                   "gmres_iters": it64, "rel_l2_err_vs_reference": perturbation_errors(q64, qref, q_bg)}
    out["mixed"] = {"value": 5.0 * N * steps / (msmx / 1e3) / 1e9, "ms_per_step": msmx / steps,
                    "gmres_inner_iters": itmx, "fp64_refinement_sweeps": refmx,
                    "rel_l2_err_vs_reference": perturbation_errors(qmx, qref, q_bg),
                    "rel_l2_err_vs_fp64": perturbation_errors(qmx, q64, q_bg)}
    out["pairs"] = {"value": 5.0 * N * steps / (mspr / 1e3) / 1e9, "ms_per_step": mspr / steps,
                    "gmres_iters": itpr, "rel_l2_err_vs_reference": perturbation_errors(qpr, qref, q_bg),
                    "what": "Schur vmults in pairs of FP32 numbers (an FP64-class emulation), FP64 GMRES"}
    out["mixed_speedup_vs_fp64"] = ms64 / msmx
    out["pairs_speedup_vs_fp64"] = ms64 / mspr
    out["unit"] = "GDoF-updates/s"
    return out


def run_refined_configs(D, I, ctx, steps, warmup, err_steps=3):
    """The non-conforming hill (2:1 hanging faces around the hill, Section
    4.3's refinement shape): FP64 with the headline's solver settings
    (config 3) and the precision pattern with iterative refinement to 1e-8
    (config 4), `steps` steps each timed with CUDA events; then, from the
    background state over `err_steps` steps, the per-field error of the
    config-4 setting and of FP64 at the same 1e-8 tolerance against an FP64
    run at 1e-12."""
    import torch
    case = I.hill3d_case(refine=True)
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    mesh.autotune("mixed")
    st = mesh.stats()
    xyz = mesh.node_coords().cpu().numpy().T
    q_bg = torch.tensor(I.stratified_state(xyz, **case["state_params"]), dtype=torch.float64,
                        device="cuda").contiguous()
    dt, f = case["dt"], case["f"]
    N = st.n_nodes
    ph64 = D.make_phys(f=f, variant="R2")
    phmx = D.make_phys(f=f, variant="R2", precision="mixed")
    c4_opts = dict(STEP_OPTS, gmres_rtol=1e-8, gmres_inner_rtol=1e-4)
    geo = {"cells": st.n_elem, "nodes": N, "hanging_points": st.n_hang_points, "degree": case["degree"],
           "dt": dt, "terrain_following": st.terrain_following,
           "schedule_tiles_fp64_fp32_fused_stage": [list(st.tile_fp64), list(st.tile_fp32), list(st.fused_stage)]}
    q = q_bg.clone()
    for _ in range(warmup):
        mesh.step(ph64, q, dt, **STEP_OPTS)
    q3 = q.clone()
    ms3, it3, _ = timed_steps(mesh, ph64, q3, dt, steps, STEP_OPTS)
    cfg3 = dict(geo, workload="hill3d_nc_60x60x20_r3_fp64_R2", value=5.0 * N * steps / (ms3 / 1e3) / 1e9,
                unit="GDoF-updates/s", ms_per_step=ms3 / steps, steps=steps, gmres_iters=it3,
                solver="Picard 1e-10, GMRES(30) 1e-10, unpreconditioned")
    q4 = q.clone()
    mesh.step(phmx, q.clone(), dt, **c4_opts)
    ms4, it4, ref4 = timed_steps(mesh, phmx, q4, dt, steps, c4_opts)
    qe_ref = q_bg.clone()
    timed_steps(mesh, ph64, qe_ref, dt, err_steps, dict(PRECISION_OPTS, picard_rtol=1e-12))
    qe_mx = q_bg.clone()
    timed_steps(mesh, phmx, qe_mx, dt, err_steps, c4_opts)
    qe_64 = q_bg.clone()
    timed_steps(mesh, ph64, qe_64, dt, err_steps, dict(STEP_OPTS, gmres_rtol=1e-8))
    # the same precision pattern with refinement to 1e-12 (Picard 1e-12)
    qe_mx12 = q_bg.clone()
    ms12, _, _ = timed_steps(mesh, phmx, qe_mx12, dt, err_steps,
                             dict(PRECISION_OPTS, picard_rtol=1e-12, gmres_inner_rtol=1e-4))
    cfg4 = dict(geo, workload="hill3d_nc_60x60x20_r3_mixed_R2", value=5.0 * N * steps / (ms4 / 1e3) / 1e9,
                unit="GDoF-updates/s", ms_per_step=ms4 / steps, steps=steps, gmres_inner_iters=it4,
                fp64_refinement_sweeps=ref4, speedup_vs_config3=ms3 / ms4,
                solver="Picard 1e-10, iterative refinement to 1e-8 (FP32 GMRES(30) inner 1e-4)",
                rel_l2_err_vs_fp64_1e12=perturbation_errors(qe_mx, qe_ref, q_bg),
                fp64_same_tolerance_rel_l2_err_vs_fp64_1e12=perturbation_errors(qe_64, qe_ref, q_bg),
                mixed_refined_to_1e12={"rel_l2_err_vs_fp64_1e12": perturbation_errors(qe_mx12, qe_ref, q_bg),
                                       "ms_per_step": ms12 / err_steps},
                error_run=f"{err_steps} steps from the background state; the reference is FP64 with "
                          "Picard and GMRES to 1e-12")
    mesh.close()
    return cfg3, cfg4


def run_balance(D, I, ctx, case, hours):
    """E_geo of the planetary-scale wave after `hours` of simulated time
    (dt = 10 s, FP64, R2) with the non-stiff Rusanov floor of 1 m/s and the
    vertical-line preconditioner (the configuration that runs the paper's
    96 h stably), device-driven steps; wall time of the steps."""
    import time

    import torch
    mesh = D.Mesh(ctx, case["mesh"], case["degree"])
    xyz = mesh.node_coords().cpu().numpy().T
    q = torch.tensor(I.isothermal_state(xyz, **case["state_params"]), dtype=torch.float64,
                     device="cuda").contiguous()
    phys = D.make_phys(f=case["f"], lambda_min=1.0)
    nsteps = int(round(hours * 3600.0 / case["dt"]))
    its = 0
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(nsteps):
        its += mesh.step(phys, q, case["dt"], picard_rtol=1e-10, picard_maxit=10, gmres_rtol=1e-10,
                         gmres_restart=30, gmres_maxit=1000, gmres_precond=True, graph=True).gmres_iters_total
    torch.cuda.synchronize()
    wall = time.time() - t0
    out = {"hours": hours, "steps": nsteps, "dt": case["dt"], "lambda_min": 1.0, "gmres_precond": "vline",
           "graph": True,
           "E_geo": mesh.geostrophic_error(phys, q), "max_abs_w": (q[3] / q[0]).abs().max().item(),
           "gmres_iters": its, "wall_s": wall, "paper_level": "E_geo < 1e-7 over 96 h"}
    mesh.close()
    return out


def gpu_main(args):
    import torch

    from paper_2605_29598_gb300 import build as B
    from paper_2605_29598_gb300 import dgimex as D
    from paper_2605_29598_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    B.build()

    case = I.hill3d_case()
    mesh_h = case["mesh"]
    r = case["degree"]
    ctx = D.Context(dev)
    mesh = D.Mesh(ctx, mesh_h, r)
    tiles = mesh.autotune("mixed")
    tiles = [tiles[0], tiles[1], mesh.autotune("pairs")[2]]
    if args.schedule is not None:
        # fixed fused vmult schedule (a profiler slows launches unevenly, so
        # the timed choice made under it can differ from the plain run's)
        mesh.set_fused_stage(*args.schedule)
        tiles[2] = list(args.schedule)
    st = mesh.stats()
    N = st.n_nodes
    xyz = mesh.node_coords().cpu().numpy().T
    q0 = I.stratified_state(xyz, **case["state_params"])
    q = torch.tensor(q0, dtype=torch.float64, device="cuda").contiguous()
    q_bg = q.clone()
    # FP64 / FP32 FMA roofs of this GPU (library probe, before the timed work)
    fma_peaks = {}
    for bits in (64, 32):
        runs = [D.probe_fma(ctx, bits) for _ in range(5)]
        fma_peaks["fp%d_fma" % bits] = {"tflops_best": max(x[0] for x in runs),
                                         "tflops_median": statistics.median(x[0] for x in runs)}
    phys = D.make_phys(f=case["f"], variant="R2")
    dt = case["dt"]
    stream = torch.cuda.current_stream()

    def step(qq):
        return mesh.step(phys, qq, dt, **STEP_OPTS)

    infos = []
    for _ in range(args.warmup):
        infos.append(step(q))
    torch.cuda.synchronize()

    # one profiled step with every class timed: breakdown and dominant class
    D.profile_begin(mesh, timed=D.KERNEL_CLASSES)
    step(q)
    prof_all = D.profile_end(mesh)
    dominant = max(prof_all, key=lambda k: prof_all[k][2])

    q_start = q.clone()
    # timed region: launches counted, dominant class bracketed by events
    clocks = ClockSampler(dev)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    D.profile_begin(mesh, timed=[dominant])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    picard, gm_its, relres = [], 0, 0.0
    for _ in range(args.steps):
        inf = step(q)
        picard.append(list(inf.picard_iters)[1:])
        gm_its += inf.gmres_iters_total
        relres = max(relres, inf.max_relres)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = D.profile_end(mesh)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = throughput(N, args.steps, world, ms_max)

    # end to end: the timed steps again from the same start state (same
    # iterations), with the host state copied in and out around every step
    qh = torch.empty_like(q, device="cpu").pin_memory()
    qh.copy_(q_start)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    qd = torch.empty_like(q)
    e2e_gmres = 0
    e2.record(stream)
    for _ in range(args.steps):
        qd.copy_(qh, non_blocking=True)
        e2e_gmres += step(qd).gmres_iters_total
        qh.copy_(qd, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist, "cuda")
    e2e_value = throughput(N, args.steps, world, ms_e2e)
    state_bytes = 5 * N * 8

    # mixed precision (FP32 Schur vmults under FP64 refinement) at the
    # headline's solver settings, from the same start state
    mixed = None
    if not args.no_mixed:
        phys_mx = D.make_phys(f=case["f"], variant="R2", precision="mixed")
        mx_opts = dict(STEP_OPTS, gmres_inner_rtol=1e-4)
        mesh.step(phys_mx, q_start.clone(), dt, **mx_opts)       # allocates FP32 copies once
        qm = q_start.clone()
        ms_mx, mx_its, mx_ref = timed_steps(mesh, phys_mx, qm, dt, args.steps, mx_opts)
        ms_mx = max_over_ranks(ms_mx, dist, "cuda")
        qp = q_start.clone()
        D.profile_begin(mesh, timed=D.KERNEL_CLASSES)
        mesh.step(phys_mx, qp, dt, **mx_opts)
        prof_mx = D.profile_end(mesh)
        mixed = {"value": throughput(N, args.steps, world, ms_mx), "unit": "GDoF-updates/s",
                 "ms_per_step": ms_mx / args.steps, "speedup_vs_fp64": ms_max / ms_mx,
                 "gmres_inner_total": mx_its, "fp64_refinement_sweeps": mx_ref, "inner_rtol": 1e-4,
                 "what_is_fp32": "Schur vmults inside the Krylov solves (FP32 accumulation)",
                 "accuracy": "see precision_pattern (same mode at 1e-12 tolerances, per-field errors)",
                 "kernel_breakdown_one_step": {k: {"launches": v[0], "ms": round(v[2], 3)}
                                               for k, v in prof_mx.items() if v[0]}}

    # roofline of the dominant class, against the FP64 FMA rate measured by
    # the library's probe in this run (best of 5 launches)
    pk, src = peaks()
    fp64_peak = fma_peaks["fp64_fma"]["tflops_best"]
    nnz = (5 if st.dim == 3 else 3) if st.terrain_following else st.dim * st.dim
    work = work_model(st.dim, st.n1d, N, N // st.nodes_per_elem * 2 * st.dim * st.n1d ** (st.dim - 1),
                      st.n_face_points, nnz)
    launches, timed_launches, tms = prof[dominant]
    roof = None
    if timed_launches:
        per_launch_ms = tms / timed_launches
        flops = work.get(dominant)
        achieved = flops / (per_launch_ms / 1e3) / 1e12 if flops else None
        roof = {"bound": "alu", "kernel": dominant, "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak if achieved else None,
                # the capture is of the trace-array FP64 schedule only
                "traffic": (NCU_TRAFFIC_B_PER_NODE[dominant] * N
                            if dominant in NCU_TRAFFIC_B_PER_NODE and st.dim == 3 and st.n1d == 4
                            and tiles[2][0] == 0 else None),
                "peak_source": "measured in this run: dg_probe_fma, FP64 FMA chains filling every SM "
                               "(best of 5); nominal GB300 FP64 1.25 TFLOP/s",
                "frac_of_nominal_fp64": achieved / FP64_NOMINAL_TFLOPS if achieved else None,
                "launches": timed_launches, "ms_per_launch": per_launch_ms,
                "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": bytes_model(
                    st.dim, st.n1d, N, st.n_elem * 2 * st.dim * st.n1d ** (st.dim - 1),
                    st.n_face_points, nnz).get(dominant),
                "nonzero_metric_terms_per_node": nnz}
    total_launches = sum(v[0] for v in prof.values())
    breakdown = {k: {"launches": v[0], "ms": round(v[2], 3)} for k, v in prof_all.items() if v[0]}

    precision = None
    if not args.no_mixed and world == 1:
        precision = run_precision_pattern(D, mesh, q_bg, case["f"], dt, min(args.steps, 10))

    variants = {}
    per_op = None
    cfg3 = cfg4 = None
    if not args.no_variants and world == 1:
        per_op = run_per_operator(D, mesh, q, case["f"], 0.29289321881345254 * dt, pk["hbm_gbs"])
        cfg3, cfg4 = run_refined_configs(D, I, ctx, args.steps, 1)
        variants["hill3d_vline_precond"] = run_variant(D, I, ctx, I.hill3d_case(), steps=2, warmup=1,
                                                       precond=True)
        h3 = I.hill3d_case()
        variants["hill3d_damped"] = run_variant(
            D, I, ctx, h3, steps=2, warmup=1,
            sponge=dict(lambda_bar=1.2 / h3["dt"], z_b=14e3, z_t=20e3, x_layers=(0.0, 200e3, 20e3),
                        y_layers=(0.0, 200e3, 20e3)))
        pw = I.planetary_igw_case()
        variants["planetary_igw"] = run_variant(D, I, ctx, pw, steps=4, warmup=1, state=I.isothermal_state)
        variants["planetary_igw_vline_precond"] = run_variant(D, I, ctx, pw, steps=4, warmup=1, precond=True,
                                                              state=I.isothermal_state)
        variants["planetary_igw_balance_6h"] = run_balance(D, I, ctx, pw, hours=6.0)
        variants["ensemble32"] = run_ensemble(D, I, ctx, steps=2, warmup=1)
        variants["graph_mode_hill3d"] = run_graph_modes(D, I, ctx, I.hill3d_case(), steps=3, warmup=2)
        variants["graph_mode_igw2d"] = run_graph_modes(D, I, ctx, I.igw2d_case(), steps=10, warmup=2)

    if dist and rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_oracle_sample(steps=2, warmup=0, all_cores=True)
        except Exception as exc:  # report, do not fail the bench
            cpu = {"error": str(exc)[:200]}

    def r3(x):
        if isinstance(x, float):
            return float("%.3g" % x)
        if isinstance(x, dict):
            return {k: r3(v) for k, v in x.items()}
        return x

    # the driver keeps the end of stdout: the compact summary goes last
    summary = {"fp64": {"gdof_s": r3(value), "ms_step": r3(ms_max / args.steps)}}
    if mixed:
        summary["mixed_same_tol"] = {"gdof_s": r3(mixed["value"]), "speedup": r3(mixed["speedup_vs_fp64"])}
    if precision:
        summary["precision_1e-12"] = {
            "fp64_ms": r3(precision["fp64"]["ms_per_step"]), "mixed_ms": r3(precision["mixed"]["ms_per_step"]),
            "speedup": r3(precision["mixed_speedup_vs_fp64"]),
            "mixed_err": r3(max(precision["mixed"]["rel_l2_err_vs_reference"].values())),
            "fp64_err": r3(max(precision["fp64"]["rel_l2_err_vs_reference"].values())),
            "pairs_ms": r3(precision["pairs"]["ms_per_step"]),
            "pairs_speedup": r3(precision["pairs_speedup_vs_fp64"]),
            "pairs_err": r3(max(precision["pairs"]["rel_l2_err_vs_reference"].values()))}
    if cfg3:
        summary["config3_nc_fp64"] = {"gdof_s": r3(cfg3["value"]), "ms_step": r3(cfg3["ms_per_step"]),
                                      "gmres": cfg3["gmres_iters"], "steps": cfg3["steps"]}
        summary["config4_nc_mixed"] = {"gdof_s": r3(cfg4["value"]), "ms_step": r3(cfg4["ms_per_step"]),
                                       "speedup": r3(cfg4["speedup_vs_config3"]),
                                       "err_1e-8": r3(max(cfg4["rel_l2_err_vs_fp64_1e12"].values())),
                                       "fp64_err_1e-8": r3(max(
                                           cfg4["fp64_same_tolerance_rel_l2_err_vs_fp64_1e12"].values())),
                                       "err_1e-12": r3(cfg4["mixed_refined_to_1e12"]["rel_l2_err_vs_fp64_1e12"])}
    if per_op:
        vk = {p: per_op["vmult_kernels_" + p] for p in ("fp64", "mixed", "pairs")}
        summary["vmult_fused_us"] = {p: r3(1e3 * v["fused_passes_ms"]) for p, v in vk.items()}
        summary["fp32_vmult_frac_hbm"] = r3(vk["mixed"]["frac_of_measured_hbm"])
    if roof:
        summary["roofline"] = {"kernel": dominant, "frac_of_measured_fp64": r3(roof["frac"]),
                               "fp64_peak_tflops": r3(fp64_peak),
                               "fp32_peak_tflops": r3(fma_peaks["fp32_fma"]["tflops_best"])}
    line = {
        "metric": METRIC, "value": value, "unit": "GDoF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "hill3d_60x60x20_r3_fp64_R2", "cells": st.n_elem, "degree": r,
                   "nodes": N, "dof": 5 * N, "dt": dt, "variant": "R2",
                   "picard_rtol": STEP_OPTS["picard_rtol"], "gmres_rtol": STEP_OPTS["gmres_rtol"],
                   "gmres_restart": STEP_OPTS["gmres_restart"],
                   "l2": "state (%.0f MB) and Krylov basis exceed the 126 MB L2" % (state_bytes / 1e6),
                   "parallelism": "replicas" if world > 1 else "single",
                   "schedule_tiles_fp64_fp32_fused_stage": tiles},
        "variants": variants,
        "per_operator": per_op,
        "kernel_breakdown_one_step": breakdown,
        "mixed_precision": mixed,
        "precision_pattern": precision,
        "config3": cfg3,
        "config4": cfg4,
        "fma_peaks": fma_peaks,
        "peaks_source": src,
        "iterations": {"picard_per_stage": picard[:3], "gmres_total": gm_its, "gmres_max_relres": relres},
        "e2e": {"value": e2e_value, "unit": "GDoF-updates/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "gmres_total": e2e_gmres},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": total_launches,
        "summary": summary,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference_main(args):
    """The oracle as it stands, on host cores, on a bounded sample of the
    same workload (rank 0 only)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle_sample(steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": "GDoF-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["seconds_per_step"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "hill3d_60x60x20_r3_fp64_R2", "sample": res["sample"]},
        "cpu_baseline": {"value": res["value"], "unit": res["unit"], "cores": res["cores"],
                         "kind": "oracle", "sample": res["sample"], "nproc": res.get("nproc"),
                         "cpu_model": res.get("cpu_model")},
        "e2e": {"value": res["value"], "unit": "GDoF-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--schedule", type=int, nargs=3, default=None,
                    help="fused vmult schedule of FP64, FP32, pairs (1: node lines, 0: trace array, "
                         "2: one thread per x-line) "
                         "instead of the timed choice")
    ap.add_argument("--oracle-child", default=None)
    args = ap.parse_args()
    if args.oracle_child:
        oracle_sample_main(args.steps, args.warmup, args.oracle_child)
        return
    if args.warmup < 3 and args.oracle_child is None and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_main(args)
    else:
        gpu_main(args)


if __name__ == "__main__":
    main()
