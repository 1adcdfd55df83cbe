"""Measure the FP64 and FP32 FMA roofs of the current GPU.

``python -m paper_2605_29598_gb300.peaks`` runs the library's FMA probe
(``dg_probe_fma``) a few times per precision while ``nvidia-smi`` samples
the SM clock, and prints one JSON line: best and median TFLOP/s per
precision, the kernel times, and the clocks seen during the probes.  The
FP64 figure is the arithmetic roof of the FP64 cell kernels (their
roofline denominator); the FP32 one that of the mixed-precision kernels.
"""
from __future__ import annotations

import json
import statistics
import subprocess
import tempfile
import time


def _clock_sampler(index):
    fd, path = tempfile.mkstemp(suffix=".csv")
    f = open(path, "w")
    try:
        proc = subprocess.Popen(["nvidia-smi", "-i", str(index),
                                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                                 "--format=csv,noheader,nounits", "-lms", "100"],
                                stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        proc = None
    return proc, path, f


def measure(reps: int = 5):
    import torch

    from . import build, dgimex as D
    build.build()
    dev = torch.cuda.current_device()
    ctx = D.Context(dev)
    proc, path, fh = _clock_sampler(dev)
    time.sleep(0.3)
    out = {"device": torch.cuda.get_device_name(dev)}
    for bits in (64, 32):
        runs = [D.probe_fma(ctx, bits) for _ in range(reps)]
        tf = [r[0] for r in runs]
        out[f"fp{bits}_fma"] = {"tflops_best": max(tf), "tflops_median": statistics.median(tf),
                                "ms_per_launch": [round(r[1], 3) for r in runs],
                                "iters": 8192 if bits == 64 else 524288}
    clocks = None
    if proc is not None:
        proc.terminate()
        proc.wait(timeout=5)
        fh.close()
        sm, mx, reasons = [], [], set()
        with open(path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 3 and parts[0].replace(".", "").isdigit():
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                    reasons.add(parts[2])
        if sm:
            clocks = {"sm_mhz_median": statistics.median(sm), "sm_mhz_min": min(sm),
                      "sm_max_mhz": max(mx), "reasons_active_masks": sorted(reasons), "samples": len(sm)}
    out["clocks"] = clocks
    ctx.close()
    return out


if __name__ == "__main__":
    print(json.dumps(measure()), flush=True)
