"""Accuracy of the reduced-precision storage modes against FP64 on the GPU.

Runs the thermoacoustic case (Gaussian density pulse 1e-2, sigma 8 cells, plus
a 16^3-Fourier-box temperature perturbation of max 1e-3, nu = 0.01) on an n^3
grid for `steps` steps in FP64 (the GPU FP64 mode, itself matched to the CPU
oracle to 1e-12 on small grids), FP32, FP32 + FP16 storage and FP32 + BF16
storage, and reports for each the relative L2 error of the density
fluctuation rho - 1 and of the temperature fluctuation theta - theta0 against
FP64, the maximum absolute density error, and the drift of the global mass
and energy sums.

    python -m paper_1909_08406_gb300.accuracy_report [--n 512] [--steps 500]

Prints one JSON object.  The reductions are the library's own kernels
(lb_conserved) plus the field comparison below, done with the fields on the
device.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import torch

NU = 0.01


def run(n, steps, prec, fields):
    from . import lb
    th0 = lb.lb_theta0()
    ctx = lb.lb_init((n, n, n), NU / th0, prec)
    try:
        lb.lb_set_fields(ctx, fields["rho"], fields["u"], fields["theta"])
        c0 = lb.lb_conserved(ctx)
        if prec != "f64":
            lb.lb_tune(ctx, reps=2)
        t0 = time.perf_counter()
        lb.lb_step(ctx, steps)
        lb.lb_sync(ctx)
        el = time.perf_counter() - t0
        c1 = lb.lb_conserved(ctx)
        rho = torch.empty((2, n, n, n), dtype=torch.float64, device="cuda")
        th = torch.empty_like(rho)
        lb.lb_get_moments(ctx, rho, None, th)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    return rho, th, c0, c1, el


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--steps", type=int, default=500)
    a = p.parse_args(argv)
    from . import lb
    from . import workloads as wl
    torch.cuda.set_device(0)
    th0 = lb.lb_theta0()
    fields = wl.thermoacoustic_pulse(a.n, th0, device="cuda")
    out = {"n": a.n, "steps": a.steps, "workload": "thermoacoustic pulse (1e-2, sigma 8) + theta Fourier box (1e-3)"}
    ref_rho, ref_th, c0, c1, el = run(a.n, a.steps, "f64", fields)
    out["f64"] = {"seconds": el, "mass_drift": (c1[0] - c0[0]) / c0[0], "energy_drift": (c1[4] - c0[4]) / c0[4]}
    dr = ref_rho - 1.0
    dt = ref_th - th0
    nr, nt = float(torch.linalg.vector_norm(dr)), float(torch.linalg.vector_norm(dt))
    for prec in ("f32", "f16", "bf16"):
        rho, th, c0, c1, el = run(a.n, a.steps, prec, fields)
        er = float(torch.linalg.vector_norm(rho - ref_rho)) / nr
        et = float(torch.linalg.vector_norm(th - ref_th)) / nt
        out[prec] = {"rel_l2_rho_fluct": er, "rel_l2_theta_fluct": et,
                     "max_abs_rho_err": float((rho - ref_rho).abs().max()),
                     "mass_drift": (c1[0] - c0[0]) / c0[0], "energy_drift": (c1[4] - c0[4]) / c0[4],
                     "seconds": el}
        del rho, th
        torch.cuda.empty_cache()
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
