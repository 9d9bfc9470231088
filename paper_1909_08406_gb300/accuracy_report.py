"""Accuracy of the reduced-precision storage modes against FP64 on the GPU.

Runs the thermoacoustic case (Gaussian density pulse 1e-2, sigma 8 cells, plus
a 16^3-Fourier-box temperature perturbation of max 1e-3, nu = 0.01) on an n^3
grid for `steps` steps in FP64 (the GPU FP64 mode, itself matched to the CPU
oracle to 1e-12 on small grids), FP32, FP32 + FP16 storage, FP32 + BF16
storage rounded to nearest and FP32 + BF16 storage rounded stochastically
("bf16sr", lb_set_stochastic_rounding), and reports for each the relative L2 error of the density
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
SR_SEED = 20191909


def run(n, steps, prec, fields, kernel=None):
    """Sets the fields, steps and returns (rho, theta, conserved before, conserved after, seconds).
    `kernel` fixes the step kernel (an LB_KERNEL_* id); None lets the autotuner pick."""
    from . import lb
    th0 = lb.lb_theta0()
    ctx = lb.lb_init((n, n, n), NU / th0, "bf16" if prec == "bf16sr" else prec)
    try:
        lb.lb_set_fields(ctx, fields["rho"], fields["u"], fields["theta"])
        if prec == "bf16sr":
            lb.lb_set_stochastic_rounding(ctx, SR_SEED)
        c0 = lb.lb_conserved(ctx)
        if kernel is not None:
            lb.lb_set_step_kernel(ctx, kernel)
        elif prec != "f64":
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


def compare(n, steps, precs, fields, kernels=None):
    """Error of each storage precision in `precs` against the GPU FP64 mode after `steps` steps
    of the same initial fields.  `kernels` maps a precision to a fixed step kernel id."""
    from . import lb
    th0 = lb.lb_theta0()
    ref_rho, ref_th, c0, c1, el = run(n, steps, "f64", fields)
    nr = float(torch.linalg.vector_norm(ref_rho - 1.0))
    nt = float(torch.linalg.vector_norm(ref_th - th0))
    out = {"f64": {"seconds": el, "mass_drift": (c1[0] - c0[0]) / c0[0], "energy_drift": (c1[4] - c0[4]) / c0[4],
                   "l2_rho_fluct": nr, "l2_theta_fluct": nt}}
    for prec in precs:
        rho, th, c0, c1, el = run(n, steps, prec, fields, (kernels or {}).get(prec))
        out[prec] = {"rel_l2_rho_fluct": float(torch.linalg.vector_norm(rho - ref_rho)) / nr,
                     "rel_l2_theta_fluct": float(torch.linalg.vector_norm(th - ref_th)) / nt,
                     "max_abs_rho_err": float((rho - ref_rho).abs().max()),
                     "mass_drift": (c1[0] - c0[0]) / c0[0], "energy_drift": (c1[4] - c0[4]) / c0[4],
                     "seconds": el}
        del rho, th
        torch.cuda.empty_cache()
    del ref_rho, ref_th
    torch.cuda.empty_cache()
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--steps", type=int, default=500)
    a = p.parse_args(argv)
    from . import lb
    from . import workloads as wl
    torch.cuda.set_device(0)
    fields = wl.thermoacoustic_pulse(a.n, lb.lb_theta0(), device="cuda")
    out = {"n": a.n, "steps": a.steps, "workload": "thermoacoustic pulse (1e-2, sigma 8) + theta Fourier box (1e-3)"}
    out.update(compare(a.n, a.steps, ("f32", "f16", "bf16", "bf16sr"), fields))
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
