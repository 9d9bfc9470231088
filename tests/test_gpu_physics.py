"""The 3D acoustic spherical pulse (Sec. VII) on the GPU, in every storage
precision, against the exact solution (``oracle/acoustics.py``, itself pinned
in two independent forms).

An isentropic pulse rho' = 1e-3 exp(-alpha r^2) of half-width b cells runs for
t = 5 b steps at nu = 1e-3 (the front, at c_s t + 4 b < n / 2, has not met
its periodic images).  The error against the loss-free solution is the
scheme's discretisation error, second order in 1 / b (the oracle shows
relative L2 errors of 10.6% at b = 2 and 2.0% at b = 4), plus the storage
rounding: one rounding of h per step, growing like sqrt(t), i.e. about
sqrt(40) * 2^-12 = 0.15% (FP16) and sqrt(40) * 2^-9 = 1.2% (BF16) of the pulse.
Bounds: FP64/FP32 0.8% at b = 8 and an error ratio of at least 3.5 between
b = 4 and b = 8; FP16 1%; BF16 3%."""
import math

import numpy as np
import pytest
import torch

from oracle import acoustics as ac
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

EPS = 1e-3
NU = 1e-3


def _pulse_error(n, b, prec):
    th0 = lb.lb_theta0()
    t = int(round(5 * b))
    fl = wl.spherical_pulse(n, th0, b=b, eps=EPS, device="cuda")
    ctx = lb.lb_init((n, n, n), NU / th0, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
        lb.lb_step(ctx, t)
        rho = torch.empty((2, n, n, n), dtype=torch.float64, device="cuda")
        lb.lb_get_moments(ctx, rho, None, None)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    d = (rho - 1.0).cpu().numpy()
    R = wl.pulse_radius(n).numpy()
    ex = ac.pulse_dalembert(R, t, EPS, math.log(2.0) / (b * b), math.sqrt(5.0 * th0 / 3.0))
    return np.linalg.norm(d - ex) / np.linalg.norm(ex), np.abs(d - ex).max() / EPS


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spherical_pulse_converges_at_second_order(prec):
    l2a, _ = _pulse_error(64, 4.0, prec)
    l2b, mxb = _pulse_error(128, 8.0, prec)
    assert l2b <= 0.008, (l2a, l2b, mxb)
    assert l2a / l2b >= 3.5, (l2a, l2b)


@pytest.mark.parametrize("prec,bound", [("f16", 0.01), ("bf16", 0.03)])
def test_spherical_pulse_16bit_storage(prec, bound):
    l2, mx = _pulse_error(128, 8.0, prec)
    assert l2 <= bound, (l2, mx)
