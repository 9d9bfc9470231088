"""The exact entropic equilibrium mode (LB_FLAG_ENTROPIC) on the GPU against the
oracle's Newton solution of Eqs. (discreteentropiceq) and
(fivelagrangemultipliersystem).

Bounds: FP64 1e-12 (both sides converge Newton to round-off; only summation
order differs); FP32 arithmetic the same bounds as the series equilibrium
(one storage rounding per step plus FP32 evaluation in deviation form,
sqrt(steps) growth, factor 4 margin), at amplitude 0.02, where an FP32 Newton
solution is within ~5e-8 of the exact one (5% amplitude: ~1e-7)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import to_oracle_order
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-7, "f16": 1e-4, "bf16": 8e-4}


@pytest.fixture(scope="module")
def perm():
    from helpers import lib_to_oracle_perm
    return lib_to_oracle_perm()


def _np(fl):
    return fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()


def _gpu(shape, prec, fl, steps, tau=0.3):
    ctx = lb.lb_init(shape, tau, prec, flags=lb.LB_FLAG_ENTROPIC)
    try:
        assert lb.lb_step_variant(ctx) == lb.LB_KERNEL_DIRECT1
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_step(ctx, steps)
        nx, ny, nz = shape
        f = np.empty((2, 41, nz, ny, nx))
        lb.lb_get_populations(ctx, f)
        c = lb.lb_conserved(ctx)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    return f, c


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(133, 5, 3), (16, 4, 6)])
def test_entropic_step_parity(prec, shape, perm):
    amp = 0.05 if prec == "f64" else 0.02
    fl = wl.random_fields(*shape, oracle.theta0(), seed=31, du=amp, drho=amp, dtheta=amp)
    steps = 10
    got, _ = _gpu(shape, prec, fl, steps)
    ref = oracle.step(oracle.init_fields(*_np(fl), project="entropic"), 0.3, steps, project="entropic")
    rel = np.abs(to_oracle_order(got, perm) - ref) / np.abs(ref)
    assert rel.max() <= TOL[prec], rel.max()


def test_entropic_init_has_the_given_moments():
    """f^eq of the exact entropic equilibrium reproduces rho, u and theta to round-off, even at
    large amplitude (|u| = 0.3, theta = 1.3 theta0), where the series equilibrium does not
    reproduce the stress and heat flux of the exact minimiser."""
    shape = (8, 4, 4)
    fl = wl.random_fields(*shape, oracle.theta0(), seed=32, du=0.3, drho=0.2, dtheta=0.3)
    ctx = lb.lb_init(shape, 0.3, "f64", flags=lb.LB_FLAG_ENTROPIC)
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        rho = torch.empty_like(fl["rho"]).cuda()
        u = torch.empty_like(fl["u"]).cuda()
        th = torch.empty_like(fl["theta"]).cuda()
        lb.lb_get_moments(ctx, rho, u, th)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    assert torch.allclose(rho.cpu(), fl["rho"], rtol=0, atol=1e-13)
    assert torch.allclose(u.cpu(), fl["u"], rtol=0, atol=1e-13)
    assert torch.allclose(th.cpu(), fl["theta"], rtol=0, atol=1e-13)


def test_entropic_large_amplitude_conserves():
    shape = (12, 6, 4)
    fl = wl.random_fields(*shape, oracle.theta0(), seed=33, du=0.25, drho=0.2, dtheta=0.25)
    ctx = lb.lb_init(shape, 0.7, "f64", flags=lb.LB_FLAG_ENTROPIC)
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        c0 = np.array(lb.lb_conserved(ctx))
        lb.lb_step(ctx, 20)
        c1 = np.array(lb.lb_conserved(ctx))
    finally:
        lb.lb_destroy(ctx)
    assert np.abs(c1 - c0).max() <= 1e-12 * np.abs(c0).max(), (c0, c1)


def test_newton_failure_is_reported():
    """A temperature far outside the lattice's range (theta = 40 theta0) defeats Newton from the
    linearised start within the fixed iteration count: the step reports LB_ERR_UNSTABLE."""
    shape = (4, 4, 4)
    fl = wl.random_fields(*shape, oracle.theta0(), seed=34, du=0.0, drho=0.0, dtheta=0.0)
    fl["theta"][0, 1, 2, 3] = 40 * oracle.theta0()
    ctx = lb.lb_init(shape, 0.3, "f32", flags=lb.LB_FLAG_ENTROPIC)
    try:
        with pytest.raises(lb.LbError) as e:
            lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
            lb.lb_step(ctx, 1)
            lb.lb_sync(ctx)
        assert e.value.status == -5
    finally:
        lb.lb_destroy(ctx)


def test_entropic_flag_rules():
    with pytest.raises(lb.LbError):
        lb.lb_init((4, 4, 4), 0.3, "f32", flags=lb.LB_FLAG_ENTROPIC | lb.LB_FLAG_PAPER_LITERAL)
