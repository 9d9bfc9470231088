"""The isothermal nonideal fluid on the GPU (lb_set_nonideal) against the
oracle's ``oracle/nonideal.py`` and against Maxwell's construction.

Tolerances: FP64 1e-12 relative over every population after 5 steps (only
summation order differs, in the force's stencil sums as in the collision);
FP32 arithmetic 2e-6 (deviations of order 1 across the interface, so the
FP32 rounding of h is about 1e-7 per step, plus the FP32 collision)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import lib_to_oracle_perm, to_oracle_order
from oracle import nonideal as ni
from paper_1909_08406_gb300 import lb

pytestmark = pytest.mark.gpu

TH0 = lb.lb_theta0()
KAPPA = 0.05


def _slab(shape, width=3.0, noise=0.0, seed=5):
    """Liquid slab in vapour along x at the Maxwell densities of theta/theta_c = 0.9."""
    nx, ny, nz = shape
    e = ni.VdW(0.9)
    g, l = e.maxwell()
    x = np.array([[[[ix + 0.5 * s for ix in range(nx)] for _ in range(ny)] for _ in range(nz)] for s in (0, 1)])
    rho = g + (l - g) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
    if noise:
        rho = rho * (1 + noise * np.random.default_rng(seed).standard_normal(rho.shape))
    return e, rho


def _gpu(shape, prec, e, rho, steps, tau=0.5):
    n = rho.size
    ctx = lb.lb_init(shape, tau, prec)
    try:
        lb.lb_set_fields(ctx, torch.from_numpy(rho.ravel()).cuda(), torch.zeros(3 * n, dtype=torch.float64).cuda(),
                         torch.full((n,), TH0, dtype=torch.float64).cuda())
        lb.lb_set_nonideal(ctx, e.a, e.b, KAPPA, 0.5)
        c0 = lb.lb_conserved(ctx)
        lb.lb_step(ctx, steps)
        c1 = lb.lb_conserved(ctx)
        nx, ny, nz = shape
        f = np.empty((2, 41, nz, ny, nx))
        lb.lb_get_populations(ctx, f)
    finally:
        lb.lb_destroy(ctx)
    return f, c0, c1


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_nonideal_step_matches_oracle(prec, tol):
    shape, steps = (12, 4, 6), 5
    e, rho = _slab(shape, noise=0.02)
    got, _, _ = _gpu(shape, prec, e, rho, steps)
    f0 = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    ref = ni.step(f0, 0.5, e, KAPPA, nsteps=steps)
    rel = np.abs(to_oracle_order(got, lib_to_oracle_perm()) - ref) / np.abs(ref)
    assert rel.max() <= tol, rel.max()


def test_nonideal_conserves_mass_and_global_momentum():
    shape = (16, 4, 4)
    e, rho = _slab(shape, noise=0.02, seed=9)
    _, c0, c1 = _gpu(shape, "f64", e, rho, 50)
    nodes = 2 * 16 * 4 * 4
    assert abs(c1[0] - c0[0]) <= 1e-12 * nodes
    assert np.abs(c1[1:4] - c0[1:4]).max() <= 1e-12 * nodes  # the force sums to zero over the grid


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_flat_interface_reaches_maxwell_densities_on_gpu(prec):
    """The oracle's interface test (64 cells, 1500 steps) on the GPU: vapour within 2% and liquid
    within 0.3% of Maxwell's construction, as the oracle reaches them."""
    shape = (64, 1, 1)
    e, rho = _slab(shape)
    f, _, _ = _gpu(shape, prec, e, rho, 1500)
    r = f.sum(axis=1)
    g, l = e.maxwell()
    gas, liquid = r[0, 0, 0, 0], r[0, 0, 0, 32]
    assert abs(gas / g - 1) <= 0.02 and abs(liquid / l - 1) <= 0.003, (gas, liquid, g, l)


def test_nonideal_arguments():
    ctx = lb.lb_init((8, 4, 4), 0.5, "f32", flags=lb.LB_FLAG_ENTROPIC)
    try:
        with pytest.raises(lb.LbError):
            lb.lb_set_nonideal(ctx, 0.3, 0.3, 0.05, 0.5)
    finally:
        lb.lb_destroy(ctx)
    ctx = lb.lb_init((8, 4, 4), 0.5, "f32")
    try:
        with pytest.raises(lb.LbError):
            lb.lb_set_nonideal(ctx, 0.3, 0.3, 0.05, 1.5)
        with pytest.raises(lb.LbError):
            lb.lb_set_nonideal(ctx, 0.3, -1.0, 0.05, 0.5)
        lb.lb_set_nonideal(ctx, 0.3, 0.3, 0.05, 0.5)
        with pytest.raises(lb.LbError) as ex:
            lb.lb_set_walls(ctx, (0.0, 0.0, TH0), (0.0, 0.0, TH0))
        assert ex.value.status == -7
        lb.lb_set_nonideal(ctx)
    finally:
        lb.lb_destroy(ctx)
