"""Kinetic walls normal to z on the GPU (lb_set_walls) against the oracle's
or_step_walls, element by element, and the Couette viscous-heating profile of
Eq. (eckert).

Tolerance (relative, over every population, 20 steps of random fields at
amplitude 0.03 between a warmer and a cooler moving wall): FP64 1e-12 (only
summation order differs); otherwise one rounding of each stored deviation
h = f/w - 1 per step, |dh| <= eps_store |h|, growing like sqrt(steps), at this
state's largest deviation h_max (about 0.2-0.46 here), plus 2e-7 for the FP32
evaluation: eps_store h_max sqrt(steps) + 2e-7.  Every step kernel runs the
bulk of the grid, so the wall pass is checked behind each of them."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import lib_to_oracle_perm, to_oracle_order
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

EPS_STORE = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
TH0 = lb.lb_theta0()
BOTTOM = (0.02, -0.01, TH0 * 1.01)
TOP = (-0.03, 0.0, TH0 * 0.98)


@pytest.fixture(scope="module")
def perm():
    return lib_to_oracle_perm()


def _fields(shape, seed=11):
    return wl.random_fields(*shape, TH0, seed=seed, du=0.03, drho=0.03, dtheta=0.03)


def _gpu(shape, prec, fl, steps, kernel=lb.LB_KERNEL_AUTO, flags=0, tau=0.35):
    ctx = lb.lb_init(shape, tau, prec, flags=flags)
    try:
        lb.lb_set_step_kernel(ctx, kernel)
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_set_walls(ctx, BOTTOM, TOP)
        lb.lb_step(ctx, steps)
        nx, ny, nz = shape
        f = np.empty((2, 41, nz, ny, nx))
        lb.lb_get_populations(ctx, f)
        rho_w = lb.lb_wall_density(ctx)
        used = lb.lb_step_variant(ctx)
    finally:
        lb.lb_destroy(ctx)
    return f, rho_w, used


def _oracle(fl, steps, project=True, tau=0.35):
    f0 = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy(), project=project)
    return oracle.step_walls(f0, tau, steps, BOTTOM, TOP, project=project, wall_rho=True)


CASES = [("f64", (12, 6, 8), lb.LB_KERNEL_DIRECT1), ("f64", (7, 5, 4), lb.LB_KERNEL_DIRECT1),
         ("f32", (12, 6, 8), lb.LB_KERNEL_DIRECT1), ("f32", (12, 6, 8), lb.LB_KERNEL_DIRECT2),
         ("f32", (7, 5, 4), lb.LB_KERNEL_AUTO), ("f32", (128, 2, 6), lb.LB_KERNEL_STAGED),
         ("f32", (128, 2, 6), lb.LB_KERNEL_WARPSPEC),
         ("f16", (12, 6, 8), lb.LB_KERNEL_DIRECT2XL), ("f16", (12, 6, 8), lb.LB_KERNEL_DIRECT2X),
         ("f16", (7, 5, 4), lb.LB_KERNEL_DIRECT1), ("bf16", (12, 6, 8), lb.LB_KERNEL_DIRECT2XL),
         ("bf16", (262, 2, 5), lb.LB_KERNEL_AUTO)]


@pytest.mark.parametrize("prec,shape,kernel", CASES)
def test_walls_match_oracle(prec, shape, kernel, perm):
    steps = 20
    fl = _fields(shape)
    got, rho_w, used = _gpu(shape, prec, fl, steps, kernel)
    ref, ref_rho = _oracle(fl, steps)
    w = oracle.velocities()[1][None, :, None, None, None]
    f0 = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
    h_max = max(np.abs(ref / w - 1).max(), np.abs(f0 / w - 1).max())
    tol = 1e-12 if prec == "f64" else EPS_STORE[prec] * h_max * np.sqrt(steps) + 2e-7
    rel = np.abs(to_oracle_order(got, perm) - ref) / np.abs(ref)
    assert rel.max() <= tol, (prec, shape, lb.KERNEL_NAMES[used], rel.max(), tol)
    assert np.abs(np.array(rho_w) - ref_rho[-1]).max() <= tol, (rho_w, ref_rho[-1])


def test_walls_with_entropic_equilibrium_match_oracle(perm):
    shape, steps = (8, 4, 6), 10
    fl = _fields(shape, seed=13)
    got, _, _ = _gpu(shape, "f64", fl, steps, flags=lb.LB_FLAG_ENTROPIC)
    ref, _ = _oracle(fl, steps, project="entropic")
    rel = np.abs(to_oracle_order(got, perm) - ref) / np.abs(ref)
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_walls_conserve_mass(prec, tol):
    shape = (16, 8, 12)
    fl = _fields(shape, seed=17)
    ctx = lb.lb_init(shape, 0.35, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        c0 = lb.lb_conserved(ctx)
        lb.lb_set_walls(ctx, BOTTOM, TOP)
        lb.lb_step(ctx, 100)
        c1 = lb.lb_conserved(ctx)
    finally:
        lb.lb_destroy(ctx)
    nodes = 2 * 16 * 8 * 12
    assert abs(c1[0] - c0[0]) <= tol * nodes, (c0[0], c1[0])


def test_rest_gas_between_rest_walls_stays_at_rest():
    shape = (8, 4, 6)
    ctx = lb.lb_init(shape, 0.3, "f32")
    try:
        n = 2 * 8 * 4 * 6
        rho = torch.ones(n, dtype=torch.float64, device="cuda")
        u = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
        th = torch.full((n,), TH0, dtype=torch.float64, device="cuda")
        lb.lb_set_fields(ctx, rho, u, th)
        lb.lb_set_walls(ctx, (0.0, 0.0, TH0), (0.0, 0.0, TH0))
        before = np.empty((2, 41, 6, 4, 8))
        lb.lb_get_populations(ctx, before)
        lb.lb_step(ctx, 10)
        after = np.empty_like(before)
        lb.lb_get_populations(ctx, after)
        # every absorbed population comes back as the same rest equilibrium (to the rounding of
        # the FP64 equilibrium constants)
        assert np.abs(after - before).max() <= 1e-13 * before.max()
        rw = lb.lb_wall_density(ctx)
        assert rw.shape == (2, 4, 8) and np.abs(rw - 1.0).max() <= 1e-14, rw
    finally:
        lb.lb_destroy(ctx)


def _couette_gpu(H, ec, prec, nu=0.05, u0=0.02, n=4):
    dT = u0 * u0 / (2.5 * ec)
    ctx = lb.lb_init((n, n, H), nu / TH0, prec)
    try:
        nodes = 2 * n * n * H
        lb.lb_set_fields(ctx, torch.ones(nodes, dtype=torch.float64, device="cuda"),
                         torch.zeros(3 * nodes, dtype=torch.float64, device="cuda"),
                         torch.full((nodes,), TH0, dtype=torch.float64, device="cuda"))
        lb.lb_set_walls(ctx, (0.0, 0.0, TH0 - dT / 2), (u0, 0.0, TH0 + dT / 2))
        lb.lb_step(ctx, int(3 * H * H / nu))
        u = torch.empty((3, 2, H, n, n), dtype=torch.float64, device="cuda")
        th = torch.empty((2, H, n, n), dtype=torch.float64, device="cuda")
        lb.lb_get_moments(ctx, None, u, th)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    th = th.mean(dim=(2, 3)).cpu().numpy()
    ux = u[0].mean(dim=(2, 3)).cpu().numpy()
    y = np.array([[(2 * z + s) / 2.0 + 0.25 for z in range(H)] for s in range(2)]) / H
    o = np.argsort(y.ravel())
    y = y.ravel()[o]
    tn = ((th - (TH0 - dT / 2)) / dT).ravel()[o]
    un = (ux / u0).ravel()[o]
    return y, tn, un, y + ec / 2 * y * (1 - y)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_couette_viscous_heating_on_gpu(prec):
    """The steady profile of Eq. (eckert) at H = 16, Ec = 2, as the oracle reaches it (max
    error 0.037), and agreement with the oracle's own steady profile."""
    y, tn, un, ex = _couette_gpu(16, 2.0, prec)
    assert np.abs(tn - ex).max() <= 0.04, np.abs(tn - ex).max()
    assert np.abs(un - y).max() <= 0.01, np.abs(un - y).max()
    dT = 0.02 ** 2 / 5.0
    f = oracle.init_fields(np.ones((2, 16, 1, 1)), np.zeros((3, 2, 16, 1, 1)), np.full((2, 16, 1, 1), TH0))
    f = oracle.step_walls(f, 0.05 / TH0, int(3 * 16 * 16 / 0.05), (0.0, 0.0, TH0 - dT / 2), (0.02, 0.0, TH0 + dT / 2))
    _, _, th = oracle.get_moments(f)
    ref = ((th.reshape(2, 16) - (TH0 - dT / 2)) / dT).ravel()
    o = np.argsort(np.array([[(2 * z + s) for z in range(16)] for s in range(2)]).ravel())
    # FP32: the temperature differences are 8e-5 of theta0, so FP32 rounding of h (2^-24 of
    # order-1 sums) shows as ~1e-3 of dT
    assert np.abs(tn - ref[o]).max() <= (1e-8 if prec == "f64" else 5e-3), np.abs(tn - ref[o]).max()


def test_wall_arguments_and_batch_refusal():
    ctx = lb.lb_init((4, 4, 3), 0.3, "f32")
    try:
        with pytest.raises(lb.LbError) as e:
            lb.lb_set_walls(ctx, (0.0, 0.0, TH0), (0.0, 0.0, TH0))  # nz < 4
        assert e.value.status == -1
        with pytest.raises(lb.LbError) as e:
            lb.lb_wall_density(ctx)
        assert e.value.status == -7
    finally:
        lb.lb_destroy(ctx)
    ctx = lb.lb_init((4, 4, 4), 0.3, "f32")
    try:
        with pytest.raises(lb.LbError):
            lb.lb_set_walls(ctx, (0.0, 0.0, -1.0), (0.0, 0.0, TH0))
        L = lb.lib()
        b = (ctypes.c_double * 4)(0.0, 0.0, 0.01, TH0)  # moving along z
        assert L.lb_set_walls(ctx, 1, ctypes.cast(b, ctypes.c_void_p), ctypes.cast(b, ctypes.c_void_p)) == -1
    finally:
        lb.lb_destroy(ctx)
    b = lb.lb_batch_init([(4, 4, 4), (4, 4, 6)], [0.3, 0.4], "f32")
    try:
        lb.lb_set_walls(lb.lb_batch_sim(b, 1), (0.0, 0.0, TH0), (0.0, 0.0, TH0))
        with pytest.raises(lb.LbError) as e:
            lb.lb_batch_step(b, 1)
        assert e.value.status == -7
    finally:
        lb.lb_batch_destroy(b)


def test_walls_off_restores_periodic_update(perm):
    shape = (8, 4, 6)
    fl = _fields(shape, seed=19)
    ctx = lb.lb_init(shape, 0.35, "f64")
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_set_walls(ctx, BOTTOM, TOP)
        lb.lb_set_walls(ctx)
        lb.lb_step(ctx, 5)
        f = np.empty((2, 41, 6, 4, 8))
        lb.lb_get_populations(ctx, f)
    finally:
        lb.lb_destroy(ctx)
    ref = oracle.step(oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()), 0.35, 5)
    assert np.abs(to_oracle_order(f, perm) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_checkpoint_restart_with_walls_is_bitwise(prec):
    """The wall columns' densities are summed from the stored state in a fixed order every step,
    so a restarted run repeats the uninterrupted one bit for bit."""
    shape = (12, 6, 8)
    fl = _fields(shape, seed=23)
    ctx = lb.lb_init(shape, 0.35, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_set_walls(ctx, BOTTOM, TOP)
        lb.lb_step(ctx, 4)
        saved = torch.empty(lb.lb_state_bytes(ctx), dtype=torch.uint8, device="cuda")
        lb.lb_get_state(ctx, saved)
        lb.lb_step(ctx, 5)
        a = torch.empty_like(saved)
        lb.lb_get_state(ctx, a)
        rho_a = lb.lb_wall_density(ctx)
    finally:
        lb.lb_destroy(ctx)
    ctx = lb.lb_init(shape, 0.35, prec)
    try:
        lb.lb_set_state(ctx, saved)
        lb.lb_set_walls(ctx, BOTTOM, TOP)
        lb.lb_step(ctx, 5)
        b = torch.empty_like(saved)
        lb.lb_get_state(ctx, b)
        rho_b = lb.lb_wall_density(ctx)
    finally:
        lb.lb_destroy(ctx)
    assert torch.equal(a, b)
    assert np.array_equal(rho_a, rho_b)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_thermoacoustic_column_on_gpu_follows_nsf(prec):
    """The thermoacoustic column of the oracle's test (H = 64, nu = 0.05, top wall heated by
    0.01 theta0) on the GPU, against the linearised NSF solution, with the oracle's bounds."""
    from oracle import nsf1d
    H, nu, dT, n = 64, 0.05, 0.01 * TH0, 2
    nodes = 2 * n * n * H
    ctx = lb.lb_init((n, n, H), nu / TH0, prec)
    out, t = {}, 0
    try:
        lb.lb_set_fields(ctx, torch.ones(nodes, dtype=torch.float64, device="cuda"),
                         torch.zeros(3 * nodes, dtype=torch.float64, device="cuda"),
                         torch.full((nodes,), TH0, dtype=torch.float64, device="cuda"))
        lb.lb_set_walls(ctx, (0.0, 0.0, TH0), (0.0, 0.0, TH0 + dT))
        for tt in (90, 400):
            lb.lb_step(ctx, tt - t)
            t = tt
            th = torch.empty((2, H, n, n), dtype=torch.float64, device="cuda")
            lb.lb_get_moments(ctx, None, None, th)
            lb.lb_sync(ctx)
            out[tt] = th.mean(dim=(2, 3)).cpu().numpy().ravel() - TH0
    finally:
        lb.lb_destroy(ctx)
    y = np.array([[(2 * z + s) / 2.0 + 0.25 for z in range(H)] for s in range(2)]).ravel()
    ref = nsf1d.column(float(H), nu, dT, TH0, [90, 400])
    err = {tt: np.abs(out[tt] - np.interp(y, ref[tt][0], ref[tt][2])).max() / dT for tt in (90, 400)}
    assert err[90] <= 0.09 and err[400] <= 0.04, err
    assert err[90] / err[400] >= 1.8, err


def test_walls_with_varying_columns_match_oracle(perm):
    """Every wall column with its own velocity and temperature (seeded), FP64 and FP32."""
    shape, steps = (10, 6, 6), 12
    nx, ny, _ = shape
    rng = np.random.default_rng(29)
    cols = [(0.02 * rng.standard_normal((ny, nx)), 0.02 * rng.standard_normal((ny, nx)),
             TH0 * (1 + 0.02 * rng.standard_normal((ny, nx)))) for _ in range(2)]
    fl = _fields(shape, seed=31)
    f0 = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
    ref, ref_rho = oracle.step_walls(f0, 0.35, steps, cols[0], cols[1], wall_rho=True)
    w = oracle.velocities()[1][None, :, None, None, None]
    h_max = max(np.abs(ref / w - 1).max(), np.abs(f0 / w - 1).max())
    for prec in ("f64", "f32"):
        ctx = lb.lb_init(shape, 0.35, prec)
        try:
            lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
            lb.lb_set_walls(ctx, cols[0], cols[1])
            lb.lb_step(ctx, steps)
            got = np.empty((2, 41, 6, 6, 10))
            lb.lb_get_populations(ctx, got)
            rho_w = lb.lb_wall_density(ctx)
        finally:
            lb.lb_destroy(ctx)
        tol = 1e-12 if prec == "f64" else EPS_STORE[prec] * h_max * np.sqrt(steps) + 2e-7
        rel = np.abs(to_oracle_order(got, perm) - ref) / np.abs(ref)
        assert rel.max() <= tol, (prec, rel.max(), tol)
        assert np.abs(rho_w - ref_rho[-1]).max() <= tol, prec


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_wall_with_varying_temperature_gives_laplace_field_on_gpu(prec):
    """theta0 (1 + a cos kx) below, theta0 above: the steady field follows
    a cos(kx) sinh(k (H - y)) / sinh(kH) within the oracle's bound (0.089 of a measured there)."""
    nx, H, nu, a = 32, 16, 0.1, 0.01
    k = 2 * np.pi / nx
    tb = (TH0 * (1 + a * np.cos(k * (np.arange(nx) + 0.25))))[None, :].repeat(2, 0)
    n = 2 * nx * 2 * H
    ctx = lb.lb_init((nx, 2, H), nu / TH0, prec)
    try:
        lb.lb_set_fields(ctx, torch.ones(n, dtype=torch.float64, device="cuda"),
                         torch.zeros(3 * n, dtype=torch.float64, device="cuda"),
                         torch.full((n,), TH0, dtype=torch.float64, device="cuda"))
        lb.lb_set_walls(ctx, (0.0, 0.0, tb), (0.0, 0.0, TH0))
        lb.lb_step(ctx, int(4 * H * H / (5.0 / 3.0 * nu)))
        th = torch.empty((2, H, 2, nx), dtype=torch.float64, device="cuda")
        lb.lb_get_moments(ctx, None, None, th)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    th = th.cpu().numpy()
    err = 0.0
    for s in (0, 1):
        X = np.arange(nx) + 0.5 * s
        for z in range(H):
            Y = z + 0.5 * s + 0.25
            exact = a * np.cos(k * X) * np.sinh(k * (H - Y)) / np.sinh(k * H)
            err = max(err, np.abs(th[s, z] / TH0 - 1 - exact[None, :]).max())
    assert err / a <= 0.10, err / a


def _cavity_gpu(L, prec, nu=0.1, dT=0.01):
    """The cavity heated at the top, L = H, side walls by images (see the oracle's test); the
    largest deviation from the paper's series over the paper's sections, in units of dT."""
    from oracle.conduction import cavity_series
    H, nx, ny = L, 2 * L, 2
    top = TH0 * (1 + dT * np.sign(np.sin(np.pi * (np.arange(nx) - 0.25) / L)))[None, :].repeat(ny, 0)
    n = 2 * nx * ny * H
    ctx = lb.lb_init((nx, ny, H), nu / TH0, prec)
    try:
        lb.lb_set_fields(ctx, torch.ones(n, dtype=torch.float64, device="cuda"),
                         torch.zeros(3 * n, dtype=torch.float64, device="cuda"),
                         torch.full((n,), TH0, dtype=torch.float64, device="cuda"))
        lb.lb_set_walls(ctx, (0.0, 0.0, TH0), (0.0, 0.0, top))
        lb.lb_step(ctx, int(4 * H * H / (5.0 / 3.0 * nu)))
        th = torch.empty((2, H, ny, nx), dtype=torch.float64, device="cuda")
        lb.lb_get_moments(ctx, None, None, th)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    T = th[:, :, 0, :].cpu().numpy() / TH0 - 1
    X = np.array([[np.arange(nx) + 0.5 * s - 0.25 for _ in range(H)] for s in (0, 1)])
    Y = np.array([[np.full(nx, z + 0.5 * s + 0.25) for z in range(H)] for s in (0, 1)])
    err = np.abs(T - dT * cavity_series(X, Y, L, H)) / dT
    xl, yh = X / L, Y / H
    worst = 0.0
    for x0 in (0.1, 0.2, 0.5):
        worst = max(worst, err[(np.abs(xl - x0) <= 0.5 / L + 1e-9) & (yh <= 0.8)].max())
    for y0 in (0.25, 0.5, 0.75):
        worst = max(worst, err[(np.abs(yh - y0) <= 0.5 / H + 1e-9) & (xl > 0.05) & (xl < 0.95)].max())
    return worst


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cavity_heated_at_the_top_converges_to_the_series(prec):
    """L = H = 16 as the oracle's test (0.043 dT there), and 32: the kinetic wall's temperature
    jump shrinks at first order in 1/L."""
    e16, e32 = _cavity_gpu(16, prec), _cavity_gpu(32, prec)
    assert e16 <= 0.045 and e32 <= 0.025, (e16, e32)
    assert e16 / e32 >= 1.7, (e16, e32)
