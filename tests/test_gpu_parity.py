"""GPU parity: the CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (max |f_gpu - f_oracle| / f_oracle over every population):
  * streaming (tau = inf, collision is the identity): bit-exact in every
    storage type;
  * FP64: 1e-12 after 200 steps of the 32^3 standing wave, 1e-12 after 20
    steps of random fields (only summation order differs);
  * FP32 arithmetic: each step rounds h = f/w - 1 to the storage type and
    evaluates the equilibrium in FP32 in deviation form, so the error per step
    is ~ eps_store |h| + ~1e-7 |h|; the bounds below allow sqrt(steps) growth
    with a factor 4 margin for |h| <~ 0.05 (f32 2e-7, f16 1e-4, bf16 8e-4 after
    20 steps).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import STORE_EPS, TORCH_DTYPE, decode, lib_to_oracle_perm, to_lib_order, to_oracle_order
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PRECS = ["f64", "f32", "f16", "bf16"]
RANDOM_FIELD_TOL = {"f64": 1e-12, "f32": 2e-7, "f16": 1e-4, "bf16": 8e-4}


@pytest.fixture(scope="module")
def perm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return lib_to_oracle_perm()


@pytest.fixture(scope="module")
def w_lib():
    return lb.lb_velocity_set()[1]


def _fields_np(fl):
    return fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()


def _run_gpu(shape, tau, prec, fields, steps, flags=0, kernel=lb.LB_KERNEL_AUTO):
    ctx = lb.lb_init(shape, tau, prec, flags=flags)
    try:
        lb.lb_set_step_kernel(ctx, kernel)
        lb.lb_set_fields(ctx, fields["rho"].cuda(), fields["u"].cuda(), fields["theta"].cuda())
        lb.lb_step(ctx, steps)
        nx, ny, nz = shape
        f = np.empty((2, 41, nz, ny, nx))
        lb.lb_get_populations(ctx, f)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    return f


# Every step kernel on every shape it applies to: DIRECT2/DIRECT2R need ny even (odd ny falls back
# to DIRECT1); STAGED needs nx a multiple of 128 (nx = 128: one tile per row; 256, 384: first,
# middle and last tiles of a row) and falls back to DIRECT2/DIRECT1 elsewhere; DIRECT2X needs 16-bit
# storage and nx even (nx = 2: the x-2 and x+2 pairs coincide; 262: a ragged second block of
# pairs); FP64 always runs DIRECT1.
KERNELS = [lb.LB_KERNEL_DIRECT1, lb.LB_KERNEL_DIRECT2, lb.LB_KERNEL_DIRECT2R, lb.LB_KERNEL_STAGED,
           lb.LB_KERNEL_WARPSPEC, lb.LB_KERNEL_DIRECT2X, lb.LB_KERNEL_DIRECT2XL]
STREAM_SHAPES = [(4, 4, 4), (3, 5, 7), (1, 2, 5), (133, 4, 3), (128, 2, 3), (256, 2, 1), (384, 2, 3),
                 (2, 3, 2), (262, 2, 3)]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", STREAM_SHAPES)
def test_streaming_is_bit_exact(prec, shape, kernel, perm, w_lib):
    nx, ny, nz = shape
    rng = np.random.default_rng(100 + nx)
    h = 0.1 * rng.uniform(-1, 1, size=(2, 41, nz, ny, nx))
    if prec == "f64":
        stored = np.asarray(w_lib)[None, :, None, None, None] * (1 + h)
    else:
        stored = h
    raw = torch.from_numpy(stored).to(TORCH_DTYPE[prec]).cuda().contiguous()
    ctx = lb.lb_init(shape, math.inf, prec)
    try:
        lb.lb_set_step_kernel(ctx, kernel)
        lb.lb_set_state(ctx, raw)
        lb.lb_step(ctx, 1)
        out = torch.empty_like(raw)
        lb.lb_get_state(ctx, out)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    exact_in = raw.cpu().to(torch.float64).numpy()  # stored values are exact in float64
    ref = oracle.stream(to_oracle_order(exact_in, perm))
    got = to_oracle_order(out.cpu().to(torch.float64).numpy(), perm)
    assert np.array_equal(got, ref)


def test_config1_f64_standing_wave_200_steps(perm):
    """32^3, FP64, nu = 0.01, rho = 1 + 1e-3 sin(2 pi x / 32): every population after 200 steps."""
    N = 32
    th0 = lb.lb_theta0()
    tau = 0.01 / th0
    fl = wl.standing_wave(N, N, N, th0, amplitude=1e-3)
    got = to_oracle_order(_run_gpu((N, N, N), tau, "f64", fl, 200), perm)
    ref = oracle.step(oracle.init_fields(*_fields_np(fl)), tau, 200)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("project", [True, False])
@pytest.mark.parametrize("shape", [(133, 5, 3), (133, 4, 3), (384, 2, 3), (128, 4, 3), (262, 5, 3)])
def test_random_fields_parity(prec, project, shape, kernel, perm):
    # (133, *, 3): two x-blocks with a ragged tail, odd and even ny; (384, 2, 3): three tiles
    # per row for the staged kernel; (128, 4, 3): one tile per row; (262, 5, 3): x pairs with a
    # ragged second block
    th0 = lb.lb_theta0()
    amp = 0.05 if prec in ("f64", "f32") else 0.02
    fl = wl.random_fields(*shape, th0, seed=7, du=amp, drho=amp, dtheta=amp)
    tau = 0.3
    steps = 20
    flags = 0 if project else lb.LB_FLAG_PAPER_LITERAL
    got = to_oracle_order(_run_gpu(shape, tau, prec, fl, steps, flags=flags, kernel=kernel), perm)
    ref = oracle.step(oracle.init_fields(*_fields_np(fl), project=project), tau, steps, project=project)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() <= RANDOM_FIELD_TOL[prec], rel.max()


@pytest.mark.parametrize("prec", PRECS)
def test_init_from_fields(prec, perm):
    shape = (37, 4, 3)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=8, du=0.05, drho=0.05, dtheta=0.05)
    got = to_oracle_order(_run_gpu(shape, 0.5, prec, fl, 0), perm)
    ref = oracle.init_fields(*_fields_np(fl))
    h_ref_max = np.max(np.abs(ref / oracle.velocities()[1][None, :, None, None, None] - 1))
    tol = {"f64": 1e-14}.get(prec, STORE_EPS[prec] * h_ref_max + 2e-7 * h_ref_max)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() <= tol, (rel.max(), tol)


@pytest.mark.parametrize("on_device", [False, True])
def test_moments_and_conserved_f64(on_device, perm):
    shape = (9, 7, 5)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=9, du=0.05, drho=0.05, dtheta=0.05)
    f_or = oracle.step(oracle.init_fields(*_fields_np(fl)), 0.4, 3)
    nx, ny, nz = shape
    ctx = lb.lb_init(shape, 0.4, "f64")
    try:
        f_lib = to_lib_order(f_or, perm)
        if on_device:
            lb.lb_set_populations(ctx, torch.from_numpy(f_lib).cuda())
            rho = torch.empty((2, nz, ny, nx), dtype=torch.float64, device="cuda")
            u = torch.empty((3, 2, nz, ny, nx), dtype=torch.float64, device="cuda")
            th = torch.empty_like(rho)
            lb.lb_get_moments(ctx, rho, u, th)
            lb.lb_sync(ctx)
            rho, u, th = rho.cpu().numpy(), u.cpu().numpy(), th.cpu().numpy()
        else:
            lb.lb_set_populations(ctx, f_lib)
            rho = np.empty((2, nz, ny, nx))
            u = np.empty((3, 2, nz, ny, nx))
            th = np.empty_like(rho)
            lb.lb_get_moments(ctx, rho, u, th)
        cons = lb.lb_conserved(ctx)
    finally:
        lb.lb_destroy(ctx)
    r_or, u_or, t_or = oracle.get_moments(f_or)
    assert np.max(np.abs(rho - r_or)) < 1e-14
    assert np.max(np.abs(u - u_or)) < 1e-14
    assert np.max(np.abs(th - t_or) / t_or) < 1e-13
    c_or = oracle.conserved(f_or)
    assert cons[0] == pytest.approx(c_or[0], rel=1e-13)
    assert np.max(np.abs(cons[1:4] - c_or[1:4])) < 1e-12
    assert cons[4] == pytest.approx(c_or[4], rel=1e-13)


@pytest.mark.parametrize("prec", PRECS)
def test_checkpoint_restart_is_bitwise(prec):
    shape = (20, 6, 5)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=10, du=0.02, drho=0.02, dtheta=0.02)
    ctx = lb.lb_init(shape, 0.3, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
        lb.lb_step(ctx, 7)
        saved = np.empty(lb.lb_state_bytes(ctx), dtype=np.uint8)
        lb.lb_get_state(ctx, saved)
        lb.lb_step(ctx, 9)
        a = np.empty_like(saved)
        lb.lb_get_state(ctx, a)
        lb.lb_set_state(ctx, saved)
        lb.lb_step(ctx, 9)
        b = np.empty_like(saved)
        lb.lb_get_state(ctx, b)
    finally:
        lb.lb_destroy(ctx)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, saved)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_conservation_over_steps(prec):
    shape = (16, 12, 8)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=11, du=0.03, drho=0.03, dtheta=0.03)
    ctx = lb.lb_init(shape, 0.25, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
        c0 = lb.lb_conserved(ctx)
        lb.lb_step(ctx, 100)
        c1 = lb.lb_conserved(ctx)
    finally:
        lb.lb_destroy(ctx)
    n = 2 * 16 * 12 * 8
    tol = 1e-13 if prec == "f64" else 1e-6
    assert abs(c1[0] - c0[0]) < tol * n
    assert np.max(np.abs(c1[1:4] - c0[1:4])) < tol * n
    assert abs(c1[4] - c0[4]) < tol * c0[4]


def test_unstable_state_is_reported():
    shape = (8, 4, 4)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=12, du=0.01, drho=0.01, dtheta=0.01)
    fl["rho"][0, 1, 2, 3] = -1.0
    ctx = lb.lb_init(shape, 0.5, "f32")
    try:
        lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
        with pytest.raises(lb.LbError) as e:
            lb.lb_sync(ctx)
        assert e.value.status == -5
    finally:
        lb.lb_destroy(ctx)


def test_step_kernel_selection_and_fallbacks():
    K = lb
    cases = [((256, 2, 2), "f16", K.LB_KERNEL_STAGED, K.LB_KERNEL_STAGED),
             ((256, 2, 2), "f16", K.LB_KERNEL_AUTO, K.LB_KERNEL_DIRECT2XL),
             ((256, 2, 2), "f32", K.LB_KERNEL_AUTO, K.LB_KERNEL_DIRECT2),
             ((255, 2, 2), "bf16", K.LB_KERNEL_AUTO, K.LB_KERNEL_DIRECT2),  # odd nx
             ((256, 3, 2), "f32", K.LB_KERNEL_DIRECT2, K.LB_KERNEL_DIRECT1),   # odd ny
             ((130, 2, 2), "f32", K.LB_KERNEL_STAGED, K.LB_KERNEL_DIRECT2),    # nx not a multiple of 128
             ((256, 2, 2), "f64", K.LB_KERNEL_STAGED, K.LB_KERNEL_DIRECT1),
             ((256, 2, 2), "bf16", K.LB_KERNEL_DIRECT2R, K.LB_KERNEL_DIRECT2R),
             ((130, 3, 2), "f16", K.LB_KERNEL_DIRECT2X, K.LB_KERNEL_DIRECT2X),
             ((133, 2, 2), "bf16", K.LB_KERNEL_DIRECT2X, K.LB_KERNEL_DIRECT2),  # odd nx
             ((256, 2, 2), "f16", K.LB_KERNEL_DIRECT2XL, K.LB_KERNEL_DIRECT2XL),
             ((256, 2, 2), "f32", K.LB_KERNEL_DIRECT2X, K.LB_KERNEL_DIRECT2)]   # 32-bit storage
    for shape, prec, req, expect in cases:
        ctx = lb.lb_init(shape, 0.5, prec)
        try:
            lb.lb_set_step_kernel(ctx, req)
            assert lb.lb_step_variant(ctx) == expect, (shape, prec, req)
        finally:
            lb.lb_destroy(ctx)
    ctx = lb.lb_init((256, 2, 2), 0.5, "f16", flags=lb.LB_FLAG_STAGED)
    try:
        assert lb.lb_step_variant(ctx) == K.LB_KERNEL_STAGED
    finally:
        lb.lb_destroy(ctx)


def test_step_autotuner_keeps_state():
    shape = (256, 4, 3)
    fl = wl.random_fields(*shape, lb.lb_theta0(), seed=14, du=0.02, drho=0.02, dtheta=0.02)
    ctx = lb.lb_init(shape, 0.3, "f16")
    try:
        lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
        lb.lb_step(ctx, 2)
        a = np.empty(lb.lb_state_bytes(ctx), dtype=np.uint8)
        lb.lb_get_state(ctx, a)
        k, ms = lb.lb_tune(ctx, reps=2)
        assert k == lb.lb_step_variant(ctx) and ms > 0
        b = np.empty_like(a)
        lb.lb_get_state(ctx, b)
        assert np.array_equal(a, b)
    finally:
        lb.lb_destroy(ctx)


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_step_kernels_agree(prec):
    shape = (256, 4, 3)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=13, du=0.02, drho=0.02, dtheta=0.02)
    outs = []
    for kernel in KERNELS:
        ctx = lb.lb_init(shape, 0.3, prec)
        try:
            lb.lb_set_step_kernel(ctx, kernel)
            lb.lb_set_fields(ctx, fl["rho"], fl["u"], fl["theta"])
            lb.lb_step(ctx, 10)
            f = np.empty((2, 41, 3, 4, 256))
            lb.lb_get_populations(ctx, f)
        finally:
            lb.lb_destroy(ctx)
        outs.append(f)
    # every kernel meets the oracle bound; they may differ from each other by as much (different
    # but equally valid FP32 evaluation orders, each rounded to the storage type)
    for o in outs[1:]:
        rel = np.abs(o - outs[0]) / outs[0]
        assert rel.max() <= RANDOM_FIELD_TOL[prec], rel.max()


def test_free_streaming_time_counter():
    ctx = lb.lb_init((4, 4, 4), 0.5, "f32")
    try:
        assert lb.lb_time(ctx) == 0
        lb.lb_step(ctx, 3)
        assert lb.lb_time(ctx) == 3
    finally:
        lb.lb_destroy(ctx)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_pinned_host_fields_match_device_path(prec):
    """lb_set_fields / lb_get_moments with page-locked host arrays (read and written by the kernels
    over the host link), pageable host arrays (staging buffer) and device arrays give the same
    state and the same moments, bit for bit."""
    shape = (20, 6, 5)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=44, du=0.02, drho=0.02, dtheta=0.02)
    pinned = {k: v.clone().pin_memory() for k, v in fl.items()}
    pageable = {k: v.clone() for k, v in fl.items()}
    device = {k: v.cuda() for k, v in fl.items()}
    outs = []
    for src, where in ((pinned, "host"), (pageable, "host"), (device, "device")):
        ctx = lb.lb_init(shape, 0.3, prec)
        try:
            lb.lb_set_fields(ctx, src["rho"], src["u"], src["theta"])
            lb.lb_step(ctx, 3)
            state = np.empty(lb.lb_state_bytes(ctx), dtype=np.uint8)
            lb.lb_get_state(ctx, state)
            if where == "device":
                m = {k: torch.empty_like(v) for k, v in device.items()}
            elif src is pinned:
                m = {k: torch.empty_like(v).pin_memory() for k, v in fl.items()}
            else:
                m = {k: torch.empty_like(v) for k, v in fl.items()}
            lb.lb_get_moments(ctx, m["rho"], m["u"], m["theta"])
            lb.lb_sync(ctx)
        finally:
            lb.lb_destroy(ctx)
        outs.append((state, {k: v.cpu() for k, v in m.items()}))
    for state, m in outs[1:]:
        assert np.array_equal(state, outs[0][0])
        for k in m:
            assert torch.equal(m[k], outs[0][1][k]), k
