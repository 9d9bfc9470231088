"""The stochastic BF16 store (lb_set_stochastic_rounding) against the oracle, through the C ABI.

One step from a state both sides hold exactly: the oracle's equilibrium of random fields with
h = f/w - 1 rounded to BF16 on the host, set as the raw BF16 state.  The oracle's FP64 step gives
every post-collision h, and its generator (oracle/stochastic_rounding.py) the 16 random bits r.
The library evaluates the step in FP32, within DELTA of FP64 (absolute, in h; the FP32 parity
bound of one step).  Wherever the FP64 value lies farther than DELTA from the point where r flips
the rounding, and from both BF16 neighbours, the stored value is fixed: it must equal the
oracle's exactly.  Every other value must lie within one BF16 spacing of the FP64 value.  Most
values must be decided, so the generator's keys (step, node, population) are checked bit for bit.
Both kernels that carry the store run: the x-pair kernel (nx even) and one node per thread
(nx odd).

The accuracy gain over round to nearest is in test_gpu_storage_error.py."""
import numpy as np
import pytest
import torch

import oracle
from helpers import lib_to_oracle_perm, to_lib_order, to_oracle_order
from oracle import stochastic_rounding as sr
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DELTA = 5e-7
SEED = 0x9E3779B97F4A7C15


def _bf16_round_trip_state(shape, seed, perm, w_lib):
    """(h of the initial state in library order as float64 BF16 values, the same as oracle f)."""
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=seed, du=0.02, drho=0.02, dtheta=0.02)
    f0 = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
    w = np.asarray(w_lib)[None, :, None, None, None]
    h = sr.round_bf16_nearest(to_lib_order(f0, perm) / w - 1.0)
    return h, to_oracle_order(w * (1.0 + h), perm)


def _node_index(shape):
    nx, ny, nz = shape
    s = np.arange(2).reshape(2, 1, 1, 1, 1)
    z = np.arange(nz).reshape(1, 1, nz, 1, 1)
    y = np.arange(ny).reshape(1, 1, 1, ny, 1)
    x = np.arange(nx).reshape(1, 1, 1, 1, nx)
    return (s * (nx * ny * nz) + (z * ny + y) * nx + x).astype(np.uint64)


@pytest.mark.parametrize("shape,kernel", [((16, 6, 5), lb.LB_KERNEL_DIRECT2XL), ((262, 3, 2), lb.LB_KERNEL_DIRECT2XL),
                                          ((13, 6, 5), lb.LB_KERNEL_DIRECT1)])
@pytest.mark.parametrize("steps_before", [0, 2])
def test_stochastic_store_matches_oracle(shape, kernel, steps_before):
    perm = lib_to_oracle_perm()
    c2, w_lib = lb.lb_velocity_set()
    h0, f0_or = _bf16_round_trip_state(shape, 11 + shape[0], perm, w_lib)
    tau = 0.3
    nx, ny, nz = shape
    ctx = lb.lb_init(shape, tau, "bf16")
    try:
        lb.lb_set_state(ctx, torch.from_numpy(h0).to(torch.bfloat16).contiguous())
        back = torch.empty((2, 41, nz, ny, nx), dtype=torch.bfloat16)
        lb.lb_get_state(ctx, back)
        assert np.array_equal(back.to(torch.float64).numpy(), h0)
        lb.lb_set_stochastic_rounding(ctx, SEED)
        if steps_before:
            # the key's step number counts the steps since enabling: take some, then restore the
            # initial state, so the checked step is step number steps_before
            lb.lb_step(ctx, steps_before)
            lb.lb_set_state(ctx, torch.from_numpy(h0).to(torch.bfloat16).contiguous())
        lb.lb_step(ctx, 1)
        assert lb.lb_step_variant(ctx) == kernel
        got = torch.empty((2, 41, nz, ny, nx), dtype=torch.bfloat16)
        lb.lb_get_state(ctx, got)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    h_gpu = got.to(torch.float64).numpy()

    w = np.asarray(w_lib)[None, :, None, None, None]
    h64 = to_lib_order(oracle.step(f0_or, tau, 1), perm) / w - 1.0
    q = _node_index(shape)
    i = np.arange(41).reshape(1, 41, 1, 1, 1)
    r = sr.random_bits(sr.step_key(SEED, steps_before), q, i).astype(np.float64)

    a = np.abs(h64).astype(np.float32).view(np.uint32)
    lo = (a & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((a & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    spacing = hi - lo
    frac = (np.abs(h64) - lo) / spacing  # position between the two neighbours, in [0, 1)
    flip = 1.0 - r / 65536.0             # rounds up iff the FP32 value's fraction >= flip
    decided = ((np.abs(frac - flip) * spacing > DELTA) & (frac * spacing > DELTA)
               & ((1.0 - frac) * spacing > DELTA))
    expect = np.sign(h64) * np.where(frac >= flip, hi, lo)
    assert decided.mean() > 0.9, decided.mean()
    bad = decided & (h_gpu != expect)
    assert not bad.any(), (int(bad.sum()), h_gpu[bad][:5], expect[bad][:5], h64[bad][:5])
    assert np.all(np.abs(h_gpu - h64) <= spacing + DELTA)
    # the store is not round to nearest: a good share of the decided values went the other way
    rn = sr.round_bf16_nearest(h64)
    assert 0.05 < float((decided & (h_gpu != rn)).mean()) < 0.6


def test_arguments_and_exclusions():
    ctx = lb.lb_init((8, 4, 4), 0.3, "f16")
    try:
        with pytest.raises(lb.LbError):
            lb.lb_set_stochastic_rounding(ctx, 1)
    finally:
        lb.lb_destroy(ctx)
    ctx = lb.lb_init((8, 4, 4), 0.3, "bf16", flags=lb.LB_FLAG_PAPER_LITERAL)
    try:
        with pytest.raises(lb.LbError):
            lb.lb_set_stochastic_rounding(ctx, 1)
    finally:
        lb.lb_destroy(ctx)
    th0 = lb.lb_theta0()
    ctx = lb.lb_init((8, 4, 4), 0.3, "bf16")
    try:
        lb.lb_set_stochastic_rounding(ctx, 5)
        with pytest.raises(lb.LbError):
            lb.lb_set_walls(ctx, (0.0, 0.0, th0), (0.0, 0.0, th0))
        with pytest.raises(lb.LbError):
            lb.lb_set_nonideal(ctx, 0.1, 0.3)
        lb.lb_set_stochastic_rounding(ctx, None)
        lb.lb_set_walls(ctx, (0.0, 0.0, th0), (0.0, 0.0, th0))
        with pytest.raises(lb.LbError):
            lb.lb_set_stochastic_rounding(ctx, 5)
    finally:
        lb.lb_destroy(ctx)
