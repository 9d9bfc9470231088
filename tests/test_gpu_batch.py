"""Batched sweep (many independent simulations, uneven grids, per-simulation tau):
every mode against the FP64 oracle per simulation, every tile shape and both
rows-per-thread choices against the oracle, the modes against each other, the
autotuner, and the bounded grid barrier of the persistent mode."""
import numpy as np
import pytest
import torch

import oracle
from helpers import lib_to_oracle_perm, to_oracle_order
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GRIDS = [(12, 8, 6), (16, 16, 16), (20, 10, 8), (8, 8, 8), (33, 5, 4)]
# every ny even (two rows per thread allowed); nx odd, so linear tiles cross row ends mid-warp
GRIDS_EVEN = [(12, 8, 6), (16, 16, 16), (20, 10, 8), (8, 8, 8), (33, 6, 4)]
TAUS = [0.55, 0.9, 0.6, 0.75, 1.0]
TOL = {"f64": 1e-12, "f32": 2e-7}


def _fields(k, grids=GRIDS):
    th0 = lb.lb_theta0()
    return wl.random_fields(*grids[k], th0, seed=40 + k, du=0.03, drho=0.03, dtheta=0.03)


def _run(prec, mode, steps, tile=None, rows=None, grids=GRIDS):
    b = lb.lb_batch_init(grids, TAUS, prec)
    try:
        for k in range(len(grids)):
            fl = _fields(k, grids)
            lb.lb_set_fields(lb.lb_batch_sim(b, k), fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        if rows:
            lb.lb_batch_set_rows(b, rows)
        if tile:
            lb.lb_batch_set_tile(b, *tile)
        lb.lb_batch_step(b, steps, mode)
        lb.lb_batch_sync(b)
        out = []
        for k, (nx, ny, nz) in enumerate(grids):
            f = np.empty((2, 41, nz, ny, nx))
            lb.lb_get_populations(lb.lb_batch_sim(b, k), f)
            out.append(f)
    finally:
        lb.lb_batch_destroy(b)
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("mode", [lb.LB_BATCH_GRAPH, lb.LB_BATCH_PERSISTENT, lb.LB_BATCH_SEQUENTIAL])
def test_batch_modes_match_oracle(prec, mode):
    steps = 9  # odd: exercises the buffer parity bookkeeping
    perm = lib_to_oracle_perm()
    got = _run(prec, mode, steps)
    for k in range(len(GRIDS)):
        fl = _fields(k)
        ref = oracle.step(oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()), TAUS[k], steps)
        rel = np.abs(to_oracle_order(got[k], perm) - ref) / ref
        assert rel.max() <= TOL[prec], (k, rel.max())


@pytest.mark.parametrize("mode", [lb.LB_BATCH_GRAPH, lb.LB_BATCH_PERSISTENT])
def test_batch_config4_member_sizes_match_oracle(mode):
    """Members of the sizes the 64-simulation sweep draws (edges 48 and 128, the smallest odd multiple
    of 16 and the largest; tau at the sweep's extremes 0.51 and 1.0), FP32, stepped with the plan the
    autotuner picks for this batch (as the benchmark does), every population against the oracle."""
    grids = [(48, 48, 48), (128, 128, 128)]
    taus = [0.51, 1.0]
    steps = 3
    th0 = lb.lb_theta0()
    fields = [wl.random_fields(*g, th0, seed=60 + k, du=0.03, drho=0.03, dtheta=0.03) for k, g in enumerate(grids)]
    b = lb.lb_batch_init(grids, taus, "f32")
    got = []
    try:
        for k, fl in enumerate(fields):
            lb.lb_set_fields(lb.lb_batch_sim(b, k), fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_batch_tune(b, reps=1)
        lb.lb_batch_step(b, steps, mode)
        lb.lb_batch_sync(b)
        for k, (nx, ny, nz) in enumerate(grids):
            f = np.empty((2, 41, nz, ny, nx))
            lb.lb_get_populations(lb.lb_batch_sim(b, k), f)
            got.append(f)
    finally:
        lb.lb_batch_destroy(b)
    perm = lib_to_oracle_perm()
    for k, fl in enumerate(fields):
        ref = oracle.step(oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()), taus[k], steps)
        rel = np.abs(to_oracle_order(got[k], perm) - ref) / ref
        assert rel.max() <= TOL["f32"], (grids[k], rel.max())


TILES = [(16, 4), (16, 8), (32, 2), (32, 4), (64, 1), (64, 2), (128, 1), (64, 0), (128, 0)]


@pytest.mark.parametrize("tile", TILES)
def test_batch_tile_shapes_agree(tile):
    a = _run("f32", lb.LB_BATCH_GRAPH, 4, tile=tile)
    b = _run("f32", lb.LB_BATCH_SEQUENTIAL, 4)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y) / y) <= 1e-7


@pytest.mark.parametrize("rows", [1, 2])
@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("mode", [lb.LB_BATCH_GRAPH, lb.LB_BATCH_PERSISTENT])
def test_batch_rows_and_tiles_match_oracle(mode, tile, rows):
    steps = 5
    perm = lib_to_oracle_perm()
    got = _run("f32", mode, steps, tile=tile, rows=rows, grids=GRIDS_EVEN)
    for k in range(len(GRIDS_EVEN)):
        fl = _fields(k, GRIDS_EVEN)
        ref = oracle.step(oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy()), TAUS[k], steps)
        rel = np.abs(to_oracle_order(got[k], perm) - ref) / ref
        assert rel.max() <= TOL["f32"], (k, rel.max())


def test_two_rows_need_even_ny():
    b = lb.lb_batch_init(GRIDS, TAUS, "f32")
    try:
        assert lb.lb_batch_get_rows(b) == 1
        with pytest.raises(lb.LbError):
            lb.lb_batch_set_rows(b, 2)
        with pytest.raises(lb.LbError):
            lb.lb_batch_set_tile(b, 100, 0)
    finally:
        lb.lb_batch_destroy(b)
    b = lb.lb_batch_init(GRIDS_EVEN, TAUS, "f32")
    try:
        assert lb.lb_batch_get_rows(b) == 2
        lb.lb_batch_set_rows(b, 1)
        assert lb.lb_batch_get_rows(b) == 1
        lb.lb_batch_set_tile(b, 64, 0)
        for mode in (lb.LB_BATCH_GRAPH, lb.LB_BATCH_PERSISTENT):
            assert lb.lb_batch_get_plan(b, mode) == (64, 0, 1)
        with pytest.raises(lb.LbError):
            lb.lb_batch_get_plan(b, lb.LB_BATCH_SEQUENTIAL)
    finally:
        lb.lb_batch_destroy(b)


def test_tuned_plans_keep_results():
    """After tuning, both batched modes (each with its own plan) still match the sequential mode."""
    b = lb.lb_batch_init(GRIDS_EVEN, TAUS, "f32")
    outs = []
    try:
        for k in range(len(GRIDS_EVEN)):
            fl = _fields(k, GRIDS_EVEN)
            lb.lb_set_fields(lb.lb_batch_sim(b, k), fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_batch_tune(b, reps=1)
        for mode in (lb.LB_BATCH_GRAPH, lb.LB_BATCH_PERSISTENT, lb.LB_BATCH_SEQUENTIAL):
            lb.lb_batch_step(b, 3, mode)
            lb.lb_batch_sync(b)
            outs.append([])
            for k, (nx, ny, nz) in enumerate(GRIDS_EVEN):
                f = np.empty((2, 41, nz, ny, nx))
                lb.lb_get_populations(lb.lb_batch_sim(b, k), f)
                outs[-1].append(f)
    finally:
        lb.lb_batch_destroy(b)
    # three consecutive 3-step advances of the same batch: compare against the oracle instead
    perm = lib_to_oracle_perm()
    for k in range(len(GRIDS_EVEN)):
        fl = _fields(k, GRIDS_EVEN)
        f = oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())
        for m in range(3):
            f = oracle.step(f, TAUS[k], 3)
            rel = np.abs(to_oracle_order(outs[m][k], perm) - f) / f
            assert rel.max() <= TOL["f32"], (m, k, rel.max())


def test_autotuner_keeps_state_and_picks_a_shape():
    b = lb.lb_batch_init(GRIDS, TAUS, "f32")
    try:
        for k in range(len(GRIDS)):
            fl = _fields(k)
            lb.lb_set_fields(lb.lb_batch_sim(b, k), fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_batch_step(b, 3, lb.LB_BATCH_GRAPH)
        before = [torch.empty(lb.lb_state_bytes(lb.lb_batch_sim(b, k)), dtype=torch.uint8, device="cuda")
                  for k in range(len(GRIDS))]
        for k, t in enumerate(before):
            lb.lb_get_state(lb.lb_batch_sim(b, k), t)
        tx, ry, ms = lb.lb_batch_tune(b, reps=2)
        assert (tx, ry) == lb.lb_batch_get_tile(b)
        assert ms > 0
        assert lb.lb_batch_get_plan(b, lb.LB_BATCH_GRAPH) == (tx, ry, lb.lb_batch_get_rows(b))
        ptx, pry, prows = lb.lb_batch_get_plan(b, lb.LB_BATCH_PERSISTENT)
        assert [ptx, pry] in [list(t) for t in TILES] and prows == 1  # GRIDS has an odd ny
        for k, t in enumerate(before):
            after = torch.empty_like(t)
            lb.lb_get_state(lb.lb_batch_sim(b, k), after)
            assert torch.equal(after, t)
        lb.lb_batch_sync(b)
    finally:
        lb.lb_batch_destroy(b)


def test_persistent_barrier_timeout_is_reported_not_hung():
    """A grid barrier waiting for an arrival that never comes gives LB_ERR_TIMEOUT within its
    cycle budget, and the GPU stays usable."""
    b = lb.lb_batch_init(GRIDS[:2], TAUS[:2], "f32")
    try:
        lb.lb_batch_set_wait(b, 2_000_000, extra_arrivals=1)  # ~1 ms budget, barrier can never complete
        lb.lb_batch_step(b, 3, lb.LB_BATCH_PERSISTENT)
        with pytest.raises(lb.LbError) as e:
            lb.lb_batch_sync(b)
        assert e.value.status == -6
    finally:
        lb.lb_batch_destroy(b)
    # a fresh batch still runs normally
    out = _run("f32", lb.LB_BATCH_PERSISTENT, 2)
    assert all(np.isfinite(f).all() for f in out)


def test_batch_refuses_members_with_the_nonideal_mode_or_stochastic_rounding():
    """A batched step runs the energy-conserving update with the round-to-nearest store only: a
    member in the nonideal mode or with the stochastic BF16 store is refused before any launch."""
    for setup in ("nonideal", "stochastic"):
        prec = "bf16" if setup == "stochastic" else "f32"
        b = lb.lb_batch_init([(4, 4, 4), (4, 4, 6)], [0.3, 0.4], prec)
        try:
            sim = lb.lb_batch_sim(b, 1)
            if setup == "nonideal":
                lb.lb_set_nonideal(sim, 0.1, 0.3)
            else:
                lb.lb_set_stochastic_rounding(sim, 1)
            with pytest.raises(lb.LbError) as e:
                lb.lb_batch_step(b, 1)
            assert e.value.status == -7  # LB_ERR_STATE
        finally:
            lb.lb_batch_destroy(b)
