"""The library's z-slab path (lb_halo_pack / lb_halo_unpack, lb_conserved_planes) on one GPU.

A periodic grid is split into W slabs along z, each held by its own context padded with
LB_HALO = 2 halo planes below and above and stepped by the ordinary update; before every step
the halos are refreshed from the neighbouring slabs' interiors through the library's packed
messages (decomp.exchange_halos_lb_local: the ring of ranks emulated in one process, the
contexts stepped one after another, no kernel waiting on another).  The slab interiors must then
equal the whole grid's state bit for bit after every number of steps, since every interior node
performs the same arithmetic on the same inputs; the sums of the interiors' conserved quantities
must equal the whole grid's (FP64 sums in another order: 1e-12 relative).  The host logic of the
ring, with oracle stepping and gloo ranks, is in test_decomp.py."""
import numpy as np
import pytest
import torch

from paper_1909_08406_gb300 import decomp, lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
H = lb.LB_HALO
DT = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def _bits(t):
    return t.contiguous().view({2: torch.int16, 4: torch.int32, 8: torch.int64}[t.element_size()])


def _raw(ctx, shape, prec):
    nx, ny, nz = shape
    t = torch.empty((2, 41, nz, ny, nx), dtype=DT[prec], device="cuda")
    lb.lb_get_state(ctx, t)
    return t


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("world,nz", [(2, 12), (3, 13)])
def test_slabs_match_whole_grid(prec, world, nz):
    nx, ny = 16, 6
    th0 = lb.lb_theta0()
    fl = wl.random_fields(nx, ny, nz, th0, seed=3, du=0.03, drho=0.03, dtheta=0.03)
    tau, steps = 0.4, 6
    whole = lb.lb_init((nx, ny, nz), tau, prec)
    ctxs, bufs = [], []
    try:
        lb.lb_set_fields(whole, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        full = _raw(whole, (nx, ny, nz), prec)
        bounds = [decomp.slab_bounds(nz, world, r) for r in range(world)]
        for z0, z1 in bounds:
            nzp = z1 - z0 + 2 * H
            ctx = lb.lb_init((nx, ny, nzp), tau, prec)
            idx = torch.tensor([(z0 - H + k) % nz for k in range(nzp)], device="cuda")
            lb.lb_set_state(ctx, full.index_select(2, idx).contiguous())
            ctxs.append(ctx)
            n = lb.lb_halo_bytes(ctx)
            bufs.append([torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(2)])
        for t in range(1, steps + 1):
            decomp.exchange_halos_lb_local(ctxs, bufs)
            for ctx in ctxs:
                lb.lb_step(ctx, 1)
            lb.lb_step(whole, 1)
            ref = _raw(whole, (nx, ny, nz), prec)
            for (z0, z1), ctx in zip(bounds, ctxs):
                got = _raw(ctx, (nx, ny, z1 - z0 + 2 * H), prec)[:, :, H:H + z1 - z0]
                assert torch.equal(_bits(got), _bits(ref[:, :, z0:z1])), (prec, t)
        c_whole = np.array(lb.lb_conserved(whole))
        c_sum = sum(np.array(lb.lb_conserved_planes(ctx, H, H + z1 - z0)) for (z0, z1), ctx in zip(bounds, ctxs))
        assert np.all(np.abs(c_sum - c_whole) <= 1e-12 * np.maximum(1.0, np.abs(c_whole))), (c_sum, c_whole)
    finally:
        lb.lb_destroy(whole)
        for ctx in ctxs:
            lb.lb_destroy(ctx)


def test_halo_message_size_and_arguments():
    ctx = lb.lb_init((8, 4, 10), 0.4, "f32")
    try:
        # 15 plane-populations per direction, both sub-lattices, 8 x 4 FP32 values each
        assert lb.lb_halo_bytes(ctx) == 15 * 2 * 8 * 4 * 4
        with pytest.raises(ValueError):
            lb.lb_halo_pack(ctx, 1, torch.empty(16, dtype=torch.uint8, device="cuda"))
        with pytest.raises(lb.LbError):
            lb.lb_halo_pack(ctx, 2, torch.empty(lb.lb_halo_bytes(ctx), dtype=torch.uint8, device="cuda"))
        with pytest.raises(lb.LbError):
            lb.lb_conserved_planes(ctx, 3, 3)
    finally:
        lb.lb_destroy(ctx)
    small = lb.lb_init((8, 4, 5), 0.4, "f32")
    try:
        with pytest.raises(lb.LbError):
            lb.lb_halo_bytes(small)
    finally:
        lb.lb_destroy(small)
