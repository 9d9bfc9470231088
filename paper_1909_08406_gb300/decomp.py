"""Host-side logic for spreading the update over several ranks (one process per GPU).

Two splits of the periodic bcc grid are described here.

* Replicas: every rank advances its own independent grid (or its share of a
  batch of independent simulations).  There is no data-path exchange; the
  ranks meet only to time the run (``barrier``, ``max_over_ranks``) and to
  add up the work done (``aggregate_rate``).

* z slabs of one grid: rank r owns the sc-cell planes ``slab_bounds(nz, W, r)``
  of both sub-lattices.  The update of a node pulls from at most two cells
  away along z (integer links of the sc-2 shell shift by +-2 cells; the
  bcc-1/2 links shift by 0 or 1 cell, Sec. III), so a halo of ``HALO = 2``
  planes on each side, refreshed once per step, makes the slab's interior
  update identical to the whole grid's.  A slab padded with its halos can be
  stepped by the periodic kernel as it is: the wrap only touches halo planes,
  and those are overwritten by the next exchange.  The global conserved sums
  are the FP64 sums of the ranks' interior sums.

The functions take array-like tensors in the population layout
``f[s][i][z][y][x]`` and a ``torch.distributed`` process group; with NCCL they
move device tensors, with gloo host tensors.  ``exchange_halos_lb`` does the
same exchange on a library context holding the padded slab, with the
library's packed halo messages (lb_halo_pack / lb_halo_unpack) in device
memory.
"""
from __future__ import annotations

HALO = 2


def slab_bounds(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Planes [z0, z1) of rank `rank` when nz planes are split over `world` ranks as evenly as
    possible (the first nz % world ranks get one plane more).  Every slab must hold at least
    HALO planes so that a halo comes from one neighbour only."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(nz, world)
    if base < HALO:
        raise ValueError(f"nz = {nz} over {world} ranks leaves slabs thinner than the halo ({HALO})")
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def pad(f_slab, halo: int = HALO):
    """A new tensor [2][Q][nz_local + 2 halo][ny][nx] with the slab in the middle and the halo
    planes zero; ``exchange_halos`` fills them."""
    import torch
    s, q, nzl, ny, nx = f_slab.shape
    out = torch.zeros((s, q, nzl + 2 * halo, ny, nx), dtype=f_slab.dtype, device=f_slab.device)
    out[:, :, halo:halo + nzl] = f_slab
    return out


def interior(f_padded, halo: int = HALO):
    return f_padded[:, :, halo:f_padded.shape[2] - halo]


def halo_populations(cz2, halo: int = HALO):
    """Which populations each halo plane must carry.  An interior node pulls population i from
    ceil(|c_iz|) cells away at most, on the side c_iz points from (doubled components cz2 =
    2 c_z: 1 for a bcc-1/2 link, 2 and 4 for integer links), so the halo plane at distance d from
    the interior is read only through populations with ceil(|cz2| / 2) >= d.  Returns
    (lower, upper): for each halo plane, innermost first, the population indices with c_z > 0
    (lower halo) or c_z < 0 (upper halo) that reach it."""
    cz2 = [int(v) for v in cz2]
    reach = [(abs(v) + 1) // 2 for v in cz2]
    lower = [[i for i, v in enumerate(cz2) if v > 0 and reach[i] >= d] for d in range(1, halo + 1)]
    upper = [[i for i, v in enumerate(cz2) if v < 0 and reach[i] >= d] for d in range(1, halo + 1)]
    return lower, upper


def halo_fraction(cz2, halo: int = HALO) -> float:
    """Bytes a selective exchange moves relative to sending every population of every halo plane."""
    lower, upper = halo_populations(cz2, halo)
    return sum(len(p) for p in lower + upper) / (2 * halo * len(cz2))


def exchange_halos(f_padded, group=None, halo: int = HALO, cz2=None):
    """Refresh the halo planes of a padded slab from the periodic neighbours' interiors: the
    lower halo receives the top `halo` interior planes of rank - 1, the upper halo the bottom
    `halo` interior planes of rank + 1.  One exchange per step; with one rank the slab is its
    own neighbour (the periodic wrap).  With `cz2` (the doubled z components of the populations
    in the array's velocity order) only the populations an interior node reads from each halo
    plane are sent (``halo_populations``: 15 of the 82 plane-populations of a 2-plane halo per
    sub-lattice pair and direction); the others keep stale values that no interior update reads."""
    import numpy as np
    import torch
    import torch.distributed as dist
    nzp = f_padded.shape[2]
    if cz2 is None:
        every = list(range(f_padded.shape[1]))
        lower, upper = [every] * halo, [every] * halo
    else:
        lower, upper = halo_populations(cz2, halo)
    # receiver's lower halo plane at distance d (index halo - d) <- sender's plane nzp - halo - d;
    # receiver's upper halo plane at distance d (index nzp - halo + d - 1) <- sender's plane halo + d - 1
    def pack(planes_pops):
        return torch.cat([f_padded[:, pops, z].reshape(-1) for z, pops in planes_pops]).contiguous()

    def unpack(buf, planes_pops):
        k = 0
        for z, pops in planes_pops:
            shape = f_padded[:, pops, z].shape
            n = int(np.prod(shape))
            f_padded[:, pops, z] = buf[k:k + n].reshape(shape)
            k += n

    hi_src = [(nzp - halo - d, lower[d - 1]) for d in range(1, halo + 1)]  # to rank + 1
    lo_src = [(halo + d - 1, upper[d - 1]) for d in range(1, halo + 1)]    # to rank - 1
    lo_dst = [(halo - d, lower[d - 1]) for d in range(1, halo + 1)]        # from rank - 1
    hi_dst = [(nzp - halo + d - 1, upper[d - 1]) for d in range(1, halo + 1)]  # from rank + 1
    hi_send, lo_send = pack(hi_src), pack(lo_src)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        unpack(hi_send, lo_dst)
        unpack(lo_send, hi_dst)
        return f_padded
    rank = dist.get_rank(group)
    down, up = (rank - 1) % world, (rank + 1) % world
    lo_recv = torch.empty_like(hi_send)
    hi_recv = torch.empty_like(lo_send)
    # tag 0: planes going up (they land in the receiver's lower halo); tag 1: going down
    ops = [dist.P2POp(dist.isend, hi_send, up, group, 0), dist.P2POp(dist.isend, lo_send, down, group, 1),
           dist.P2POp(dist.irecv, lo_recv, down, group, 0), dist.P2POp(dist.irecv, hi_recv, up, group, 1)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    unpack(lo_recv, lo_dst)
    unpack(hi_recv, hi_dst)
    return f_padded


def exchange_halos_lb(ctx, bufs, group=None):
    """The exchange of ``exchange_halos`` on a library context that holds this rank's padded slab
    (lb_init with nz = nz_r + 2 HALO): the library packs the populations an interior node reads
    from each halo plane into device buffers and unpacks the received ones (lb_halo_pack,
    lb_halo_unpack); the ranks swap them by NCCL point-to-point.  ``bufs`` = four uint8 device
    tensors of ``lb.lb_halo_bytes(ctx)`` bytes (top and bottom to send, lower and upper to
    receive), reused from step to step.  With one rank the slab is its own neighbour."""
    import torch.distributed as dist
    from . import lb
    send_up, send_down, recv_low, recv_high = bufs
    lb.lb_halo_pack(ctx, 1, send_up)
    lb.lb_halo_pack(ctx, 0, send_down)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        lb.lb_halo_unpack(ctx, 0, send_up)
        lb.lb_halo_unpack(ctx, 1, send_down)
        return
    lb.lb_sync(ctx)  # the packed messages are complete before the communicator reads them
    rank = dist.get_rank(group)
    down, up = (rank - 1) % world, (rank + 1) % world
    ops = [dist.P2POp(dist.isend, send_up, up, group, 0), dist.P2POp(dist.isend, send_down, down, group, 1),
           dist.P2POp(dist.irecv, recv_low, down, group, 0), dist.P2POp(dist.irecv, recv_high, up, group, 1)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    lb.lb_halo_unpack(ctx, 0, recv_low)
    lb.lb_halo_unpack(ctx, 1, recv_high)


def exchange_halos_lb_local(ctxs, bufs):
    """The same exchange among slabs held by one process, in rank order around the ring (used to
    check the library's slab path on one device): rank r's top interior goes to rank r + 1's
    lower halo, its bottom interior to rank r - 1's upper halo.  ``bufs[r]`` as above."""
    from . import lb
    n = len(ctxs)
    for r in range(n):  # earlier unpacks from the buffers are complete before they are refilled
        lb.lb_sync(ctxs[r])
    for r in range(n):
        lb.lb_halo_pack(ctxs[r], 1, bufs[r][0])
        lb.lb_halo_pack(ctxs[r], 0, bufs[r][1])
    for r in range(n):
        lb.lb_sync(ctxs[r])
    for r in range(n):
        lb.lb_halo_unpack(ctxs[r], 0, bufs[(r - 1) % n][0])
        lb.lb_halo_unpack(ctxs[r], 1, bufs[(r + 1) % n][1])


def allreduce_sum_f64(values, group=None, device="cpu"):
    """Sum of a few FP64 numbers over the ranks (the global conserved quantities)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.cpu()]


def barrier(group=None):
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.barrier(group)


def max_over_ranks(x: float, group=None, device="cpu") -> float:
    """The largest of the ranks' values (the time of the slowest rank bounds the job)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def aggregate_rate(units_this_rank: float, seconds_this_rank: float, group=None, device="cpu") -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    total = allreduce_sum_f64([units_this_rank], group, device)[0]
    return total / max_over_ranks(seconds_this_rank, group, device)
