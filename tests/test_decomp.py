"""Host logic for more than one rank, on CPU ranks over gloo (world size 2 and 3).

The z-slab split with 2-plane halos is checked against the whole-grid oracle:
each rank steps its padded slab with the oracle's periodic update, the ranks
exchange halos after every step, and the gathered interiors must equal the
oracle's whole-grid result bit for bit (the per-node arithmetic does not
depend on the array it sits in).  The replica helpers (max over ranks,
aggregate rate) are checked on the same ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1909_08406_gb300 import decomp
from paper_1909_08406_gb300 import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SHAPE = (6, 5, 9)  # nx, ny, nz: nz split 5/4 over two ranks, 3/3/3 over three
TAU = 0.37
STEPS = 4


def _initial():
    th0 = oracle.theta0()
    fl = wl.random_fields(*SHAPE, th0, seed=21, du=0.05, drho=0.05, dtheta=0.05)
    return oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())


def _worker(rank, world, port, out_dir, selective):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = _initial()
        nz = f.shape[2]
        z0, z1 = decomp.slab_bounds(nz, world, rank)
        slab = decomp.pad(torch.from_numpy(np.ascontiguousarray(f[:, :, z0:z1])))
        cz2 = oracle.velocities_doubled()[:, 2]  # the oracle's velocity order
        decomp.exchange_halos(slab, cz2=cz2 if selective else None)
        for _ in range(STEPS):
            slab = torch.from_numpy(oracle.step(slab.numpy(), TAU, 1, nthreads=1))
            decomp.exchange_halos(slab, cz2=cz2 if selective else None)
        mine = decomp.interior(slab).contiguous()
        # slabs differ in thickness: rank 0 receives each one by a point-to-point message
        if rank == 0:
            parts = [mine]
            for r in range(1, world):
                a, b = decomp.slab_bounds(nz, world, r)
                parts.append(torch.empty((2, 41, b - a) + mine.shape[3:], dtype=torch.float64))
                dist.recv(parts[-1], src=r)
        else:
            dist.send(mine, dst=0)
        c = oracle.conserved(np.ascontiguousarray(mine.numpy()))
        total = decomp.allreduce_sum_f64(c)
        rate = decomp.aggregate_rate(units_this_rank=(z1 - z0) * 10.0, seconds_this_rank=1.0 + rank)
        slowest = decomp.max_over_ranks(0.5 + rank)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), torch.cat(parts, dim=2).numpy())
            np.save(os.path.join(out_dir, "conserved.npy"), np.array(total))
            np.save(os.path.join(out_dir, "replica.npy"), np.array([rate, slowest]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("selective", [True, False], ids=["selective", "full"])
@pytest.mark.parametrize("world", [2, 3])
def test_z_slabs_with_halo_exchange_match_whole_grid(world, selective, tmp_path):
    """Halos refreshed by sending every population of both halo planes, or (selective) only the
    populations an interior node reads from each plane: 18% of the bytes."""
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path), selective), nprocs=world, start_method="spawn")
    got = np.load(tmp_path / "gathered.npy")
    f0 = _initial()
    ref = oracle.step(f0, TAU, STEPS)
    assert np.array_equal(got, ref)
    # conserved sums: per-rank FP64 sums added over ranks equal the whole-grid sums to rounding
    tot = np.load(tmp_path / "conserved.npy")
    c = oracle.conserved(ref)
    assert np.allclose(tot, c, rtol=1e-13, atol=1e-13)
    rate, slowest = np.load(tmp_path / "replica.npy")
    assert slowest == 0.5 + (world - 1)
    assert rate == pytest.approx(SHAPE[2] * 10.0 / world)  # all units / slowest time (= world s)


def test_slab_bounds_cover_and_reject_thin_slabs():
    for nz, world in [(9, 2), (9, 3), (512, 8), (17, 4)]:
        spans = [decomp.slab_bounds(nz, world, r) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    with pytest.raises(ValueError):
        decomp.slab_bounds(5, 3, 0)  # slabs of 1-2 planes: thinner than the 2-plane halo


def test_single_rank_exchange_is_the_periodic_wrap():
    """With one rank a padded slab's halos are its own periodic images, so a step of the padded
    array equals a step of the whole grid on the interior."""
    f = _initial()
    p = decomp.exchange_halos(decomp.pad(torch.from_numpy(f)))
    assert torch.equal(p[:, :, :2], torch.from_numpy(f[:, :, -2:]))
    assert torch.equal(p[:, :, -2:], torch.from_numpy(f[:, :, :2]))
    stepped = oracle.step(p.numpy(), TAU, 1)
    assert np.array_equal(stepped[:, :, 2:-2], oracle.step(f, TAU, 1))


def test_selective_exchange_sends_only_what_is_read():
    """From the lower halo an interior node reads the populations with c_z > 0 (14 of 41) from the
    nearest plane and only the sc-2 one (c_z = 2) from the far plane; the upper halo mirrors it.
    Stepping a single-rank slab whose halos carry just those, with every other halo entry
    poisoned, gives the whole grid's interior bit for bit; leaving out the far plane's sc-2
    population breaks the slab's edge planes."""
    cz2 = oracle.velocities_doubled()[:, 2]
    lower, upper = decomp.halo_populations(cz2)
    assert [len(p) for p in lower] == [14, 1] and [len(p) for p in upper] == [14, 1]
    assert all(cz2[i] == 4 for i in lower[1]) and all(cz2[i] == -4 for i in upper[1])
    assert decomp.halo_fraction(cz2) == pytest.approx(30 / 164)
    f = _initial()
    ref = oracle.step(f, TAU, 1)
    p = decomp.pad(torch.from_numpy(f))
    p[:, :, :2] = float("nan")
    p[:, :, -2:] = float("nan")
    decomp.exchange_halos(p, cz2=cz2)
    assert np.array_equal(oracle.step(p.numpy(), TAU, 1)[:, :, 2:-2], ref)
    # planted omission: the far plane without its sc-2 population
    q = decomp.pad(torch.from_numpy(f))
    decomp.exchange_halos(q, cz2=cz2)
    q[:, lower[1], 0] = 0.0
    assert not np.array_equal(oracle.step(q.numpy(), TAU, 1)[:, :, 2:-2], ref)


def test_one_plane_halo_is_too_thin():
    """The sc-2 links reach two planes: with a 1-plane halo the slab's edge planes go wrong."""
    f = _initial()
    p = decomp.exchange_halos(decomp.pad(torch.from_numpy(f), halo=1), halo=1)
    stepped = oracle.step(p.numpy(), TAU, 1)
    ref = oracle.step(f, TAU, 1)
    assert not np.array_equal(stepped[:, :, 1:-1], ref)
    # planes two or more away from the slab edges are still right
    assert np.array_equal(stepped[:, :, 2:-2], ref[:, :, 1:-1])
