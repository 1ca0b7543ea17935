"""Domain decomposition on host ranks: world-size 2 and 4 gloo process groups, each rank
running the FP64 oracle on its own strip of rows.  Before the first step and after every
step the ranks swap their boundary rows (all populations of the row) with
paper_2205_04658_gb300.strips.exchange, the point-to-point exchange the strip contexts of
the library use between processes; the totals are summed over ranks with an FP64
all-reduce.  The fields must equal the single-domain oracle run bit for bit, periodic in y
and between walls with discs that straddle the strip edges."""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs
from paper_2205_04658_gb300 import strips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEPS = 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _config(walls):
    nx, ny = 24, 32
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=13, eps_amp=0.02, u_amp=0.05)
    cfg = dict(nx=nx, ny=ny, init_eps=e, init_ux=ux, init_uy=uy, eta_over_s=0.05, kmin=2, kmax=4,
               force_amp=1e-3, seed=19)
    if walls:
        # discs centred on strip edges (rows 8, 16, 24 split the lattice into 2 or 4 strips)
        mask = np.zeros((ny, nx), np.uint8)
        Y, X = np.mgrid[0:ny, 0:nx]
        for cx, cy in ((5, 8), (17, 16), (11, 24)):
            mask[(X - cx) ** 2 + (Y - cy) ** 2 <= 4] = 1
        cfg.update(walls_y=1, solid=mask, body_force=(2e-4, -1e-4))
    return cfg


def _interior_totals(o):
    """(sum T^00, T^0x, T^0y, 1/2 |v|^2) over the fluid cells of the window's interior rows."""
    f = o.streamed()[:, 1:-1]
    fluid = ~o.win.solid[1:-1]
    T = O.moments(f[:, fluid], o.v)
    eps, u = O.landau(T)
    vx, vy = u[:, 1] / u[:, 0], u[:, 2] / u[:, 0]
    return np.array([T[:, 0, 0].sum(), T[:, 0, 1].sum(), T[:, 0, 2].sum(), 0.5 * (vx * vx + vy * vy).sum()])


def _rank(rank, world, port, walls, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _config(walls)
    periodic = not walls
    y0, y1 = strips.strip_rows(cfg["ny"], world)[rank]
    o = O.Oracle(cfg, xs=np.arange(cfg["nx"]), ys=np.arange(y0 - 1, y1 + 1))
    lo, hi = strips.neighbours(rank, world, periodic)

    def swap():
        send_lo = torch.from_numpy(np.ascontiguousarray(o.fstar[:, 1]))
        send_hi = torch.from_numpy(np.ascontiguousarray(o.fstar[:, -2]))
        recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
        strips.exchange(dist, send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic)
        if lo is not None:
            o.fstar[:, 0] = recv_lo.numpy()
        if hi is not None:
            o.fstar[:, -1] = recv_hi.numpy()

    swap()
    for _ in range(NSTEPS):
        o.step()
        swap()
    E, UX, UY, _ = o.fields()
    tot = torch.from_numpy(_interior_totals(o))
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    q.put((rank, y0, E[1:-1], UX[1:-1], UY[1:-1], tot.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("walls", [0, 1])
def test_strips_on_gloo_ranks_equal_the_whole_lattice(world, walls):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, walls, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    E = np.concatenate([o[2] for o in out])
    UX = np.concatenate([o[3] for o in out])
    UY = np.concatenate([o[4] for o in out])
    Er, UXr, UYr, totr = O.run(_config(walls), NSTEPS)
    assert np.array_equal(E, Er) and np.array_equal(UX, UXr) and np.array_equal(UY, UYr)
    for o in out:  # every rank holds the same all-reduced totals
        assert np.array_equal(o[5], out[0][5])
        assert np.abs(o[5] - totr).max() <= 1e-13 * totr[0]


def test_neighbours_and_rows():
    assert strips.strip_rows(100, 3) == [(0, 33), (33, 66), (66, 100)]
    assert strips.neighbours(0, 4, True) == (3, 1) and strips.neighbours(3, 4, True) == (2, 0)
    assert strips.neighbours(0, 4, False) == (None, 1) and strips.neighbours(3, 4, False) == (2, None)
    assert strips.neighbours(0, 1, True) == (0, 0) and strips.neighbours(0, 1, False) == (None, None)
