"""A lattice decomposed over two processes (gloo process group), each holding one strip
context of the library on the GPU and exchanging the crossing planes with the other after
every step (strips.DistributedStrip: pack on the device, messages staged through pinned
host memory, point-to-point gloo messages, unpack): the fields equal one context's bit for
bit and the FP64 all-reduced totals equal its totals.  The two processes share the one GPU;
no kernel of one waits on the other's, only the host exchange orders them."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2205_04658_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, NSTEPS = 96, 100, 30


def _config(walls):
    e, ux, uy = inputs.smooth_random_fields(NX, NY, seed=41, eps_amp=0.02, u_amp=0.04, kmax=4)
    kw = dict(eta_over_s=0.05, kmin=2, kmax=5, force_amp=1e-3, seed=29, init_eps=e, init_ux=ux, init_uy=uy)
    if walls:
        mask = np.zeros((NY, NX), np.uint8)
        Y, X = np.mgrid[0:NY, 0:NX]
        for cx, cy in ((12, 50), (60, 49), (80, 20)):  # two discs across the strip edge at row 50
            mask[(X - cx) ** 2 + (Y - cy) ** 2 <= 9] = 1
        kw.update(walls_y=1, solid=mask, body_force=(2e-4, 0.0))
    return kw


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, precision, walls, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2205_04658_gb300 import strips
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = strips.DistributedStrip(dist, NX, NY, precision=precision, **_config(walls))
    s.step(NSTEPS)
    E, UX, UY, tot = s.moments()
    q.put((rank, s.y0, E, UX, UY, tot, s.lat.current_step))
    s.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("walls", [0, 1])
def test_two_processes_equal_one_context(precision, walls):
    import multiprocessing as mp
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04658_gb300 import build as B
    from paper_2205_04658_gb300 import rlbm
    if not os.path.exists(rlbm.LIB_PATH):
        B.build()
    one = rlbm.Lattice(NX, NY, precision=precision, **_config(walls))
    one.step(NSTEPS)
    E, UX, UY, tot = one.moments()
    one.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, precision, walls, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(o[6] == NSTEPS for o in out)
    assert np.array_equal(np.concatenate([o[2] for o in out]), E)
    assert np.array_equal(np.concatenate([o[3] for o in out]), UX)
    assert np.array_equal(np.concatenate([o[4] for o in out]), UY)
    for o in out:
        assert np.abs(o[5] - tot).max() <= 1e-12 * abs(tot[0])
