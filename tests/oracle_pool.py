"""Oracle work for the GPU checks at full workload sizes, spread over the host cores.

Worker processes are spawned (never forked), one BLAS thread each.  Two kinds of job:

  * develop(): the oracle on the whole lattice for a few steps, computed as horizontal
    strips, each with nsteps + 1 rows of halo on both sides (the rows the strip's
    cells depend on), so that the strips' interiors are exactly the whole-lattice run;
  * blocks(): sample_block of the oracle, a block of cells after nsteps steps on its own
    shrinking window, from the initial fields or from a state of the whole lattice.

The fold / unfold helpers move populations between the oracle's 26 directions and the
library's folded planes (the plane order of rlbm_get_state / rlbm_set_state)."""
import multiprocessing as mp
import os

import numpy as np

from oracle import rlbm_oracle as O

_POOL = None


def pool():
    global _POOL
    if _POOL is None:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        _POOL = mp.get_context("spawn").Pool(os.cpu_count() or 1)
    return _POOL


def close():
    global _POOL
    if _POOL is not None:
        _POOL.terminate()
        _POOL.join()
        _POOL = None


def _strip_job(a):
    cfg, y0, y1, nsteps = a
    c = dict(O.DEFAULTS)
    c.update(cfg)
    nx, ny = c["nx"], c["ny"]
    halo = nsteps + 1
    lo, hi = y0 - halo, y1 + halo
    if c["walls_y"]:
        lo, hi = max(lo, -1), min(hi, ny + 1)
    ys = np.arange(lo, hi)
    o = O.Oracle(c, xs=np.arange(nx), ys=ys).run(nsteps)
    E, UX, UY, _ = o.fields()
    i0, i1 = y0 - lo, y1 - lo
    return y0, o.fstar[:, i0:i1].copy(), E[i0:i1].copy(), UX[i0:i1].copy(), UY[i0:i1].copy()


def develop_async(cfg, nsteps, nstrips=None):
    """Starts the whole-lattice run of nsteps steps from the initial fields of cfg as
    strips; .get() of the result gives the strips for assemble()."""
    ny = cfg["ny"]
    n = nstrips or (os.cpu_count() or 1)
    cuts = np.linspace(0, ny, n + 1).astype(int)
    jobs = [(cfg, int(cuts[i]), int(cuts[i + 1]), nsteps) for i in range(n) if cuts[i + 1] > cuts[i]]
    return pool().map_async(_strip_job, jobs)


def assemble(strips, ny):
    """(f* (Q, N_y, N_x), eps, u^x, u^y (N_y, N_x)) of the developed lattice."""
    strips = sorted(strips, key=lambda s: s[0])
    f = np.concatenate([s[1] for s in strips], axis=1)
    E = np.concatenate([s[2] for s in strips], axis=0)
    UX = np.concatenate([s[3] for s in strips], axis=0)
    UY = np.concatenate([s[4] for s in strips], axis=0)
    assert f.shape[1] == ny
    return f, E, UX, UY


def _block_job(a):
    cfg, x, y, nsteps, half, fw, step0 = a
    return O.sample_block(cfg, x, y, nsteps, half, fw, step0)


def blocks_async(cfg, nsteps, centres, half, fstar=None, step0=0):
    """Starts sample_block at each centre; .get() gives [(E, UX, UY), ...] in order."""
    r = nsteps + half + 1
    jobs = [(cfg, x, y, nsteps, half, None if fstar is None else O.window_populations(cfg, fstar, x, y, r), step0)
            for (x, y) in centres]
    return pool().map_async(_block_job, jobs)


def block_cells(centre, half, nx, ny, walls):
    """Lattice coordinates (y, x) of each cell of a block, or None beyond a wall."""
    out = []
    cx, cy = centre
    for dy in range(-half, half + 1):
        row = []
        for dx in range(-half, half + 1):
            y = cy + dy
            if walls and not 0 <= y < ny:
                row.append(None)
            else:
                row.append((y % ny, (cx + dx) % nx))
        out.append(row)
    return out


# --------------------------------------------------------------------------------------
# Oracle directions <-> library planes
# --------------------------------------------------------------------------------------
def class_map(R, v):
    """Index of the library's folded class of each of the oracle's 26 directions,
    matched on (v_x, v_y, v_z^2), and the class table (v_x, v_y, v_z^2, w)."""
    C = R.rlbm_velocity_classes(3)
    idx = np.empty(len(v), dtype=int)
    for i, d in enumerate(v):
        key = np.array([d[0], d[1], d[2] ** 2])
        j = np.argmin(np.abs(C[:, :3] - key).sum(axis=1))
        assert np.abs(C[j, :3] - key).sum() < 1e-12
        idx[i] = j
    return idx, C


def fold(R, fstar, eps0=1.0):
    """Oracle populations f*_i (26 directions, ...) -> library planes h_q = f_q / (w_q eps0) - 1."""
    v, _ = O.velocity_set(3)
    idx, C = class_map(R, v)
    f = np.zeros((len(C),) + fstar.shape[1:])
    for i, q in enumerate(idx):
        f[q] += fstar[i]
    f /= (C[:, 3] * eps0).reshape((-1,) + (1,) * (f.ndim - 1))
    f -= 1.0
    return f


def unfold(R, h, eps0=1.0):
    """Library planes h_q -> oracle populations: each direction takes its share w_i / w_q of
    its class (the two directions of a class differ only in the sign of v_z)."""
    v, w = O.velocity_set(3)
    idx, C = class_map(R, v)
    out = np.empty((len(v),) + h.shape[1:])
    for i, q in enumerate(idx):
        out[i] = (1.0 + h[q]) * (w[i] * eps0)
    return out


def quantise(h, precision):
    """The values of h representable in the storage type (round to nearest): FP16 by numpy,
    BF16 by rounding the FP32 bit pattern to its upper 16 bits (ties to even)."""
    if precision == "f16":
        return h.astype(np.float16).astype(np.float64)
    if precision == "bf16":
        b = np.ascontiguousarray(h, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
        return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(h.shape)
    if precision == "f32":
        return h.astype(np.float32).astype(np.float64)
    return np.array(h, dtype=np.float64)


def common_start(h):
    """A state near h that FP16, BF16 and FP32 all represent exactly (round to nearest in
    BF16, then FP16, repeated until neither changes it): the common start of runs in every
    storage type."""
    x = np.array(h, dtype=np.float64)
    for _ in range(8):
        y = quantise(quantise(x, "bf16"), "f16")
        if np.array_equal(y, x):
            return x
        x = y
    raise AssertionError("no common 16-bit representation reached")
