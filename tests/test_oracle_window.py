"""The oracle's windowed evaluation (used for sampled checks at full lattice
size) agrees with its full-lattice run at the sampled cells: from the initial
fields, and from a population state of the whole lattice at a later step (the
windows shrink by one ring per step)."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def _cfg(walls):
    nx, ny = 20, 14
    ex, ux, uy = inputs.smooth_random_fields(nx, ny, seed=4, u_amp=0.1)
    mask = None
    if walls:
        mask, _ = inputs.disc_mask(nx, ny, radius=2, fraction=0.05, seed=2, walls_y=True)
    return dict(nx=nx, ny=ny, walls_y=walls, solid=mask, init_eps=ex, init_ux=ux, init_uy=uy,
                eta_over_s=0.05, kmin=2, kmax=4, force_amp=1e-3, seed=11, body_force=(1e-4, 0.0))


@pytest.mark.parametrize("walls", [0, 1])
def test_sampled_equals_full(walls):
    cfg = _cfg(walls)
    E, UX, UY, _ = O.run(cfg, 3)
    pts = [(0, 0), (5, 13), (19, 7), (11, 1)]
    got = O.run_sampled(cfg, 3, pts)
    for (x, y), g in zip(pts, got):
        assert abs(g[0] - E[y, x]) < 1e-14 and abs(g[1] - UX[y, x]) < 1e-14 and abs(g[2] - UY[y, x]) < 1e-14


@pytest.mark.parametrize("walls", [0, 1])
def test_sampled_from_a_state_equals_full(walls):
    """Develop the whole lattice for 4 steps, then continue 5 steps: once on the whole
    lattice, once on shrinking windows started from the developed populations (with the
    step counter of the stirring draws carried over).  Windows of radius 6 are wider than
    the 14 rows, so they wrap (periodic) or reach past both walls."""
    cfg = _cfg(walls)
    full = O.Oracle(cfg).run(4)
    fstar = full.fstar[:, 1:-1] if walls else full.fstar  # the interior rows (N_y x N_x)
    full.run(5)
    E, UX, UY, _ = full.fields()
    if walls:
        E, UX, UY = E[1:-1], UX[1:-1], UY[1:-1]
    pts = [(0, 0), (5, 13), (19, 7), (11, 1), (3, 6)]
    got = O.run_sampled(cfg, 5, pts, fstar=fstar, step0=4)
    for (x, y), g in zip(pts, got):
        assert abs(g[0] - E[y, x]) < 1e-14 and abs(g[1] - UX[y, x]) < 1e-14 and abs(g[2] - UY[y, x]) < 1e-14


def test_window_populations_wrap_and_wall_rows():
    """x wraps; y wraps on a periodic lattice and reads zero beyond the walls."""
    q, ny, nx = 3, 6, 5
    f = np.arange(q * ny * nx, dtype=np.float64).reshape(q, ny, nx) + 1.0
    w = O.window_populations(dict(nx=nx, ny=ny, walls_y=0), f, 0, 0, 2)
    assert w.shape == (q, 5, 5)
    assert np.array_equal(w[:, 2, 2], f[:, 0, 0]) and np.array_equal(w[:, 0, 0], f[:, ny - 2, nx - 2])
    w = O.window_populations(dict(nx=nx, ny=ny, walls_y=1), f, 4, 0, 2)
    assert np.all(w[:, :2] == 0.0) and np.array_equal(w[:, 2, 3], f[:, 0, 0]) and np.array_equal(w[:, 4, 0], f[:, 2, 2])


@pytest.mark.parametrize("walls", [0, 1])
def test_sampled_block_from_a_state_equals_full(walls):
    """A block of radius 2 around the corner cell (0, 0) after 3 steps from a developed
    state: on a periodic lattice it holds the four corner cells of the lattice."""
    cfg = _cfg(walls)
    nx, ny = cfg["nx"], cfg["ny"]
    full = O.Oracle(cfg).run(2)
    fstar = full.fstar[:, 1:-1] if walls else full.fstar
    full.run(3)
    E, UX, UY, _ = full.fields()
    if walls:
        E, UX, UY = E[1:-1], UX[1:-1], UY[1:-1]
    fw = O.window_populations(cfg, fstar, 0, 0, 3 + 2 + 1)
    Eb, UXb, UYb = O.sample_block(cfg, 0, 0, 3, 2, fw, 2)
    assert Eb.shape == (5, 5)
    ys, xs = np.arange(-2, 3), np.arange(-2, 3) % nx
    for j, yy in enumerate(ys):
        if walls and not 0 <= yy < ny:
            assert np.all(Eb[j] == 0.0)  # beyond the walls: solid ghost rows
            continue
        yy %= ny
        assert np.abs(Eb[j] - E[yy, xs]).max() < 1e-14
        assert np.abs(UXb[j] - UX[yy, xs]).max() < 1e-14 and np.abs(UYb[j] - UY[yy, xs]).max() < 1e-14
