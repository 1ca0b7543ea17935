"""The oracle's windowed evaluation (used for sampled checks at full lattice
size) agrees with its full-lattice run at the sampled cells."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


@pytest.mark.parametrize("walls", [0, 1])
def test_sampled_equals_full(walls):
    nx, ny = 20, 14
    ex, ux, uy = inputs.smooth_random_fields(nx, ny, seed=4, u_amp=0.1)
    mask = None
    if walls:
        mask, _ = inputs.disc_mask(nx, ny, radius=2, fraction=0.05, seed=2, walls_y=True)
    cfg = dict(nx=nx, ny=ny, walls_y=walls, solid=mask, init_eps=ex, init_ux=ux, init_uy=uy,
               eta_over_s=0.05, kmin=2, kmax=4, force_amp=1e-3, seed=11, body_force=(1e-4, 0.0))
    E, UX, UY, _ = O.run(cfg, 3)
    pts = [(0, 0), (5, 13), (19, 7), (11, 1)]
    got = O.run_sampled(cfg, 3, pts)
    for (x, y), g in zip(pts, got):
        assert abs(g[0] - E[y, x]) < 1e-14 and abs(g[1] - UX[y, x]) < 1e-14 and abs(g[2] - UY[y, x]) < 1e-14
