"""Pins of the oracle's open channel (Part II, "Model and Methods": inflow at fixed velocity
on one border, outflow on the opposite one, periodic sides, bounce-back impurities)."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def _brute_stream_open(fstar, v, C, solid, opp, f_in, wall_rows):
    """Each streamed population from its definition, one at a time: the bilinear corners of
    the departure point x - C v; a corner beyond x = 0 takes the inflow equilibrium, beyond
    x = W - 1 the last column, a solid corner the reversed population of the cell itself;
    y wraps.  Solid cells hold zero."""
    q, h, w = fstar.shape
    out = np.zeros_like(fstar)
    for i in range(q):
        dx, dy = C * v[i, 0], C * v[i, 1]
        sx, sy = int(np.sign(dx)), int(np.sign(dy))
        ax, ay = abs(dx), abs(dy)
        corners = (((0, 0), (1 - ax) * (1 - ay)), ((sx, 0), ax * (1 - ay)),
                   ((0, sy), (1 - ax) * ay), ((sx, sy), ax * ay))
        for y in range(h):
            for x in range(w):
                if solid[y, x]:
                    continue
                acc = 0.0
                for (ox, oy), beta in corners:
                    if beta == 0.0:
                        continue
                    yy, xx = (y - oy) % h, x - ox
                    if wall_rows[yy]:
                        val = fstar[opp[i], y, x]
                    elif xx < 0:
                        val = f_in[i]
                    elif xx >= w:
                        val = fstar[i, yy, w - 1]
                    elif solid[yy, xx]:
                        val = fstar[opp[i], y, x]
                    else:
                        val = fstar[i, yy, xx]
                    acc += beta * val
                out[i, y, x] = acc
    return out


@pytest.mark.parametrize("walls", [False, True])
def test_stream_open_matches_its_definition(walls):
    v, w = O.velocity_set(3)
    opp = O.opposite(v)
    h, wd = 7, 9
    rng = np.random.default_rng(3)
    fstar = rng.random((26, h, wd))
    solid = np.zeros((h, wd), bool)
    solid[3, 4] = True
    wall_rows = np.zeros(h, bool)
    if walls:
        wall_rows[0] = wall_rows[-1] = True
        solid[0, :] = solid[-1, :] = True
    fstar[:, solid] = 0.0
    f_in = rng.random(26)
    got = O.stream_open(fstar, v, 0.5, solid, opp, f_in, wall_rows)
    ref = _brute_stream_open(fstar, v, 0.5, solid, opp, f_in, wall_rows)
    assert np.abs(got - ref).max() <= 1e-14


def test_uniform_inflow_state_is_steady():
    """The equilibrium moving with the inflow velocity everywhere is a fixed point."""
    nx, ny = 20, 8
    cfg = dict(nx=nx, ny=ny, open_x=1, inflow_ux=0.1, eta_over_s=0.05,
               init_ux=np.full((ny, nx), 0.1))
    E, UX, UY, _ = O.run(cfg, 15)
    assert np.abs(E - 1.0).max() <= 1e-13
    assert np.abs(UX - 0.1).max() <= 1e-13
    assert np.abs(UY).max() <= 1e-13


def test_flow_from_rest_enters_through_the_inflow_border():
    """Starting at rest, momentum arrives from the inflow side first: after a few steps the
    columns next to x = 0 move along +x and the far columns are still at rest."""
    nx, ny = 40, 6
    cfg = dict(nx=nx, ny=ny, open_x=1, inflow_ux=0.1, eta_over_s=0.05)
    E, UX, UY, _ = O.run(cfg, 6)
    jx, jy = O.column_means(UX, UY)
    assert jx[0] > 1e-3 and jx[1] > 0.0
    assert np.abs(jx[20:]).max() < 1e-12
    assert np.abs(jy).max() < 1e-14


def test_column_means():
    ux = np.array([[0.1, 0.0], [0.3, 0.0]])
    uy = np.array([[0.0, 0.2], [0.0, 0.0]])
    jx, jy = O.column_means(ux, uy)
    assert jx[0] == pytest.approx(0.5 * (0.1 / np.sqrt(1.01) + 0.3 / np.sqrt(1.09)), rel=1e-15)
    assert jy[1] == pytest.approx(0.5 * 0.2 / np.sqrt(1.04), rel=1e-15)
    jx2, _ = O.column_means(ux, uy, solid=np.array([[False, False], [True, False]]))
    assert jx2[0] == pytest.approx(0.5 * 0.1 / np.sqrt(1.01), rel=1e-15)
