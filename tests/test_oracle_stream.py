"""Pins of the oracle's streaming (Sec. "Boltzmann to Lattice Boltzmann": linear
interpolation for the off-lattice momenta; Part II "Model and Methods":
bounce-back at impurity nodes)."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def tent_matrix(nx, ny, d):
    """Dense pull operator of one direction by geometric overlap: the value at x is
    the area-weighted average over the unit square centred at the departure point
    x - d, i.e. every source cell y (with its periodic images) gets weight
    max(0, 1 - |p_x - y_x|) max(0, 1 - |p_y - y_y|)."""
    M = np.zeros((nx * ny, nx * ny))
    for ty in range(ny):
        for tx in range(nx):
            px, py = tx - d[0], ty - d[1]
            for sy in range(ny):
                for sx in range(nx):
                    wx = max(0.0, 1.0 - min(abs(px - sx - k * nx) for k in (-1, 0, 1)))
                    wy = max(0.0, 1.0 - min(abs(py - sy - k * ny) for k in (-1, 0, 1)))
                    M[ty * nx + tx, sy * nx + sx] += wx * wy
    return M


@pytest.mark.parametrize("courant", [0.5, 0.83])
def test_stream_equals_dense_geometric_operator_8x8(courant):
    v, w = O.velocity_set(3)
    rng = np.random.default_rng(0)
    fstar = rng.uniform(0.0, 1.0, (26, 8, 8))
    solid = np.zeros((8, 8), bool)
    out = O.stream(fstar, v, courant, solid, O.opposite(v))
    for i in range(26):
        M = tent_matrix(8, 8, courant * v[i, :2])
        assert np.abs(out[i].ravel() - M @ fstar[i].ravel()).max() < 1e-14


def test_unit_courant_axis_directions_shift_exactly():
    v, w = O.velocity_set(3)
    rng = np.random.default_rng(1)
    fstar = rng.uniform(0.0, 1.0, (26, 6, 7))
    out = O.stream(fstar, v, 1.0, np.zeros((6, 7), bool), O.opposite(v))
    for i in range(26):
        if np.count_nonzero(np.abs(v[i]) > 1e-12) == 1 and abs(v[i, 2]) < 1e-12:
            sx, sy = int(round(v[i, 0])), int(round(v[i, 1]))
            assert np.array_equal(out[i], np.roll(fstar[i], (sy, sx), axis=(0, 1)))


@pytest.mark.parametrize("walls", [0, 1])
def test_streaming_with_bounce_back_conserves_total_energy(walls):
    """With solids the share of f*_i pulled into a solid cell is exactly the share
    bounced back into the reversed population (equal bilinear weights of i and its
    reverse), so sum over fluid cells and directions of f is unchanged."""
    nx, ny = 24, 20
    mask, _ = inputs.disc_mask(nx, ny, radius=2, fraction=0.12, seed=7, walls_y=bool(walls))
    o = O.Oracle(dict(nx=nx, ny=ny, walls_y=walls, solid=mask))
    rng = np.random.default_rng(2)
    fstar = rng.uniform(0.0, 1.0, o.fstar.shape)
    fstar[:, o.win.solid] = 0.0
    out = O.stream(fstar, o.v, o.courant, o.win.solid, o.opp)
    assert abs(out.sum() - fstar.sum()) < 1e-12 * fstar.sum()
    assert np.all(out[:, o.win.solid] == 0.0)


def test_bounce_back_channel_flow_is_poiseuille():
    """A wall-bounded channel driven by a body force settles to a symmetric
    parabolic (Poiseuille) profile whose zeros lie just outside the fluid rows,
    beyond the ghost wall rows by less than two cells (interpolated bounce-back
    places the effective wall between the ghost row and the next cell out)."""
    nx, ny = 4, 16
    o = O.Oracle(dict(nx=nx, ny=ny, walls_y=1, body_force=(1e-3, 0.0), eta_over_s=0.2)).run(300)
    E, UX, UY, _ = o.fields()
    prof = UX[1:-1, 0]
    y = np.arange(ny)
    assert np.all(prof > 0) and np.allclose(prof, prof[::-1], rtol=1e-10)
    c = np.polyfit(y, prof, 2)
    assert c[0] < 0
    assert np.abs(np.polyval(c, y) - prof).max() < 1e-2 * prof.max()
    lo, hi = sorted(np.roots(c).real)
    assert -3.0 < lo < -1.0 and ny < hi < ny + 2.0
    # mirror symmetry about the channel centre: u^y is odd, and small
    assert np.allclose(UY[1:-1, 0], -UY[1:-1, 0][::-1], rtol=1e-8, atol=1e-20)
    assert np.abs(UY).max() < 1e-3 * prof.max()


def test_translation_of_initial_field_translates_result():
    ex, ux, uy = inputs.smooth_random_fields(12, 10, seed=5, u_amp=0.1)
    base = dict(nx=12, ny=10, eta_over_s=0.05)
    a = O.run(dict(base, init_eps=ex, init_ux=ux, init_uy=uy), 6)
    b = O.run(dict(base, init_eps=np.roll(ex, (2, 3), (0, 1)), init_ux=np.roll(ux, (2, 3), (0, 1)),
                   init_uy=np.roll(uy, (2, 3), (0, 1))), 6)
    for k in range(3):
        assert np.abs(np.roll(a[k], (2, 3), (0, 1)) - b[k]).max() < 1e-14
