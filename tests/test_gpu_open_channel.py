"""GPU parity of the open channel (Part II): inflow equilibrium at x = 0, zero-gradient
outflow at x = nx - 1, periodic or walled sides, bounce-back impurities, against the FP64
oracle; and the current density (column means of v)."""
import os

import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-10, "f32": 1e-5}


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04658_gb300 import build as B
    from paper_2205_04658_gb300 import rlbm
    if not os.path.exists(rlbm.LIB_PATH):
        B.build()
    return rlbm


def _disc(nx, ny, cx, cy, r):
    Y, X = np.mgrid[0:ny, 0:nx]
    return ((X - cx) ** 2 + (Y - cy) ** 2 <= r * r).astype(np.uint8)


def _run(R, cfg, nsteps, precision):
    lat = R.Lattice(cfg["nx"], cfg["ny"], precision=precision, **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    lat.step(nsteps)
    out = lat.moments()
    jx, jy = lat.column_means()
    lat.close()
    return out, jx, jy


def _check(gpu, ref, solid, tol):
    fluid = solid == 0
    assert np.max(np.abs(gpu[0][fluid] / ref[0][fluid] - 1.0)) <= tol
    umax = max(np.abs(ref[1]).max(), np.abs(ref[2]).max())
    assert max(np.abs(gpu[1] - ref[1]).max(), np.abs(gpu[2] - ref[2]).max()) <= tol * umax


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_channel_with_impurity_periodic_sides(R, precision):
    """72 x 24, one disc of radius 3 near the inflow, uniform start at the inflow speed 0.1,
    150 steps (the vortex street's onset is not reached; the wake is)."""
    nx, ny = 72, 24
    solid = _disc(nx, ny, 14, 12, 3)
    cfg = dict(nx=nx, ny=ny, open_x=1, inflow_ux=0.1, solid=solid, eta_over_s=0.05,
               init_ux=np.full((ny, nx), 0.1))
    ref = O.run(cfg, 150)
    gpu, jx, jy = _run(R, cfg, 150, precision)
    _check(gpu, ref, solid, TOL[precision])
    rjx, rjy = O.column_means(ref[1], ref[2], solid != 0)
    assert np.abs(jx - rjx).max() <= TOL[precision] * np.abs(rjx).max()
    assert np.abs(jy - rjy).max() <= TOL[precision] * np.abs(rjx).max() + 1e-15


def test_channel_with_walls_and_two_impurities_fp64(R):
    nx, ny = 64, 20
    solid = np.maximum(_disc(nx, ny, 12, 8, 2), _disc(nx, ny, 20, 13, 2))
    cfg = dict(nx=nx, ny=ny, open_x=1, walls_y=1, inflow_ux=0.05, solid=solid, eta_over_s=0.08,
               init_ux=np.full((ny, nx), 0.05))
    ref = O.run(cfg, 120)
    gpu, _, _ = _run(R, cfg, 120, "f64")
    _check(gpu, ref, solid, 1e-10)


def test_flow_from_rest_and_sixteen_bit_storage(R):
    """From rest: the FP64 library against the oracle; FP16 storage within 1e-3 of max |u|."""
    nx, ny = 80, 16
    cfg = dict(nx=nx, ny=ny, open_x=1, inflow_ux=0.1, eta_over_s=0.05)
    ref = O.run(cfg, 100)
    g64, _, _ = _run(R, cfg, 100, "f64")
    _check(g64, ref, np.zeros((ny, nx), np.uint8), 1e-10)
    g16, _, _ = _run(R, cfg, 100, "f16")
    umax = np.abs(ref[1]).max()
    assert np.abs(g16[1] - ref[1]).max() <= 1e-3 * umax


def test_uniform_inflow_state_is_steady_on_the_gpu(R):
    nx, ny = 96, 40
    cfg = dict(nx=nx, ny=ny, open_x=1, inflow_ux=0.1, eta_over_s=0.05, init_ux=np.full((ny, nx), 0.1))
    gpu, jx, _ = _run(R, cfg, 200, "f32")
    assert np.abs(gpu[1] - 0.1).max() <= 1e-6
    assert np.abs(jx - 0.1 / np.sqrt(1.01)).max() <= 1e-6


def test_open_channel_is_rejected_by_batches_and_the_adjoint(R):
    import torch
    s = torch.cuda.Stream()
    a = R.Lattice(32, 16, stream=s, precision="f32", open_x=1, inflow_ux=0.1)
    with pytest.raises(R.RlbmError) as e:
        R.Batch([a], stream=s)
    assert e.value.status == R.RLBM_E_INVAL
    with pytest.raises(R.RlbmError) as e:
        a.gradient(4)
    assert e.value.status == R.RLBM_E_INVAL
    a.close()


def test_current_density_pipeline(R):
    """j(t) at the outflow and j(x) downstream of an impurity in a reduced Part II channel,
    and their fluctuation spectra."""
    from paper_2205_04658_gb300 import analysis as A, inputs as I, units as U
    nx, ny = 256, 64
    mask = I.channel_impurities(nx, ny, 13)
    es = U.eta_over_s_for_reynolds(6.37, 13, 0.1)
    lat = R.Lattice(nx, ny, precision="f32", open_x=1, inflow_ux=0.1, solid=mask, eta_over_s=es,
                    init_ux=np.full((ny, nx), 0.1))
    out = A.current_density_run(lat, 600, every=5)
    lat.close()
    assert out["j_t"].shape == (120,) and out["j_x"].shape == (nx // 2,)
    assert np.all(np.isfinite(out["j_t"])) and np.all(out["j_t"] > 0.0)
    # the impurity blocks part of the cross-section: downstream j stays below the inflow's
    assert out["j_x"].max() < 0.1 / np.sqrt(1.01) * 1.05
    pw = A.fluctuation_spectrum(out["j_t"])
    assert pw.shape == (61,) and np.all(pw >= 0.0) and pw[0] < 1e-20
