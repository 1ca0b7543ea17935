"""Accuracy of the 16-bit deviation storage (FP16 / BF16, relaxed in FP32) against the
FP64 oracle over 200-step slices, as the velocity error relative to max |u|:

  (i)   the decaying shear wave (64 x 64, u = 0.01) from its initial state;
  (ii)  a stirred flow developed for 400 steps by the oracle;
  (iii) the graphene-like shape at reduced size (walls, discs, body force), a plug flow
        with perturbations relaxed for 40 steps by the oracle.

In (ii) and (iii) the oracle's state is folded into the library's planes and rounded once
to values both 16-bit types hold exactly: the common start of both runs.

FP16 with stochastic rounding meets 1e-3.  BF16 (an 8-bit significand) does not: its
cases are expected failures at the same 1e-3 bar (strict, so a pass would be reported),
and the measured error is printed."""
import os

import numpy as np
import pytest

import oracle_pool as P
from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs

pytestmark = pytest.mark.gpu

BAR = 1e-3
BF16_MISS = pytest.mark.xfail(strict=True, raises=AssertionError, reason="BF16 deviation storage misses 1e-3 of max|u| at 200 steps")
PRECISIONS = ["f16", pytest.param("bf16", marks=BF16_MISS)]


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


def u_error(gpu, ref):
    umax = max(np.abs(ref[1]).max(), np.abs(ref[2]).max())
    return max(np.abs(gpu[1] - ref[1]).max(), np.abs(gpu[2] - ref[2]).max()) / umax


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shear_wave_200_steps(R, precision):
    e, ux, uy = inputs.shear_wave(64, 64, 0.01)
    cfg = dict(nx=64, ny=64, eta_over_s=0.1, init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 200)
    lat = R.Lattice(64, 64, precision=precision, **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    lat.step(200)
    gpu = lat.moments()
    lat.close()
    err = u_error(gpu, ref)
    print("shear wave %s: u error / max|u| = %.2e" % (precision, err))
    assert np.abs(gpu[0] / ref[0] - 1.0).max() <= BAR
    assert err <= BAR


def _slice(R, precision, cfg, dev, h, walls):
    """200 steps of the oracle and of the library in `precision` from the common start h
    (library planes) at step dev; returns the velocity error and max|u| of the reference."""
    nx, ny = cfg["nx"], cfg["ny"]
    o = O.Oracle(cfg)
    start = P.unfold(R, h)
    if walls:  # the oracle's whole-domain window carries the wall rows y = -1, ny
        o.fstar = np.zeros((start.shape[0], ny + 2, nx))
        o.fstar[:, 1:-1] = start
    else:
        o.fstar = start
    o.fstar[:, o.win.solid] = 0.0
    o.step_index = dev
    o.run(200)
    E, UX, UY, _ = o.fields()
    ref = (E[1:-1], UX[1:-1], UY[1:-1]) if walls else (E, UX, UY)
    lat = R.Lattice(nx, ny, precision=precision, **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    lat.set_state(h, dev)
    lat.step(200)
    gpu = lat.moments()
    lat.close()
    return u_error(gpu, ref), np.abs(ref[1]).max(), gpu, ref


@pytest.mark.parametrize("precision", PRECISIONS)
def test_developed_stirred_slice_200_steps(R, precision):
    n = 64
    cfg = dict(nx=n, ny=n, eta_over_s=0.05, kmin=4, kmax=6, force_amp=2e-3, seed=3)
    dev = O.Oracle(cfg).run(400)
    h = P.common_start(P.fold(R, dev.fstar))
    err, umax, _, ref = _slice(R, precision, cfg, dev.step_index, h, False)
    print("stirred slice %s: u error / max|u| = %.2e (max|u| = %.2e)" % (precision, err, umax))
    if precision == "f16":  # the same start in FP32 storage reproduces the oracle closely
        lat = R.Lattice(n, n, precision="f32", **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
        lat.set_state(h, dev.step_index)
        lat.step(200)
        assert u_error(lat.moments(), ref) <= 1e-5
        lat.close()
    assert err <= BAR


@pytest.mark.parametrize("precision", PRECISIONS)
def test_walls_discs_body_force_slice_200_steps(R, precision):
    """The graphene-like shape at reduced size: x periodic, bounce-back walls in y, discs
    of radius 6 at 5 % area, a uniform body force along x.  The start: a plug flow
    u^x = 7.5e-3 (what the body force 2e-4 builds in 1000 steps) with 5 % perturbations,
    relaxed for 40 steps by the oracle."""
    nx, ny = 192, 64
    mask, _ = inputs.disc_mask(nx, ny, radius=6, fraction=0.05, seed=35, walls_y=True)
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=36, eps_amp=3e-4, u_amp=3.75e-4, kmax=4)
    ux += 7.5e-3
    cfg = dict(nx=nx, ny=ny, walls_y=1, solid=mask, body_force=(2e-4, 0.0), eta_over_s=0.05)
    dev = O.Oracle(dict(cfg, init_eps=e, init_ux=ux, init_uy=uy)).run(40)
    h = P.common_start(P.fold(R, dev.fstar[:, 1:-1]))
    err, umax, gpu, _ = _slice(R, precision, cfg, dev.step_index, h, True)
    print("walls+discs slice %s: u error / max|u| = %.2e (max|u| = %.2e)" % (precision, err, umax))
    assert np.all(gpu[0][mask != 0] == 0.0)
    assert err <= BAR


def test_stochastic_rounding_repeats_exactly(R):
    kw = dict(eta_over_s=0.05, kmin=2, kmax=4, force_amp=1e-3, seed=9)
    outs = []
    for _ in range(2):
        lat = R.Lattice(48, 40, precision="f16", **kw)
        lat.step(30)
        outs.append(lat.get_state()[0])
        lat.close()
    assert np.array_equal(outs[0], outs[1])
