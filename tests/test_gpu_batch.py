"""The batched form: many lattices of uneven sizes advanced by one persistent launch
per step (CUDA-graph replay for whole chunks) must give exactly the results of
stepping each lattice on its own, and every member must match the FP64 oracle run of
its own configuration."""
import os

import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs

pytestmark = pytest.mark.gpu


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


MEMBERS = [  # (nx, ny, seed, walls/discs)
    (64, 48, 11, False), (96, 80, 12, False), (40, 40, 13, False), (128, 64, 14, True), (72, 56, 15, False),
]


def member_config(nx, ny, seed, solid):
    """Members share the physics (eta/s, stirring shell and amplitude, body force); they
    differ in size, seeds, initial fields, walls and solids."""
    kw = dict(eta_over_s=0.05, kmin=2, kmax=5, force_amp=1e-3, seed=seed, body_force=(1e-4, -5e-5))
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=seed, eps_amp=0.02, u_amp=0.02)
    kw.update(init_eps=e, init_ux=ux, init_uy=uy)
    if solid:
        mask, _ = inputs.disc_mask(nx, ny, radius=3, fraction=0.05, seed=seed, walls_y=True)
        kw.update(walls_y=1, solid=mask)
    return kw


def make(R, precision, stream, nx, ny, seed, solid):
    return R.Lattice(nx, ny, stream=stream, precision=precision, **member_config(nx, ny, seed, solid))


@pytest.mark.parametrize("precision", ["f32", "f16", "bf16", "f64"])
def test_batch_equals_members_stepped_alone(R, precision):
    import torch
    stream = torch.cuda.Stream()
    alone, batched = [], []
    for (nx, ny, seed, solid) in MEMBERS:
        alone.append(make(R, precision, stream, nx, ny, seed, solid))
        batched.append(make(R, precision, stream, nx, ny, seed, solid))
    # members need not be at the same step: advance one of them first, in both sets
    alone[2].step(5)
    batched[2].step(5)
    nsteps = 70  # one captured chunk of 64 steps + 6 direct launches
    for lat in alone:
        lat.step(nsteps)
    b = R.Batch(batched, stream=stream)
    # tuned before the first step too (the member table is valid from rlbm_batch_init on)
    assert b.autotune(1) > 0.0
    b.step(nsteps)
    # the autotuner changes the launch shape only: the members are not advanced and the
    # next steps are the same arithmetic
    assert b.autotune(2) > 0.0
    b.step(3)
    for lat in alone:
        lat.step(3)
    for a, c in zip(alone, batched):
        assert a.current_step == c.current_step
        ma, mc = a.moments(), c.moments()
        for k in range(3):
            assert np.array_equal(ma[k], mc[k])
    b.close()
    for lat in alone + batched:
        lat.close()


def test_batch_rejects_mismatched_physics(R):
    import torch
    stream = torch.cuda.Stream()
    a = R.Lattice(32, 32, stream=stream, precision="f32", eta_over_s=0.05)
    c = R.Lattice(32, 32, stream=stream, precision="f32", eta_over_s=0.06)
    with pytest.raises(R.RlbmError) as e:
        R.Batch([a, c], stream=stream)
    assert e.value.status == R.RLBM_E_INVAL
    a.close()
    c.close()


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_many_small_members_and_a_single_member(R, precision):
    """40 members of two to nine tiles each (the staging thread's member search steps over
    several members per tile; each CTA's share of the next-step tables spans several
    members), and a batch of one member: both equal the members stepped alone."""
    import torch
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(1, 4)) * 32 - int(rng.integers(0, 20)), int(rng.integers(1, 3)) * 8 + 8)
              for _ in range(40)]
    for group in (shapes, [(200, 136)]):
        alone = [make(R, precision, stream, nx, ny, 100 + i, False) for i, (nx, ny) in enumerate(group)]
        batched = [make(R, precision, stream, nx, ny, 100 + i, False) for i, (nx, ny) in enumerate(group)]
        for lat in alone:
            lat.step(12)
        b = R.Batch(batched, stream=stream)
        b.step(12)
        for a, c in zip(alone, batched):
            ma, mc = a.moments(), c.moments()
            for k in range(3):
                assert np.array_equal(ma[k], mc[k])
        b.close()
        for lat in alone + batched:
            lat.close()


AHEAD, NSTEPS = 5, 70  # member 2 starts AHEAD steps later in the run; then NSTEPS batched steps


@pytest.fixture(scope="module")
def oracle_members():
    """The oracle's eps, u^x, u^y (and solid mask) of every member after its steps."""
    out = []
    for m, (nx, ny, seed, solid) in enumerate(MEMBERS):
        cfg = dict(nx=nx, ny=ny, **member_config(nx, ny, seed, solid))
        out.append((O.run(cfg, NSTEPS + (AHEAD if m == 2 else 0)), cfg.get("solid")))
    return out


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-5), ("f16", 1e-3)])
def test_batched_members_match_the_oracle(R, oracle_members, precision, tol):
    """Five members of uneven sizes, all with a body force, one with walls and discs, one AHEAD
    steps further on, advanced together by the batched launch (a captured chunk of 64
    steps and direct launches), each compared cell by cell with the FP64 oracle run of its
    own configuration: eps relative per cell, |u - u_ref| / max |u_ref| (FP64 1e-10, FP32
    1e-5, FP16 1e-3)."""
    import torch
    stream = torch.cuda.Stream()
    lats = [make(R, precision, stream, nx, ny, seed, solid) for (nx, ny, seed, solid) in MEMBERS]
    lats[2].step(AHEAD)
    b = R.Batch(lats, stream=stream)
    b.step(NSTEPS)
    for m, (lat, ((Er, UXr, UYr, _), solid)) in enumerate(zip(lats, oracle_members)):
        assert lat.current_step == NSTEPS + (AHEAD if m == 2 else 0)
        E, UX, UY, _ = lat.moments()
        fluid = np.ones(E.shape, bool) if solid is None else (np.asarray(solid) == 0)
        e_err = np.max(np.abs(E[fluid] - Er[fluid]) / Er[fluid])
        umax = max(np.abs(UXr).max(), np.abs(UYr).max())
        u_err = max(np.abs(UX - UXr).max(), np.abs(UY - UYr).max()) / umax
        print("member %d (%dx%d) %s: eps error %.2e, velocity error %.2e" % (m, lat.nx, lat.ny, precision, e_err, u_err))
        assert e_err <= tol and u_err <= tol, (m, e_err, u_err)
        if solid is not None:
            assert np.all(E[~fluid] == 0.0)
    b.close()
    for lat in lats:
        lat.close()
