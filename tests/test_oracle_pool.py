"""The host-side helpers of the full-size GPU checks (tests/oracle_pool.py): the
strip-parallel development of a whole lattice equals the oracle's whole-lattice run
bit for bit, the oracle <-> library plane mapping round-trips, and the 16-bit
quantisation equals torch's round-to-nearest conversions."""
import os

import numpy as np
import pytest

import oracle_pool as P
from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


@pytest.fixture(scope="module")
def R():
    from paper_2205_04658_gb300 import build as B
    from paper_2205_04658_gb300 import rlbm
    if not os.path.exists(rlbm.LIB_PATH):
        B.build()
    return rlbm


@pytest.fixture(scope="module", autouse=True)
def _pool():
    yield
    P.close()


@pytest.mark.parametrize("walls", [0, 1])
def test_strips_equal_the_whole_lattice(walls):
    nx, ny, n = 24, 30, 4
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=8, eps_amp=0.02, u_amp=0.05)
    mask = inputs.disc_mask(nx, ny, radius=2, fraction=0.05, seed=4, walls_y=True)[0] if walls else None
    cfg = dict(nx=nx, ny=ny, walls_y=walls, solid=mask, init_eps=e, init_ux=ux, init_uy=uy, eta_over_s=0.05,
               kmin=2, kmax=4, force_amp=1e-3, seed=5, body_force=(1e-4, 0.0))
    f, E, UX, UY = P.assemble(P.develop_async(cfg, n, nstrips=4).get(), ny)
    full = O.Oracle(cfg).run(n)
    Ef, UXf, UYf, _ = full.fields()
    ff = full.fstar
    if walls:
        ff, Ef, UXf, UYf = ff[:, 1:-1], Ef[1:-1], UXf[1:-1], UYf[1:-1]
    assert np.array_equal(f, ff)
    assert np.array_equal(E, Ef) and np.array_equal(UX, UXf) and np.array_equal(UY, UYf)


def test_blocks_equal_the_whole_lattice():
    nx, ny = 26, 18
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=9, eps_amp=0.02, u_amp=0.05)
    cfg = dict(nx=nx, ny=ny, init_eps=e, init_ux=ux, init_uy=uy, eta_over_s=0.05, kmin=2, kmax=4,
               force_amp=1e-3, seed=5)
    E, UX, UY, _ = O.run(cfg, 3)
    centres = [(0, 0), (13, 9)]
    got = P.blocks_async(cfg, 3, centres, 2).get()
    for c, (Eb, UXb, UYb) in zip(centres, got):
        for j, row in enumerate(P.block_cells(c, 2, nx, ny, 0)):
            for i, cell in enumerate(row):
                assert abs(Eb[j, i] - E[cell]) < 1e-14 and abs(UXb[j, i] - UX[cell]) < 1e-14
                assert abs(UYb[j, i] - UY[cell]) < 1e-14


def test_fold_unfold_round_trip(R):
    rng = np.random.default_rng(1)
    v, w = O.velocity_set(3)
    h = rng.normal(scale=0.1, size=(17, 5, 4))
    assert np.allclose(P.fold(R, P.unfold(R, h)), h, rtol=0, atol=1e-15)
    # a state even in v_z (the oracle's equilibria are) folds and unfolds back exactly
    e, ux, uy = inputs.smooth_random_fields(10, 9, seed=2, u_amp=0.2, kmax=2)
    f = O.equilibrium(O.ideal_T(e, O.four_velocity(ux, uy, 3), 3), v, w)
    assert np.allclose(P.unfold(R, P.fold(R, f)), f, rtol=0, atol=1e-15)


def test_quantise_matches_torch_round_to_nearest():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(scale=s, size=2000) for s in (1e-1, 1e-3, 1e-5, 3e-8)])
    for prec, dt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        ref = torch.tensor(x, dtype=torch.float32).to(dt).to(torch.float64).numpy()
        assert np.array_equal(P.quantise(x, prec), ref), prec


def test_common_start_is_representable_in_every_storage_type():
    rng = np.random.default_rng(4)
    h = np.concatenate([rng.normal(scale=s, size=5000) for s in (3e-2, 1e-4, 2e-6)])
    c = P.common_start(h)
    for prec in ("f16", "bf16", "f32"):
        assert np.array_equal(P.quantise(c, prec), c), prec
    assert np.abs(c - h).max() <= 2.0 ** -8 * np.abs(h).max()
