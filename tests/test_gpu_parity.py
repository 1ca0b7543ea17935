"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances: FP64 <= 1e-10 and FP32 <= 1e-5 in eps (relative, per
cell) and in u (|du| relative to max |u| of the reference), after up to 200 steps."""
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


def gpu_run(R, cfg, nsteps, precision):
    kw = {k: v for k, v in cfg.items()}
    lat = R.Lattice(cfg["nx"], cfg["ny"], precision=precision, **{k: v for k, v in kw.items() if k not in ("nx", "ny")})
    lat.step(nsteps)
    out = lat.moments()
    assert lat.current_step == nsteps
    lat.close()
    return out


def errors(gpu, ref, solid=None):
    E, UX, UY = gpu[:3]
    Er, UXr, UYr = ref[:3]
    fluid = np.ones(E.shape, bool) if solid is None else (np.asarray(solid) == 0)
    e_err = np.max(np.abs(E[fluid] - Er[fluid]) / Er[fluid])
    umax = max(np.abs(UXr).max(), np.abs(UYr).max())
    u_err = max(np.abs(UX - UXr).max(), np.abs(UY - UYr).max()) / umax
    return e_err, u_err


def test_shear_wave_64_fp64_200_steps(R):
    e, ux, uy = inputs.shear_wave(64, 64, 0.01)
    cfg = dict(nx=64, ny=64, eta_over_s=0.1, init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 200)
    gpu = gpu_run(R, cfg, 200, "f64")
    ee, ue = errors(gpu, ref)
    assert ee <= TOL["f64"] and ue <= TOL["f64"], (ee, ue)
    assert np.abs(gpu[3] - ref[3]).max() <= 1e-10 * abs(ref[3][0])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_stirred_ragged_lattice(R, precision):
    """100 x 76 (ragged against the 32 x 8 tile), stirring shell 2 <= |k| <= 5,
    smooth random initial flow, 200 steps (FP64) / 200 steps (FP32)."""
    nx, ny = 100, 76
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=7, eps_amp=0.02, u_amp=0.03)
    cfg = dict(nx=nx, ny=ny, eta_over_s=0.05, kmin=2, kmax=5, force_amp=2e-3, seed=12345,
               init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 200)
    gpu = gpu_run(R, cfg, 200, precision)
    ee, ue = errors(gpu, ref)
    assert ee <= TOL[precision] and ue <= TOL[precision], (ee, ue)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_smallest_lattices_and_zero_steps(R, precision):
    """The smallest accepted lattices, narrower than one 32 x 8 tile: 8 x 8 periodic and
    8 x 13 between walls (one full and one partial tile row), stirred 1 <= |k| <= 3, after
    0 steps (rlbm_step(0) queues nothing), 1 step and 40 steps."""
    for nx, ny, walls in ((8, 8, 0), (8, 13, 1)):
        e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=nx * ny, eps_amp=0.02, u_amp=0.04, kmax=2)
        cfg = dict(nx=nx, ny=ny, walls_y=walls, eta_over_s=0.05, kmin=1, kmax=3, force_amp=1e-2, seed=6,
                   init_eps=e, init_ux=ux, init_uy=uy)
        for n in (0, 1, 40):
            ref = O.run(cfg, n)
            gpu = gpu_run(R, cfg, n, precision)
            ee, ue = errors(gpu, ref)
            assert ee <= TOL[precision] and ue <= TOL[precision], (nx, ny, n, ee, ue)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_walls_discs_body_force(R, precision):
    nx, ny = 72, 40
    mask, _ = inputs.disc_mask(nx, ny, radius=3, fraction=0.08, seed=31, walls_y=True)
    cfg = dict(nx=nx, ny=ny, walls_y=1, solid=mask, body_force=(2e-4, -5e-5), eta_over_s=0.05)
    ref = O.run(cfg, 150)
    gpu = gpu_run(R, cfg, 150, precision)
    ee, ue = errors(gpu, ref, mask)
    assert ee <= TOL[precision] and ue <= TOL[precision], (ee, ue)
    assert np.all(gpu[0][mask != 0] == 0.0)


def test_circle_set_fp64(R):
    nx, ny = 40, 24
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=3, u_amp=0.05)
    cfg = dict(nx=nx, ny=ny, vset=2, eta_over_s=0.08, init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 100)
    gpu = gpu_run(R, cfg, 100, "f64")
    ee, ue = errors(gpu, ref)
    assert ee <= 1e-10 and ue <= 1e-10, (ee, ue)


def test_large_velocity_fp32_uses_fp64_landau(R):
    """|v| up to ~0.6: the FP32 path re-solves Landau matching in FP64 above |v| = 0.5."""
    nx, ny = 48, 32
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=5, u_amp=0.75, kmax=2)
    cfg = dict(nx=nx, ny=ny, eta_over_s=0.1, init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 40)
    gpu = gpu_run(R, cfg, 40, "f32")
    ee, ue = errors(gpu, ref)
    assert ee <= 1e-5 and ue <= 1e-5, (ee, ue)


def test_conservation_without_force_fp64(R):
    nx, ny = 64, 48
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=9, u_amp=0.1)
    lat = R.Lattice(nx, ny, precision="f64", eta_over_s=0.05, init_eps=e, init_ux=ux, init_uy=uy)
    t0 = lat.totals()
    lat.step(300)
    t1 = lat.totals()
    lat.close()
    assert np.abs(t1[:3] - t0[:3]).max() <= 1e-12 * t0[0]


def test_spectrum_matches_oracle(R):
    nx, ny = 48, 40
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=11, u_amp=0.05, kmax=6)
    cfg = dict(nx=nx, ny=ny, eta_over_s=0.05, kmin=3, kmax=6, force_amp=1e-3, seed=4,
               init_eps=e, init_ux=ux, init_uy=uy)
    o = O.Oracle(cfg).run(30)
    E, UX, UY, _ = o.fields()
    ref = O.spectrum(UX, UY, 40)
    kw = {k: v for k, v in cfg.items() if k not in ("nx", "ny")}
    lat = R.Lattice(nx, ny, precision="f64", **kw)
    lat.step(30)
    got = lat.spectrum(40)
    lat.close()
    assert np.abs(got - ref).max() <= 1e-10 * ref.max()
    # bins beyond the lattice's largest |k| are zero
    lat = R.Lattice(16, 16, precision="f64", **{k: v for k, v in kw.items() if not k.startswith("init")
                                                  and k not in ("kmin", "kmax", "force_amp")})
    assert np.all(lat.spectrum(40)[13:] == 0.0)
    lat.close()


def test_band_energy_matches_oracle(R):
    """The velocity filter (energy of the wave vectors below the stirring shell) and its
    complement, on a stirred state after 30 steps, against the oracle's band energy."""
    nx, ny = 48, 40
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=17, u_amp=0.05, kmax=6)
    cfg = dict(nx=nx, ny=ny, eta_over_s=0.05, kmin=3, kmax=6, force_amp=1e-3, seed=4,
               init_eps=e, init_ux=ux, init_uy=uy)
    o = O.Oracle(cfg).run(30)
    E, UX, UY, _ = o.fields()
    lat = R.Lattice(nx, ny, precision="f64", **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    lat.step(30)
    for lo, hi in ((0, 9), (9, 0), (0, 0), (10, 37)):
        ref = O.band_energy(UX, UY, lo, hi)
        assert abs(lat.band_energy(lo, hi) - ref) <= 1e-10 * O.band_energy(UX, UY, 0, 0)
    assert lat.filtered_velocity(3) == pytest.approx(np.sqrt(2 * O.band_energy(UX, UY, 0, 9)), rel=1e-9)
    lat.close()


def test_spectrum_non_power_of_two_sizes(R):
    """768 = 3 * 2^8 and 90 = 2 * 3^2 * 5 exercise the mixed-radix transform."""
    for nx, ny in ((768, 24), (90, 26)):
        e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=nx, u_amp=0.05, kmax=5)
        lat = R.Lattice(nx, ny, precision="f64", init_eps=e, init_ux=ux, init_uy=uy)
        _, UX, UY, _ = lat.moments()
        got = lat.spectrum(60)
        lat.close()
        ref = O.spectrum(UX, UY, 60)
        assert np.abs(got - ref).max() <= 1e-12 * ref.max()


def test_resume_from_state_is_bit_exact(R):
    nx, ny = 64, 40
    kw = dict(eta_over_s=0.05, kmin=2, kmax=4, force_amp=1e-3, seed=77)
    a = R.Lattice(nx, ny, precision="f32", **kw)
    a.step(20)
    ref = a.moments()
    a.close()
    b = R.Lattice(nx, ny, precision="f32", **kw)
    b.step(9)
    h, step = b.get_state()
    b.close()
    assert step == 9 and h.shape == (17, ny, nx)
    c = R.Lattice(nx, ny, precision="f32", **kw)
    c.set_state(h, step)
    c.step(11)
    got = c.moments()
    assert c.current_step == 20
    c.close()
    for k in range(3):
        assert np.array_equal(got[k], ref[k])


def test_unstable_state_is_reported_then_context_is_locked(R):
    lat = R.Lattice(32, 32, precision="f32", eta_over_s=0.1)
    h, step = lat.get_state()
    h[3, 5, 7] = np.nan
    lat.set_state(h, step)
    lat.step(2)
    with pytest.raises(R.RlbmError) as e:
        lat.sync()
    assert e.value.status == R.RLBM_E_UNSTABLE
    with pytest.raises(R.RlbmError) as e:
        lat.step(1)
    assert e.value.status == R.RLBM_E_STATE
    lat.close()


def test_expired_bounded_wait_is_reported_then_context_is_locked(R):
    """A bounded device wait that runs out (an mbarrier that nothing arrives on, about 1 ms)
    is reported as RLBM_E_TIMEOUT by the next syncing call; the context then refuses work,
    and the device stays usable for a new context."""
    lat = R.Lattice(64, 32, precision="f32", eta_over_s=0.05, kmin=2, kmax=4, force_amp=1e-3, seed=3)
    lat.step(3)
    lat.sync()
    R.rlbm_wait_selftest(lat.ctx, 2_000_000)
    with pytest.raises(R.RlbmError) as e:
        lat.sync()
    assert e.value.status == R.RLBM_E_TIMEOUT and "wait expired" in str(e.value)
    with pytest.raises(R.RlbmError) as e:
        lat.step(1)
    assert e.value.status == R.RLBM_E_STATE
    lat.close()
    fresh = R.Lattice(64, 32, precision="f32", eta_over_s=0.05)
    fresh.step(3)
    fresh.sync()
    assert fresh.current_step == 3
    fresh.close()


def _sampled_check(R, nx, ny, nsteps, precision, npts, seed):
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=seed, eps_amp=0.02, u_amp=0.03, kmax=8)
    cfg = dict(nx=nx, ny=ny, eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4, seed=2,
               init_eps=e, init_ux=ux, init_uy=uy)
    gpu = gpu_run(R, cfg, nsteps, precision)
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0)] + \
          [(int(rng.integers(nx)), int(rng.integers(ny))) for _ in range(npts)]
    ref = O.run_sampled(cfg, nsteps, pts)
    umax = max(np.abs(ux).max(), np.abs(uy).max())
    for (x, y), r in zip(pts, ref):
        assert abs(gpu[0][y, x] - r[0]) <= TOL[precision] * r[0]
        assert abs(gpu[1][y, x] - r[1]) <= TOL[precision] * umax
        assert abs(gpu[2][y, x] - r[2]) <= TOL[precision] * umax


def test_full_size_1024_fp32_sampled(R):
    """The benchmark's workload shape (1024^2, FP32, stirring 8 <= |k| <= 10), checked
    at sampled cells after 3 steps (the oracle evaluates each sample on its own window)."""
    _sampled_check(R, 1024, 1024, 3, "f32", 24, 1)


def test_maximum_size_4096_fp32_sampled(R):
    _sampled_check(R, 4096, 4096, 2, "f32", 12, 2)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_maximum_width_ragged_height_sampled(R, precision):
    """The largest lattice width the library accepts (32768) with a height that leaves a
    partial last tile row (4100 = 512 x 8 + 4): 17 planes of about 32768 x 4102 padded
    cells put the later planes at element offsets beyond 2^31, so every index on the
    path has to be 64-bit.  Sampled cells include the four corners."""
    _sampled_check(R, 32768, 4100, 2, precision, 12, 3)


def test_launch_shapes_give_identical_results(R):
    """The launch shape (pipeline depth, CTA count) and the autotuner change nothing in
    the results: every cell is computed by the same arithmetic wherever it runs."""
    nx, ny = 160, 72
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=21, u_amp=0.03)
    kw = dict(eta_over_s=0.05, kmin=3, kmax=6, force_amp=1e-3, seed=8, init_eps=e, init_ux=ux, init_uy=uy)
    outs = []
    for shape in ((0, 2, 1), (0, 1, 1), (7, 2, 1), (3, 1, 1), (0, 2, 2), (5, 1, 2), None):
        lat = R.Lattice(nx, ny, precision="f32", **kw)
        if shape is None:
            assert lat.autotune(3) > 0
        else:
            lat.set_launch(*shape)
        lat.step(25)
        outs.append(lat.moments())
        assert lat.current_step == 25
        lat.close()
    for o in outs[1:]:
        for k in range(3):
            assert np.array_equal(o[k], outs[0][k])


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_chained_steps_match_single_steps(R, precision):
    """Steps 2..N of one rlbm_step(N) call are chained (programmatic dependent launch);
    the state is bit-identical to N calls of one step each, for lattices where a CTA takes
    one tile and where it takes many."""
    for nx, ny, shape in ((96, 40, (0, 2, 1)), (512, 256, (0, 2, 1)), (512, 256, (0, 1, 1))):
        kw = dict(eta_over_s=0.05, kmin=3, kmax=6, force_amp=1e-3, seed=9)
        states = []
        for single in (False, True):
            lat = R.Lattice(nx, ny, precision=precision, **kw)
            lat.set_launch(*shape)
            if single:
                for _ in range(30):
                    lat.step(1)
            else:
                lat.step(30)
            h, step = lat.get_state()
            assert step == 30
            states.append(h)
            lat.close()
        assert np.array_equal(states[0], states[1])


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 2e-6)])
def test_totals_match_oracle_with_walls_and_discs(R, precision, tol):
    """Totals (sum T^00, T^0x, T^0y over fluid cells, 1/2 sum |v|^2) on a ragged lattice with
    walls, discs and a body force.  FP32 states take them as FP32 deviation sums per warp
    added in FP64 to the exact count of fluid cells; FP64 states sum in FP64."""
    nx, ny = 72, 40
    mask, _ = inputs.disc_mask(nx, ny, radius=2, fraction=0.08, seed=3, walls_y=True)
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=12, eps_amp=0.02, u_amp=0.04, kmax=3)
    cfg = dict(nx=nx, ny=ny, walls_y=1, solid=mask, eta_over_s=0.05, body_force=(2e-3, -1e-3),
               kmin=2, kmax=4, force_amp=1e-3, seed=6, init_eps=e, init_ux=ux, init_uy=uy)
    ref = O.run(cfg, 30)[3]
    lat = R.Lattice(nx, ny, precision=precision, **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    lat.step(30)
    tot = lat.totals()
    lat.close()
    assert abs(tot[0] - ref[0]) <= tol * ref[0], (tot[0], ref[0])
    assert np.abs(tot[1:3] - ref[1:3]).max() <= tol * ref[0], (tot[1:3], ref[1:3])
    assert abs(tot[3] - ref[3]) <= (1e-9 if precision == "f64" else 1e-4) * ref[3], (tot[3], ref[3])
