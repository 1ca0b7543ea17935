"""Pins of the oracle's collision: conservation of T^{0 mu} (Landau matching with
the Anderson-Witting weight, Eq. boltzmanneq_rel), relaxation of the shear
stress at rate dt/tau_R, and the hydrodynamic shear viscosity
eta = tau_R (eps + P) / 5 (Sec. "Relativistic Lattice Boltzmann")."""
import numpy as np

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def test_collision_conserves_energy_and_momentum_per_cell():
    v, w = O.velocity_set(3)
    rng = np.random.default_rng(10)
    n = 500
    eps = rng.uniform(0.5, 2.0, n)
    ux, uy = rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n)
    f = O.equilibrium(O.ideal_T(eps, O.four_velocity(ux, uy, 3), 3), v, w)
    f = f * (1.0 + 0.1 * rng.standard_normal(f.shape))
    T = O.moments(f, v)
    e, u = O.landau(T)
    dC = O.moments(O.collision(f, e, u, O.temperature(e), 0.05, 0.05, v, w), v)
    assert np.abs(dC[:, 0, :]).max() < 1e-13 * np.abs(T[:, 0, 0]).max()
    # the other components do change (the collision is not the identity)
    assert np.abs(dC[:, 1:, 1:]).max() > 1e-4


def test_plain_bgk_weight_would_not_conserve():
    """Guard on the reading of the collision weight: with p.u/p^0 replaced by 1,
    T^{0 mu} is not conserved in a moving cell (so the conservation test above
    would catch a dropped weight)."""
    v, w = O.velocity_set(3)
    rng = np.random.default_rng(11)
    eps = np.array([1.0])
    u = O.four_velocity(np.array([0.3]), np.array([-0.2]), 3)
    f = O.equilibrium(O.ideal_T(eps, u, 3), v, w) * (1.0 + 0.1 * rng.standard_normal((26, 1)))
    e, uu = O.landau(O.moments(f, v))
    feq = O.equilibrium(O.ideal_T(e, uu, 3), v, w)
    assert np.abs(O.moments(feq - f, v)[:, 0, :]).max() > 1e-4


def test_rest_frame_shear_stress_relaxes_by_dt_over_tau():
    v, w = O.velocity_set(3)
    eps = np.array([1.0, 1.7])
    u = O.four_velocity(np.zeros(2), np.zeros(2), 3)
    c = 0.03
    f = O.equilibrium(O.ideal_T(eps, u, 3), v, w) + c * (w * v[:, 0] * v[:, 1])[:, None]
    T = O.moments(f, v)
    e, uu = O.landau(T)
    assert np.allclose(e, eps, rtol=1e-14) and np.abs(uu[:, 1:]).max() < 1e-14
    dt, es = 0.05, 0.1
    Tn = O.moments(f + O.collision(f, e, uu, O.temperature(e), es, dt, v, w), v)
    tau = 5.0 * es / O.temperature(eps)
    assert np.allclose(Tn[:, 1, 2], (1.0 - dt / tau) * T[:, 1, 2], rtol=1e-13)


def test_lattice_run_conserves_totals_without_force():
    ex, ux, uy = inputs.smooth_random_fields(16, 12, seed=3, u_amp=0.1)
    cfg = dict(nx=16, ny=12, eta_over_s=0.05, init_eps=ex, init_ux=ux, init_uy=uy)
    o = O.Oracle(cfg)
    t0 = o.fields()[3]
    o.run(20)
    t1 = o.fields()[3]
    assert np.abs(t1[:3] - t0[:3]).max() < 1e-13 * t0[0]


def test_uniform_state_stays_uniform():
    cfg = dict(nx=8, ny=8, init_eps=np.full((8, 8), 1.3), init_ux=np.full((8, 8), 0.2),
               init_uy=np.full((8, 8), -0.1))
    o = O.Oracle(cfg).run(5)
    E, UX, UY, _ = o.fields()
    assert np.ptp(E) < 1e-14 and np.ptp(UX) < 1e-14 and np.ptp(UY) < 1e-14
    assert abs(E[0, 0] - 1.3) < 1e-13 and abs(UX[0, 0] - 0.2) < 1e-13


def _shear_decay_rate(eta_over_s, ny, nx=4, steps=(100, 400), amp=1e-4):
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    s = np.sin(2.0 * np.pi * y / ny)
    o = O.Oracle(dict(nx=nx, ny=ny, eta_over_s=eta_over_s, init_ux=amp * s))
    A = {}
    for n in range(steps[1] + 1):
        if n in steps:
            A[n] = (o.fields()[1] * s).sum()
        if n < steps[1]:
            o.step()
    return np.log(A[steps[0]] / A[steps[1]]) / ((steps[1] - steps[0]) * 0.05)


def test_shear_wave_viscous_slope_hydrodynamic_limit():
    """Gamma = Gamma_num + k^2 (eta/s) / T for a transverse shear wave (nu = eta/(eps+P)
    = tau_R / 5); the slope d Gamma / d(eta/s) is free of the interpolation's numerical
    viscosity.  At k tau_R ~ 0.1-0.2 (N_y = 256, a = 0.1) it must equal k^2 / T0."""
    ny = 256
    k = 2.0 * np.pi / (ny * 0.1)
    slope = (_shear_decay_rate(0.2, ny) - _shear_decay_rate(0.1, ny)) / 0.1
    assert abs(slope / (k * k / O.temperature(1.0)) - 1.0) < 0.02
