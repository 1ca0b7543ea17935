"""Pins of the oracle's equilibrium, equation of state and Landau matching
(Sec. "Relativistic Lattice Boltzmann"; Sec. "Boltzmann to Lattice Boltzmann";
App. "Determination of the Equation of State")."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O


def random_states(n, seed, vmax=0.9):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.2, 3.0, n)
    speed = vmax * np.sqrt(rng.uniform(0.0, 1.0, n))
    ang = rng.uniform(0.0, 2.0 * np.pi, n)
    vx, vy = speed * np.cos(ang), speed * np.sin(ang)
    gam = 1.0 / np.sqrt(1.0 - vx * vx - vy * vy)
    return eps, gam * vx, gam * vy


@pytest.mark.parametrize("vs", [2, 3])
def test_equilibrium_reproduces_ideal_stress_energy(vs):
    v, w = O.velocity_set(vs)
    dp = v.shape[1]
    eps, ux, uy = random_states(200, 1)
    u = O.four_velocity(ux, uy, dp)
    Teq = O.ideal_T(eps, u, dp)
    feq = O.equilibrium(Teq, v, w)
    assert np.abs(O.moments(feq, v) - Teq).max() < 1e-13


@pytest.mark.parametrize("vs", [2, 3])
def test_rest_frame_matrix_and_pressure(vs):
    """At rest T^{mu nu} = diag(eps, P, P[, P]) with P = eps / D_p: the paper's EOS
    P = eps/3 for its three-dimensional momentum set, P = eps/2 for the circle set."""
    v, w = O.velocity_set(vs)
    dp = v.shape[1]
    eps = np.array([0.7, 1.0, 2.5])
    u = O.four_velocity(np.zeros(3), np.zeros(3), dp)
    T = O.moments(O.equilibrium(O.ideal_T(eps, u, dp), v, w), v)
    for n in range(3):
        assert np.abs(T[n] - np.diag([eps[n]] + [eps[n] / dp] * dp)).max() < 1e-15
    # equivalently: T^{mu nu} g_{mu nu} = 0 for massless particles
    assert np.abs(np.einsum("nmk,mk->n", T, O.metric(dp))).max() < 1e-15


@pytest.mark.parametrize("vs", [2, 3])
def test_ideal_T_is_traceless_in_motion(vs):
    dp = 3 if vs == 3 else 2
    eps, ux, uy = random_states(100, 2)
    T = O.ideal_T(eps, O.four_velocity(ux, uy, dp), dp)
    assert np.abs(np.einsum("nmk,mk->n", T, O.metric(dp))).max() < 1e-12


@pytest.mark.parametrize("vs", [2, 3])
def test_landau_round_trip_on_equilibrium(vs):
    v, w = O.velocity_set(vs)
    dp = v.shape[1]
    eps, ux, uy = random_states(300, 3)
    u = O.four_velocity(ux, uy, dp)
    T = O.moments(O.equilibrium(O.ideal_T(eps, u, dp), v, w), v)
    e2, u2 = O.landau(T)
    assert np.abs(e2 / eps - 1.0).max() < 1e-13
    assert np.abs(u2 - u).max() < 1e-12


def charpoly_largest_root(M):
    """Largest real root of det(M - lam I) by bisection, with the determinant
    expanded by cofactors (no eigen-solver)."""
    def det(A):
        if A.shape[0] == 1:
            return A[0, 0]
        return sum((-1) ** j * A[0, j] * det(np.delete(np.delete(A, 0, 0), j, 1))
                   for j in range(A.shape[0]))

    n = M.shape[0]
    bound = np.abs(M).sum()
    lo, hi = -bound, bound
    # the largest root: det(M - lam I) has sign (-1)^n for lam > largest root
    sgn_hi = (-1) ** n
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.sign(det(M - mid * np.eye(n))) == sgn_hi:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_landau_on_non_equilibrium_states_matches_second_solver():
    """Non-equilibrium populations: the oracle's eps is the largest root of the
    characteristic polynomial of T^mu_nu, and u_mu T^{mu nu} = eps u^nu holds."""
    v, w = O.velocity_set(3)
    rng = np.random.default_rng(4)
    eps, ux, uy = random_states(40, 5, vmax=0.6)
    u = O.four_velocity(ux, uy, 3)
    f = O.equilibrium(O.ideal_T(eps, u, 3), v, w)
    f = f * (1.0 + 0.2 * rng.standard_normal(f.shape))
    T = O.moments(f, v)
    e2, u2 = O.landau(T)
    g = O.metric(3)
    resid = np.einsum("nm,mk,nkl->nl", u2, g, T) - e2[:, None] * u2
    assert np.abs(resid).max() < 1e-13 * np.abs(T).max()
    assert np.abs(np.einsum("nm,mk,nk->n", u2, g, u2) - 1.0).max() < 1e-13
    assert np.all(u2[:, 0] > 0)
    for n in range(0, 40, 5):
        assert abs(charpoly_largest_root(T[n] @ g) - e2[n]) < 1e-10 * e2[n]


def test_landau_rejects_spacelike_momentum():
    v, w = O.velocity_set(3)
    px = int(np.argmax(v[:, 0]))
    mx = int(np.argmin(v[:, 0]))
    f = np.zeros((26, 1))
    f[px, 0] = 1.0  # a single beam: T^{mu nu} is null, no timelike eigenvector with eps > 0
    with pytest.raises(FloatingPointError):
        O.landau(O.moments(f, v))
    f[mx, 0] = -0.5  # momentum exceeds energy (negative population): spacelike flow
    with pytest.raises(FloatingPointError):
        O.landau(O.moments(f, v))


def test_temperature_and_relaxation_time():
    """eps = 3 T^4 / pi^2 and tau_R = 5 (eta/s) / T (Sec. "Relativistic Lattice
    Boltzmann"; Sec. "Boltzmann to Lattice Boltzmann")."""
    T = O.temperature(np.array([1.0, 2.0]))
    assert np.allclose(3.0 * T ** 4 / np.pi ** 2, [1.0, 2.0], rtol=1e-15)
    assert abs(O.temperature(1.0) - 1.3467736870885985) < 1e-15
    assert np.allclose(O.relaxation_time(T, 0.1), 0.5 / T, rtol=1e-15)
