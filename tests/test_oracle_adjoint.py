"""Pins of the oracle's FP64 adjoint (oracle/rlbm_adjoint.py) against what does not
depend on it: central finite differences of the oracle's forward objective on tiny
lattices, the transpose identity of the streaming, and finite differences of Landau
matching itself."""
import numpy as np
import pytest

from oracle import rlbm_adjoint as A
from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def _fd(cfg, nsteps, key, value, h):
    cp, cm = dict(cfg), dict(cfg)
    cp[key], cm[key] = value(+h), value(-h)
    return (A.objective(cp, nsteps) - A.objective(cm, nsteps)) / (2.0 * h)


def _close(g, fd, rel):
    g, fd = np.atleast_1d(g), np.atleast_1d(fd)
    assert np.abs(g - fd).max() <= rel * np.abs(fd).max(), (g, fd)


def _stirred_cfg():
    nx, ny = 12, 10
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=3, eps_amp=0.02, u_amp=0.05, kmax=2)
    return dict(nx=nx, ny=ny, eta_over_s=0.07, kmin=2, kmax=3, force_amp=5e-3, seed=11,
                body_force=(2e-3, -1e-3), init_eps=e, init_ux=ux, init_uy=uy)


def test_stream_adjoint_is_the_transpose():
    """<stream(a), b> = <a, stream_adjoint(b)> on a window with solid cells and wall rows."""
    cfg = dict(O.DEFAULTS, nx=11, ny=9, walls_y=1)
    mask, _ = inputs.disc_mask(11, 9, radius=1, fraction=0.1, seed=4, walls_y=True)
    cfg["solid"] = mask
    win = O.Window(cfg, np.arange(11), np.arange(-1, 10))
    v, _ = O.velocity_set(3)
    opp = O.opposite(v)
    rng = np.random.default_rng(0)
    a = rng.standard_normal((26,) + win.X.shape)
    b = rng.standard_normal((26,) + win.X.shape)
    a[:, win.solid] = 0.0
    lhs = np.sum(O.stream(a, v, 0.5, win.solid, opp) * b)
    rhs = np.sum(a * A.stream_adjoint(b, v, 0.5, win.solid, opp))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(a).sum()


def test_landau_adjoint_matches_finite_differences():
    """d/dT of (eps_bar . eps + u_bar . u) along a random symmetric dT."""
    rng = np.random.default_rng(1)
    v, w = O.velocity_set(3)
    f = w[:, None] * (1.0 + 0.3 * rng.random((26, 5)))
    f[1] *= 1.8  # a drifting state
    T = O.moments(f, v)
    eps, u = O.landau(T)
    eb = rng.standard_normal(5)
    ub = rng.standard_normal((5, 4))
    ub[:, 3] = 0.0
    Tb = A.landau_adjoint(T, eps, u, eb, ub)
    dT = rng.standard_normal((5, 4, 4))
    dT = dT + np.transpose(dT, (0, 2, 1))
    dT[:, 3, :3] = dT[:, :3, 3] = 0.0  # keep the z-reflection symmetry of the state
    h = 1e-6
    ep, up = O.landau(T + h * dT)
    em, um = O.landau(T - h * dT)
    fd = ((ep - em) * eb + ((up - um) * ub).sum(axis=1)) / (2 * h)
    an = np.einsum("nmk,nmk->n", Tb, dT)
    assert np.abs(an - fd).max() <= 1e-7 * np.abs(fd).max()


def test_gradient_stirred_periodic_matches_finite_differences():
    cfg = _stirred_cfg()
    n = 6
    G = A.gradient(cfg, n)
    assert abs(G["J"] - A.objective(cfg, n)) <= 1e-14 * G["J"]
    _close(G["eta_over_s"], _fd(cfg, n, "eta_over_s", lambda h: 0.07 + h, 1e-5), 1e-6)
    for k in range(2):
        def body(h, k=k):
            b = list(cfg["body_force"])
            b[k] += h
            return tuple(b)
        _close(G["body_force"][k], _fd(cfg, n, "body_force", body, 1e-5), 1e-6)
    nm = len(O.shell_modes(2, 3))
    fds = []
    for m in range(nm):
        def scale(h, m=m):
            s = np.ones(nm)
            s[m] += h
            return s
        fds.append(_fd(cfg, n, "mode_scale", scale, 1e-4))
    _close(G["sigma"], np.array(fds), 1e-6)


def test_gradient_walls_discs_body_force_matches_finite_differences():
    nx, ny = 14, 10
    mask, _ = inputs.disc_mask(nx, ny, radius=1, fraction=0.06, seed=6, walls_y=True)
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=5, eps_amp=0.01, u_amp=0.03, kmax=2)
    cfg = dict(nx=nx, ny=ny, walls_y=1, solid=mask, eta_over_s=0.05, body_force=(3e-3, 1e-3),
               init_eps=e, init_ux=ux, init_uy=uy)
    n = 5
    G = A.gradient(cfg, n)
    _close(G["eta_over_s"], _fd(cfg, n, "eta_over_s", lambda h: 0.05 + h, 1e-5), 1e-6)
    bx = _fd(cfg, n, "body_force", lambda h: (3e-3 + h, 1e-3), 1e-5)
    by = _fd(cfg, n, "body_force", lambda h: (3e-3, 1e-3 + h), 1e-5)
    _close(G["body_force"], np.array([bx, by]), 1e-6)


def test_gradient_circle_set_eta_matches_finite_differences():
    """The eight-direction set (D_p = 2): relaxation time 4 (eta/s) / T, T = (pi eps)^(1/3)."""
    nx, ny = 10, 8
    e, ux, uy = inputs.smooth_random_fields(nx, ny, seed=8, u_amp=0.06, kmax=2)
    cfg = dict(nx=nx, ny=ny, vset=2, eta_over_s=0.09, init_eps=e, init_ux=ux, init_uy=uy)
    G = A.gradient(cfg, 5)
    _close(G["eta_over_s"], _fd(cfg, 5, "eta_over_s", lambda h: 0.09 + h, 1e-5), 1e-6)


def test_adjoint_of_the_initial_state_matches_a_directional_derivative():
    cfg = _stirred_cfg()
    n = 4
    G = A.gradient(cfg, n)
    rng = np.random.default_rng(2)
    o0 = O.Oracle(cfg)
    d = rng.standard_normal(o0.fstar.shape) * o0.w[:, None, None] * 1e-2

    def J_from(fstar0):
        o = O.Oracle(cfg)
        o.fstar = fstar0
        acc = 0.0
        for _ in range(n):
            o.step()
            acc += A._unit_obj(o, O.stream(o.fstar, o.v, o.courant, o.win.solid, o.opp))
        return acc / n

    h = 1e-4
    fd = (J_from(o0.fstar + h * d) - J_from(o0.fstar - h * d)) / (2 * h)
    an = np.sum(G["fstar0"] * d)
    assert abs(an - fd) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("bad", ["sign", "index"])
def test_planted_mistakes_are_caught(bad, monkeypatch):
    """A wrong sign in the collision weight or a transposed streaming offset in the
    adjoint makes the finite-difference pin fail."""
    cfg = _stirred_cfg()
    n = 3
    ref = _fd(cfg, n, "eta_over_s", lambda h: 0.07 + h, 1e-5)
    if bad == "sign":
        orig = A._equilibrium_adjoint
        monkeypatch.setattr(A, "_equilibrium_adjoint", lambda fb, v, w: orig(-fb, v, w))
    else:
        orig_s = A.stream_adjoint

        def swapped(fbar, v, courant, solid, opp):
            return orig_s(fbar, -v, courant, solid, opp)
        monkeypatch.setattr(A, "stream_adjoint", swapped)
    G = A.gradient(cfg, n)
    assert abs(G["eta_over_s"] - ref) > 1e-3 * abs(ref)


def test_uniform_mode_scale_equals_a_larger_amplitude():
    """sigma_m = s for every mode is the stirring of amplitude s * amp."""
    cfg = _stirred_cfg()
    nm = len(O.shell_modes(2, 3))
    a = O.run(dict(cfg, mode_scale=np.full(nm, 1.5)), 3)
    b = O.run(dict(cfg, force_amp=1.5 * cfg["force_amp"]), 3)
    for k in range(3):
        assert np.allclose(a[k], b[k], rtol=1e-14, atol=1e-16)
