"""Plain FP64 CPU adjoint of the oracle's update: the gradient of a kinetic-energy
objective of a stirred run with respect to the per-mode amplitude multipliers
sigma_m, the ratio eta/s and the uniform body force.

TEST INFRASTRUCTURE ONLY, like `rlbm_oracle`: the tests may import it; nothing on
the product path does.  It shares no code with the CUDA library.

Objective (the paper defines none; this is the reading used throughout the
repository): the time average over the states after steps 1 .. N of the cell mean of
the kinetic energy per unit energy density,

    J = (1/N) sum_{n=1}^{N} (1/N_fluid) sum_x 1/2 |v_n(x)|^2,   v = u^i / u^0,

with u^mu of f_n = stream(f*_n) from Landau matching.  The stirring amplitude of mode
m at every step is sigma_m a_m (Sec. "The Driving Term", last paragraph, with a
multiplier per mode).

Method: reverse-mode differentiation of the oracle's own step, written out by hand
in the oracle's variables (all 26 unfolded directions, the (1 + D_p) x (1 + D_p)
energy-momentum tensor):

  * streaming is linear; its adjoint is the transpose of the pull (a push with the
    same bilinear weights; a bounce-back substitution sends the adjoint back to the
    reversed population of the receiving cell);
  * moments, equilibrium (Eq. rel_pdf_exp_coef), the Anderson-Witting collision
    (Eq. boltzmanneq_rel) and the projected force (Eq. forceTerm, App. B) are
    differentiated term by term;
  * Landau matching T^mu_nu u^nu = eps u^mu with u.u = 1 is differentiated
    implicitly: (T^mu_nu - eps delta) du - u deps = -dT^mu_nu u and u_mu du^mu = 0
    form a bordered (2 + D_p) x (2 + D_p) system; its transpose carries the adjoints
    of eps and u back to T^{mu nu}.

All states f*_0 .. f*_N are kept (the oracle runs small lattices only).
"""
import numpy as np

from . import rlbm_oracle as O


def _unit_obj(o, f):
    """Cell mean of 1/2 |v|^2 of the post-streaming state f over the fluid cells."""
    fluid, T, eps, u = o.macroscopic(f)
    v = u[:, 1:3] / u[:, :1]
    return 0.5 * (v * v).sum(axis=1).mean()


def objective(cfg, nsteps):
    """J of the module docstring by a plain forward run."""
    o = O.Oracle(cfg)
    acc = 0.0
    for _ in range(nsteps):
        o.step()
        f = O.stream(o.fstar, o.v, o.courant, o.win.solid, o.opp)
        acc += _unit_obj(o, f)
    return acc / nsteps


def stream_adjoint(fbar, v, courant, solid, opp):
    """Transpose of `rlbm_oracle.stream`: <stream(a), b> = <a, stream_adjoint(b)>."""
    fb = fbar.copy()
    fb[:, solid] = 0.0
    out = np.zeros_like(fb)
    for i in range(v.shape[0]):
        dx, dy = courant * v[i, 0], courant * v[i, 1]
        sx, sy = int(np.sign(dx)), int(np.sign(dy))
        ax, ay = abs(dx), abs(dy)
        for (ox, oy), beta in (((0, 0), (1 - ax) * (1 - ay)), ((sx, 0), ax * (1 - ay)),
                               ((0, sy), (1 - ax) * ay), ((sx, sy), ax * ay)):
            if beta == 0.0:
                continue
            src_solid = np.roll(solid, (oy, ox), axis=(0, 1))
            gi = beta * fb[i]
            out[opp[i]] += np.where(src_solid, gi, 0.0)
            out[i] += np.roll(np.where(src_solid, 0.0, gi), (-oy, -ox), axis=(0, 1))
    return out


def landau_adjoint(T, eps, u, eps_bar, u_bar):
    """Adjoint of Landau matching: given the adjoints of eps (N,) and u^mu (N, D) at the
    solution, the adjoint of T^{mu nu} (N, D, D) through the bordered system

        [ T g - eps I   -u ] [du  ]   [ -dT g u ]
        [ (g u)^T        0 ] [deps] = [    0    ]."""
    n, d, _ = T.shape
    g = O.metric(d - 1)
    gu = u @ g
    A = np.zeros((n, d + 1, d + 1))
    A[:, :d, :d] = T @ g - eps[:, None, None] * np.eye(d)
    A[:, :d, d] = -u
    A[:, d, :d] = gu
    rhs = np.concatenate([u_bar, eps_bar[:, None]], axis=1)
    z = np.linalg.solve(np.transpose(A, (0, 2, 1)), rhs[..., None])[..., 0]
    a = z[:, :d]
    # dL = -a^T dT g u  =>  dL/dT_{mu lam} = -a_mu (g u)_lam
    return -a[:, :, None] * gu[:, None, :]


def _equilibrium_adjoint(feq_bar, v, w):
    """Adjoint of `equilibrium` with respect to T_eq (linear map): (Q, N) -> (N, D, D)."""
    q, dp = v.shape
    c2 = dp * (dp + 2) / 2.0
    n = feq_bar.shape[1]
    Tb = np.zeros((n, dp + 1, dp + 1))
    for i in range(q):
        P2 = np.outer(v[i], v[i]) - np.eye(dp) / dp
        gi = w[i] * feq_bar[i]
        Tb[:, 0, 0] += gi * (1.0 - c2 / dp * np.trace(P2))
        Tb[:, 0, 1:] += gi[:, None] * (dp * v[i])[None, :]
        Tb[:, 1:, 1:] += gi[:, None, None] * (c2 * P2)[None, :, :]
    return Tb


def _ideal_T_adjoint(Teq_bar, eps, u, dp):
    """Adjoints of eps and u^mu from that of T_eq = (eps + P) u u - P g, P = eps / D_p."""
    g = O.metric(dp)
    k = 1.0 + 1.0 / dp
    eps_bar = np.einsum("nmk,nmk->n", Teq_bar, k * u[:, :, None] * u[:, None, :] - g[None] / dp)
    sym = Teq_bar + np.transpose(Teq_bar, (0, 2, 1))
    u_bar = k * eps[:, None] * np.einsum("nmk,nk->nm", sym, u)
    return eps_bar, u_bar


def _force_adjoint(f, F, v, w, T0, s_bar):
    """Adjoints of f (Q, N) and F (N, 2) of S(f, F) of `force_source`, given that of S."""
    q = v.shape[0]
    F3 = np.concatenate([F, np.zeros(F.shape[:-1] + (1,))], axis=-1)
    M0 = f.sum(axis=0)
    M1 = np.einsum("qn,qj->nj", f, v)
    Fv = np.einsum("nj,qj->qn", F3, v)
    c = -(6.0 / T0) * w[:, None] * s_bar                  # adjoint of each bracket
    M0_bar = np.zeros_like(M0)
    M1_bar = np.zeros_like(M1)
    B_bar = np.zeros(M1.shape + (3,))
    Fv_bar = np.zeros_like(Fv)
    F3_bar = np.zeros_like(F3)
    for i in range(q):
        ci = c[i]
        vM1 = M1 @ v[i]
        # bracket_i = 1/4 F.M1 - 1/2 Fv_i M0 + 5/4 v_i.B.v_i - 5/2 Fv_i (v_i.M1)
        M1_bar += ci[:, None] * (0.25 * F3 - 2.5 * Fv[i][:, None] * v[i][None, :])
        F3_bar += ci[:, None] * 0.25 * M1
        M0_bar += ci * (-0.5 * Fv[i])
        Fv_bar[i] += ci * (-0.5 * M0 - 2.5 * vM1)
        B_bar += ci[:, None, None] * 1.25 * np.outer(v[i], v[i])[None]
    f_bar = np.zeros_like(f)
    for l in range(q):
        vBv = np.einsum("njk,j,k->n", B_bar, v[l], v[l])
        f_bar[l] += Fv[l] * vBv + M0_bar + M1_bar @ v[l]
        Fv_bar[l] += f[l] * vBv
    F3_bar += np.einsum("qn,qj->nj", Fv_bar, v)
    return f_bar, F3_bar[:, :2]


def _mode_projection(o, Fbar_full, n):
    """d/d sigma_m of sum_x Fbar(x) . F_n(x): the stirring field of mode m at unit
    multiplier, projected on the adjoint of the force.  Fbar_full: (H, W, 2)."""
    c = o.cfg
    a, phi, psi = O.mode_draws(c["seed"], n, len(o.modes), c["force_amp"])
    X, Y = o.win.X, o.win.Y
    out = np.empty(len(o.modes))
    for m, (kx, ky) in enumerate(o.modes):
        cm = a[m] * np.cos(2.0 * O.PI * (kx * X / c["nx"] + ky * Y / c["ny"]) + phi[m])
        out[m] = (Fbar_full[..., 0] * np.cos(psi[m]) * cm + Fbar_full[..., 1] * np.sin(psi[m]) * cm).sum()
    return out


def gradient(cfg, nsteps):
    """J and its gradient: returns dict(J, sigma (nmodes,), eta_over_s, body_force (2,),
    fstar0 (the adjoint of the initial post-collision state, (Q, H, W)))."""
    o = O.Oracle(cfg)
    c = o.cfg
    v, w, opp = o.v, o.w, o.opp
    dp = o.dp
    fstars = [o.fstar.copy()]
    for _ in range(nsteps):
        o.step()
        fstars.append(o.fstar.copy())
    nfluid = int((~o.win.solid).sum())
    cj = 1.0 / (nsteps * nfluid)
    needs_force = bool(o.modes) or c["body_force"][0] != 0.0 or c["body_force"][1] != 0.0

    g_sigma = np.zeros(len(o.modes))
    g_eta = 0.0
    g_body = np.zeros(2)
    J = 0.0
    lam = None  # adjoint of f*_{n+1}
    for n in range(nsteps, -1, -1):
        f = O.stream(fstars[n], v, o.courant, o.win.solid, opp)
        fluid, T, eps, u = o.macroscopic(f)
        ff = f[:, fluid]
        f_bar = np.zeros_like(ff)
        eps_bar = np.zeros_like(eps)
        u_bar = np.zeros_like(u)
        T_bar = np.zeros_like(T)
        if n >= 1:  # objective term of the state after step n
            vv = u[:, 1:3] / u[:, :1]
            J += cj * 0.5 * (vv * vv).sum()
            vbar = cj * vv
            u_bar[:, 1:3] += vbar / u[:, :1]
            u_bar[:, 0] += -(vbar * vv).sum(axis=1) / u[:, 0]
        if lam is not None:  # step n: f*_{n+1} = f_n + dt C[f_n] + dt S_n[f_n]
            lf = lam[:, fluid]
            f_bar += lf
            Tl = O.temperature(eps, c["vset"])
            tau = O.relaxation_time(Tl, c["eta_over_s"], c["vset"])
            om = c["dt"] / tau
            feq = O.equilibrium(O.ideal_T(eps, u, dp), v, w)
            om_bar = np.zeros_like(eps)
            feq_bar = np.zeros_like(feq)
            for i in range(v.shape[0]):
                pu = u[:, 0] - u[:, 1:] @ v[i]
                d = feq[i] - ff[i]
                om_bar += lf[i] * pu * d
                pu_bar = lf[i] * om * d
                u_bar[:, 0] += pu_bar
                u_bar[:, 1:] -= pu_bar[:, None] * v[i][None, :]
                feq_bar[i] = lf[i] * om * pu
                f_bar[i] -= lf[i] * om * pu
            # om = dt T / (K eta/s);  T = (pi^2 eps / 3)^(1/4)  (D_p = 3)  or  (pi eps)^(1/3)
            T_l_bar = om_bar * om / Tl
            g_eta += -(om_bar * om).sum() / c["eta_over_s"]
            eps_bar += T_l_bar * Tl / (4.0 * eps if c["vset"] == 3 else 3.0 * eps)
            Teq_bar = _equilibrium_adjoint(feq_bar, v, w)
            e_b, u_b = _ideal_T_adjoint(Teq_bar, eps, u, dp)
            eps_bar += e_b
            u_bar += u_b
            if needs_force:
                F = o.force_field(n)[fluid]
                fb, Fb = _force_adjoint(ff, F, v, w, o.T0, c["dt"] * lf)
                f_bar += fb
                g_body += Fb.sum(axis=0)
                if o.modes:
                    full = np.zeros(o.win.X.shape + (2,))
                    full[fluid] = Fb
                    g_sigma += _mode_projection(o, full, n)
        T_bar += landau_adjoint(T, eps, u, eps_bar, u_bar)
        p = np.concatenate([np.ones((v.shape[0], 1)), v], axis=1)
        f_bar += np.einsum("nmk,qm,qk->qn", T_bar, p, p)
        full = np.zeros_like(fstars[n])
        full[:, fluid] = f_bar
        lam = stream_adjoint(full, v, o.courant, o.win.solid, opp)
    return dict(J=J, sigma=g_sigma, eta_over_s=g_eta, body_force=g_body, fstar0=lam)
