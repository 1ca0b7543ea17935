"""Plain FP64 CPU oracle of the relativistic lattice Boltzmann update of
M. Watson, "Turbulence in two-dimensional relativistic hydrodynamic systems
with a lattice Boltzmann model" (arXiv 2205.04658).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the timed CPU
baseline of the benchmark may import this module; nothing on the product path
does.  It shares no code, table or constant generator with the CUDA library
(the library builds its own velocity set, force tables and FFT).

What it computes, step by step, in the paper's order (Sec. "The Standard/
Classical LBM", enumerated procedure; Sec. "The Driving Term", last paragraph):

    f*_0 = f_eq(initial eps, u)                              (procedure, item 1)
    for n = 0, 1, ...:
        f_n   = stream(f*_n)          bilinear pull, bounce-back      (item 2)
        T^{mu nu}(f_n), Landau matching -> eps, u^mu, T, tau_R         (item 3)
        f_eq  from eps, u^mu                                           (item 4)
        f*_{n+1} = f_n + dt C[f_n] + dt S_n[f_n]                       (item 5)

"The state after n steps" is f_n = stream(f*_n); its moments are the reported
macroscopic fields.  The stirring force of step n is drawn with counter n.

Everything is float64, vectorised over lattice cells with explicit loops over
the discrete momenta.  The 26 directions of the paper's spherical set are all
kept (no folding of the v_z -> -v_z symmetry), and Landau matching is a
generic eigen-decomposition of the full (1+D_p) x (1+D_p) matrix T^mu_nu, so
the reductions the CUDA path makes are checked, not shared.

Readings of points the paper leaves open (each is listed with its reason in
the design notes of the repository):
  * velocity set: 26 unit vectors along the D3Q27 neighbour directions with the
    degree-7 spherical weights 1/21, 4/105, 9/280 (axis, edge, corner); the
    27th slot of "D3Q27" is the empty rest slot of a massless gas.  A second
    set, 8 directions on the unit circle with weights 1/8 (D_p = 2,
    P = eps/2), is built for the two-dimensional equation-of-state check.
  * T_eq = (eps + P) u u - P g with g = diag(+1, -1, -1, -1) (the rest-frame
    matrix of App. "Determination of the Equation of State" fixes the sign).
  * collision weight p.u / p^0 = u^0 - v.u (Anderson-Witting form of
    Eq. boltzmanneq_rel), explicit Euler in time.
  * force source: the bracket of Eq. forceTerm with the energy-weighted
    population moments and prefactor -6/T0, sign fixed so that a uniform force
    pushes the fluid along +F.
  * streaming: bilinear pull from x - (dt/a) v_parallel, bounce-back by
    substituting the reversed population of the receiving cell for each solid
    source corner.
"""
import numpy as np

PI = np.pi


# --------------------------------------------------------------------------
# Discrete momentum set (Sec. "Boltzmann to Lattice Boltzmann"; Part I,
# "Model and Methods": spherical D3Q27 set on a lattice one node thick in z).
# --------------------------------------------------------------------------
def velocity_set(vset=3):
    """Unit momentum directions v_i (Q x D_p) and quadrature weights w_i.

    vset=3: the 26 directions (a, b, c)/|(a, b, c)|, a, b, c in {-1, 0, 1},
            weights 1/21 (axis), 4/105 (edge), 9/280 (corner).
    vset=2: 8 directions at angles j*pi/4, weights 1/8.
    """
    if vset == 3:
        dirs = np.array([(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1)
                         for a in (-1, 0, 1) if (a, b, c) != (0, 0, 0)], dtype=np.float64)
        nnz = np.count_nonzero(dirs, axis=1)
        v = dirs / np.sqrt(nnz)[:, None]
        w = np.select([nnz == 1, nnz == 2, nnz == 3], [1.0 / 21.0, 4.0 / 105.0, 9.0 / 280.0])
        return v, w
    if vset == 2:
        ang = np.arange(8) * (PI / 4.0)
        v = np.stack([np.cos(ang), np.sin(ang)], axis=1)
        v[np.abs(v) < 1e-15] = 0.0
        return v, np.full(8, 1.0 / 8.0)
    raise ValueError("vset must be 2 or 3")


def opposite(v):
    """Index of the reversed direction -v_i for every i (bounce-back partner)."""
    q = v.shape[0]
    opp = np.empty(q, dtype=np.int64)
    for i in range(q):
        d = np.abs(v + v[i][None, :]).sum(axis=1)
        opp[i] = int(np.argmin(d))
        assert d[opp[i]] < 1e-12
    return opp


def metric(dp):
    """Minkowski metric diag(+1, -1, ..., -1) in 1 + D_p dimensions."""
    return np.diag([1.0] + [-1.0] * dp)


# --------------------------------------------------------------------------
# Moments, equilibrium, equation of state
# --------------------------------------------------------------------------
def moments(f, v):
    """T^{mu nu} = sum_i f_i p^mu p^nu with p = (1, v_i)  (Eq. energyMomentumIntegral
    in its discrete form; Sec. "Boltzmann to Lattice Boltzmann", T^{mu nu} from
    the expansion coefficients).  f: (Q, ...) -> (..., D, D)."""
    p = np.concatenate([np.ones((v.shape[0], 1)), v], axis=1)
    return np.einsum("q...,qm,qn->...mn", f, p, p)


def pressure(eps, dp):
    """Equation of state P = eps / D_p from the vanishing trace of T^{mu nu} for
    massless particles (App. "Determination of the Equation of State")."""
    return eps / dp


def temperature(eps, vset=3):
    """Temperature from eps (Sec. "Boltzmann to Lattice Boltzmann"):
    eps = 3 T^4 / pi^2 for the three-dimensional momentum set.  For the
    two-dimensional set (not in the paper) the massless Z = 1 gas gives
    eps = T^3 / pi."""
    if vset == 3:
        return (PI * PI * eps / 3.0) ** 0.25
    return (PI * eps) ** (1.0 / 3.0)


def relaxation_time(T, eta_over_s, vset=3):
    """tau_R = 5 (eta/s) / T (Sec. "Relativistic Lattice Boltzmann").  The
    two-dimensional set uses 4 (eta/s) / T (eta = tau (eps + P) / (D_p + 2))."""
    return (5.0 if vset == 3 else 4.0) * eta_over_s / T


def ideal_T(eps, u, dp):
    """T_eq^{mu nu} = (eps + P) u^mu u^nu - P g^{mu nu}  (Eq. stressEnergyT with the
    rest-frame sign of App. "Determination of the Equation of State")."""
    P = pressure(eps, dp)
    g = metric(dp)
    return ((eps + P)[..., None, None] * u[..., :, None] * u[..., None, :]
            - P[..., None, None] * g)


def four_velocity(ux, uy, dp):
    """u^mu = (u^0, u^x, u^y[, 0]) with u^0 = sqrt(1 + |u|^2) from the spatial
    components (u^mu = gamma (1, v), Sec. "Relativistic Lattice Boltzmann")."""
    u0 = np.sqrt(1.0 + ux * ux + uy * uy)
    comps = [u0, ux, uy] + [np.zeros_like(ux)] * (dp - 2)
    return np.stack(comps, axis=-1)


def equilibrium(Teq, v, w):
    """Discrete equilibrium projected on the orthogonal polynomials of App. A up to
    second order, with the coefficient normalisations of Eq. rel_pdf_exp_coef
    (1, 3, 15/2 for D_p = 3; the circle set has 1, 2, 4):

        f_eq,i = w_i [ T^00 + D_p T^0j v_j
                       + c2 (T^jk - delta^jk T^00 / D_p)(v_j v_k - delta_jk / D_p) ]

    Teq: (..., D, D) -> (Q, ...)."""
    dp = v.shape[1]
    c2 = dp * (dp + 2) / 2.0
    T00 = Teq[..., 0, 0]
    T0j = Teq[..., 0, 1:]
    A = Teq[..., 1:, 1:] - np.eye(dp) * (T00 / dp)[..., None, None]
    out = np.empty((v.shape[0],) + T00.shape)
    for i in range(v.shape[0]):
        P2 = np.outer(v[i], v[i]) - np.eye(dp) / dp
        out[i] = w[i] * (T00 + dp * (T0j @ v[i]) + c2 * np.einsum("...jk,jk->...", A, P2))
    return out


# --------------------------------------------------------------------------
# Landau matching  u_mu T^{mu nu} = eps u^nu   (Sec. "Relativistic Lattice
# Boltzmann"; Sec. "Boltzmann to Lattice Boltzmann": eigenvalue problem)
# --------------------------------------------------------------------------
def landau(T):
    """Timelike eigenpair of T^mu_nu = T^{mu lam} g_{lam nu}.

    Returns eps (...,) and u^mu (..., D) normalised to u.u = 1, u^0 > 0.
    Raises if a cell has no timelike eigenvector with positive eigenvalue."""
    dp = T.shape[-1] - 1
    g = metric(dp)
    shape = T.shape[:-2]
    Tm = (T @ g).reshape(-1, dp + 1, dp + 1)
    lam, vec = np.linalg.eig(Tm)
    imag = np.abs(lam.imag).max(axis=1)
    lam = lam.real
    vec = vec.real
    # Minkowski norm of each (column) eigenvector relative to its Euclidean norm.
    mink = np.einsum("nmk,m,nmk->nk", vec, np.diag(g), vec)
    eucl = np.einsum("nmk,nmk->nk", vec, vec)
    score = mink / eucl
    k = np.argmax(score, axis=1)
    idx = np.arange(Tm.shape[0])
    u = vec[idx, :, k]
    norm = mink[idx, k]
    # A physical state has real eigenvalues and one timelike eigenvector whose
    # eigenvalue is a finite fraction of T^00 (1e-6 excludes degenerate beams,
    # whose Jordan blocks give O(sqrt(machine eps)) spurious eigenvalues).
    T00 = Tm[:, 0, 0]
    bad = ((imag > 1e-12 * np.abs(T00)) | (score[idx, k] <= 1e-6)
           | (lam[idx, k] <= 1e-6 * np.abs(T00)))
    if np.any(bad):
        raise FloatingPointError("Landau matching: no timelike eigenvector with eps > 0")
    u = u / np.sqrt(norm)[:, None]
    u = u * np.sign(u[:, 0])[:, None]
    return lam[idx, k].reshape(shape), u.reshape(shape + (dp + 1,))


# --------------------------------------------------------------------------
# Collision and force  (Eq. boltzmanneq_rel, Eq. forceTerm, App. B)
# --------------------------------------------------------------------------
def collision(f, eps, u, T, eta_over_s, dt, v, w, vset=3):
    """dt C[f]_i = (dt / tau_R) (p.u / p^0)_i (f_eq,i - f_i), p.u / p^0 = u^0 - v_i.u,
    tau_R = 5 (eta/s) / T  (Eq. boltzmanneq_rel; explicit Euler, Sec. "The
    Standard/Classical LBM", item 5)."""
    dp = v.shape[1]
    feq = equilibrium(ideal_T(eps, u, dp), v, w)
    tau = relaxation_time(T, eta_over_s, vset)
    out = np.empty_like(f)
    for i in range(v.shape[0]):
        pu = u[..., 0] - u[..., 1:] @ v[i]
        out[i] = (dt / tau) * pu * (feq[i] - f[i])
    return out


def force_source(f, F, v, w, T0):
    """Projected driving term S_i (Eq. forceTerm; coefficients of App. B,
    Eqs. expCoef01, forceExpCoef00, forceExpCoef02):

        S_i = -(6 / T0) w_i [ 1/4 F.M1 - 1/2 (F.v_i) M0
                              + 5/4 v_i.B.v_i - 5/2 (F.v_i)(v_i.M1) ]

    with M0 = sum_l f_l, M1 = sum_l f_l v_l, B_jk = sum_l f_l (F.v_l) v_lj v_lk over
    the three momentum components, F = (F^x, F^y, 0) the in-plane force.
    6 = int_0^inf p^3 e^{-p} dp turns the expansion coefficients into energy-weighted
    populations; the overall sign makes a uniform force accelerate the fluid along
    +F.  F: (..., 2)."""
    q, dp = v.shape
    assert dp == 3, "the projected force is defined for the three-dimensional set"
    F3 = np.concatenate([F, np.zeros(F.shape[:-1] + (1,))], axis=-1)
    M0 = f.sum(axis=0)
    M1 = np.einsum("q...,qj->...j", f, v)
    Fv = np.einsum("...j,qj->q...", F3, v)                      # (Q, ...)
    B = np.einsum("q...,q...,qj,qk->...jk", f, Fv, v, v)
    FM1 = np.einsum("...j,...j->...", F3, M1)
    out = np.empty_like(f)
    for i in range(q):
        vBv = np.einsum("...jk,j,k->...", B, v[i], v[i])
        vM1 = M1 @ v[i]
        bracket = 0.25 * FM1 - 0.5 * Fv[i] * M0 + 1.25 * vBv - 2.5 * Fv[i] * vM1
        out[i] = -(6.0 / T0) * w[i] * bracket
    return out


# --------------------------------------------------------------------------
# Streaming (Sec. "Boltzmann to Lattice Boltzmann": off-lattice momenta,
# linear interpolation; Part II "Model and Methods": bounce-back at impurity
# nodes)
# --------------------------------------------------------------------------
def stream(fstar, v, courant, solid, opp):
    """Pull streaming with bilinear interpolation on a periodic window.

    f_i(x) = sum over the 2 x 2 cells c enclosing x - C v_i,par of beta_c f*_i(c), where
    beta_c are the bilinear weights; a solid source cell c contributes f*_{opp(i)}(x)
    instead (bounce-back).  Solid cells hold zero.  fstar: (Q, H, W), solid: (H, W)."""
    out = np.zeros_like(fstar)
    for i in range(v.shape[0]):
        dx, dy = courant * v[i, 0], courant * v[i, 1]
        sx, sy = int(np.sign(dx)), int(np.sign(dy))
        ax, ay = abs(dx), abs(dy)
        for (ox, oy), beta in (((0, 0), (1 - ax) * (1 - ay)), ((sx, 0), ax * (1 - ay)),
                               ((0, sy), (1 - ax) * ay), ((sx, sy), ax * ay)):
            if beta == 0.0:
                continue
            src = np.roll(fstar[i], (oy, ox), axis=(0, 1))       # src[y, x] = f*[y - oy, x - ox]
            src_solid = np.roll(solid, (oy, ox), axis=(0, 1))
            out[i] += beta * np.where(src_solid, fstar[opp[i]], src)
    out[:, solid] = 0.0
    return out


def stream_open(fstar, v, courant, solid, opp, f_in, wall_rows):
    """Pull streaming of an open channel (Part II, "Model and Methods"): the populations
    arriving from beyond x = 0 are those of the inflow equilibrium f_in (Q,), and beyond
    x = N_x - 1 the last column repeats itself (zero-gradient outflow).  y keeps the
    window's own wrap.  The two boundary columns are appended to a copy of the window, it is
    streamed as usual, and the interior is kept.  wall_rows (H,) marks solid wall rows,
    which stay solid in the appended columns too."""
    q, h, w = fstar.shape
    pad = np.empty((q, h, w + 2))
    pad[:, :, 1:-1] = fstar
    pad[:, :, 0] = f_in[:, None]
    pad[:, :, -1] = fstar[:, :, -1]
    pad[:, wall_rows, 0] = 0.0
    sp = np.zeros((h, w + 2), bool)
    sp[:, 1:-1] = solid
    sp[:, 0] = wall_rows
    sp[:, -1] = wall_rows
    return stream(pad, v, courant, sp, opp)[:, :, 1:-1]


def column_means(ux, uy, solid=None):
    """j(x) = mean over y of v = u^i / u^0 per column (solid cells count as zero): the current
    density of Part II in units of the particle speed."""
    u0 = np.sqrt(1.0 + ux * ux + uy * uy)
    vx, vy = ux / u0, uy / u0
    if solid is not None:
        vx = np.where(solid, 0.0, vx)
        vy = np.where(solid, 0.0, vy)
    return vx.mean(axis=0), vy.mean(axis=0)


# --------------------------------------------------------------------------
# Stirring force (Part I, "Model and Methods": random amplitude and in-plane
# direction on the wave vectors of a shell, transformed to configuration space)
# --------------------------------------------------------------------------
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
    random numbers: as easy as 1, 2, 3"), on Python integers."""
    c = [int(x) & MASK32 for x in ctr]
    k0, k1 = int(key[0]) & MASK32, int(key[1]) & MASK32
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c[0]
        p1 = PHILOX_M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK32, p1 & MASK32,
             ((p0 >> 32) ^ c[3] ^ k1) & MASK32, p0 & MASK32]
    return c


def shell_modes(kmin, kmax):
    """Half-plane integer wave vectors (k_y > 0, or k_y = 0 and k_x > 0) with
    kmin^2 <= k_x^2 + k_y^2 <= kmax^2, ordered by (k_y, k_x)."""
    out = []
    for ky in range(0, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if (ky > 0 or kx > 0) and kmin * kmin <= kx * kx + ky * ky <= kmax * kmax:
                out.append((kx, ky))
    return out


def mode_draws(seed, step, nmodes, amp):
    """Per-mode amplitude a_m (Gaussian, Box-Muller), phase phi_m and direction psi_m
    of step `step`: (r0..r3) = Philox4x32-10(counter (step lo, m, step hi, 0),
    key (seed lo, seed hi)); u_j = (r_j + 1/2) 2^-32."""
    a = np.empty(nmodes)
    phi = np.empty(nmodes)
    psi = np.empty(nmodes)
    key = (seed & MASK32, (seed >> 32) & MASK32)
    for m in range(nmodes):
        r = philox4x32_10((step & MASK32, m, (step >> 32) & MASK32, 0), key)
        u = [(x + 0.5) * 2.0 ** -32 for x in r]
        a[m] = amp * np.sqrt(-2.0 * np.log(u[0])) * np.cos(2.0 * PI * u[1])
        phi[m] = 2.0 * PI * u[2]
        psi[m] = 2.0 * PI * u[3]
    return a, phi, psi


def stirring_force(X, Y, nx, ny, modes, a, phi, psi):
    """F(x, y) = sum_m a_m (cos psi_m, sin psi_m) cos(2 pi (k_x x / N_x + k_y y / N_y) + phi_m)
    at integer lattice coordinates X, Y.  Returns (..., 2)."""
    F = np.zeros(X.shape + (2,))
    for m, (kx, ky) in enumerate(modes):
        c = a[m] * np.cos(2.0 * PI * (kx * X / nx + ky * Y / ny) + phi[m])
        F[..., 0] += np.cos(psi[m]) * c
        F[..., 1] += np.sin(psi[m]) * c
    return F


# --------------------------------------------------------------------------
# Energy spectrum (Sec. "Turbulence": E(k) = d calE / dk, calE = 1/2 <|v(k)|^2>)
# --------------------------------------------------------------------------
def spectrum(ux, uy, nbins, solid=None):
    """E(n) = 1/2 sum_{k: round|k| = n} |v^(k)|^2 / (N_x N_y)^2 with v = u^i / u^0 and
    v^(k) = sum_x v(x) e^{-i k.x} (integer wave-number indices, signed)."""
    ny, nx = ux.shape
    u0 = np.sqrt(1.0 + ux * ux + uy * uy)
    vx, vy = ux / u0, uy / u0
    if solid is not None:
        vx = np.where(solid, 0.0, vx)
        vy = np.where(solid, 0.0, vy)
    P = np.abs(np.fft.fft2(vx)) ** 2 + np.abs(np.fft.fft2(vy)) ** 2
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kmag = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    n = np.rint(kmag).astype(np.int64)
    E = np.zeros(nbins)
    sel = n < nbins
    np.add.at(E, n[sel], 0.5 * P[sel] / float(nx * ny) ** 2)
    return E


def band_energy(ux, uy, k2lo, k2hi=0):
    """(1/2) sum over integer wave vectors with k2lo <= k_x^2 + k_y^2 < k2hi (k2hi <= 0: no
    upper bound) of |v^(k)|^2 / (N_x N_y)^2, v = u^i / u^0: the kinetic energy of the field
    filtered to a band (Part I, "Model and Methods": the recorded velocities are filtered
    to remove the driven range)."""
    ny, nx = ux.shape
    u0 = np.sqrt(1.0 + ux * ux + uy * uy)
    P = np.abs(np.fft.fft2(ux / u0)) ** 2 + np.abs(np.fft.fft2(uy / u0)) ** 2
    kx = np.rint(np.fft.fftfreq(nx) * nx).astype(np.int64)
    ky = np.rint(np.fft.fftfreq(ny) * ny).astype(np.int64)
    k2 = kx[None, :] ** 2 + ky[:, None] ** 2
    sel = k2 >= k2lo
    if k2hi > 0:
        sel &= k2 < k2hi
    return 0.5 * P[sel].sum() / float(nx * ny) ** 2


# --------------------------------------------------------------------------
# Time stepping over a window of the lattice
# --------------------------------------------------------------------------
DEFAULTS = dict(walls_y=0, vset=3, a=0.1, dt=0.05, eta_over_s=0.1, eps0=1.0,
                body_force=(0.0, 0.0), kmin=0, kmax=0, force_amp=0.0, seed=0,
                solid=None, init_eps=None, init_ux=None, init_uy=None, mode_scale=None,
                open_x=0, inflow_ux=0.0)


class Window:
    """A periodic window of the lattice: populations (Q, H, W), global integer
    coordinates X, Y of its cells and its solid mask.  Walls in y are ghost solid
    rows at y = -1 and y = N_y; a window that is the whole wall-bounded domain
    carries both ghost rows so that its periodic wrap never joins fluid rows."""

    def __init__(self, cfg, xs, ys):
        self.cfg = cfg
        nx, ny = cfg["nx"], cfg["ny"]
        self.X, self.Y = np.meshgrid(np.asarray(xs) % nx, np.asarray(ys), indexing="xy")
        yin = self.Y.copy()
        if cfg["walls_y"]:
            ghost = (self.Y < 0) | (self.Y >= ny)
        else:
            yin = yin % ny
            self.Y = yin
            ghost = np.zeros(self.Y.shape, bool)
        yc = np.clip(yin, 0, ny - 1)
        solid = np.zeros(self.Y.shape, bool) if cfg["solid"] is None else \
            np.asarray(cfg["solid"], bool)[yc, self.X]
        self.solid = solid | ghost


def _field(cfg, name, default, win):
    arr = cfg[name]
    if arr is None:
        return np.full(win.X.shape, default, dtype=np.float64)
    yc = np.clip(win.Y, 0, cfg["ny"] - 1)
    return np.asarray(arr, np.float64)[yc, win.X]


class Oracle:
    """Runs the update of the module docstring on a window of the lattice."""

    def __init__(self, cfg, xs=None, ys=None):
        c = dict(DEFAULTS)
        c.update(cfg)
        self.cfg = c
        nx, ny = c["nx"], c["ny"]
        if c["open_x"] and xs is not None and len(xs) != nx:
            raise ValueError("an open channel is run on the whole lattice width")
        if xs is None:
            xs = np.arange(nx)
        if ys is None:
            ys = np.arange(-1, ny + 1) if c["walls_y"] else np.arange(ny)
        self.win = Window(c, xs, ys)
        self.v, self.w = velocity_set(c["vset"])
        self.dp = self.v.shape[1]
        self.opp = opposite(self.v)
        self.courant = c["dt"] / c["a"]
        self.T0 = temperature(c["eps0"], c["vset"])
        self.modes = shell_modes(c["kmin"], c["kmax"]) if c["force_amp"] != 0.0 else []
        self.step_index = 0
        eps = _field(c, "init_eps", c["eps0"], self.win)
        ux = _field(c, "init_ux", 0.0, self.win)
        uy = _field(c, "init_uy", 0.0, self.win)
        u = four_velocity(ux, uy, self.dp)
        self.fstar = equilibrium(ideal_T(eps, u, self.dp), self.v, self.w)
        self.fstar[:, self.win.solid] = 0.0
        if c["open_x"]:
            u_in = four_velocity(np.array([c["inflow_ux"]]), np.array([0.0]), self.dp)
            self.f_in = equilibrium(ideal_T(np.array([c["eps0"]]), u_in, self.dp), self.v, self.w)[:, 0]
            self.wall_rows = (self.win.Y < 0) | (self.win.Y >= ny) if c["walls_y"] else np.zeros(self.win.Y.shape, bool)
            self.wall_rows = self.wall_rows[:, 0]

    def streamed(self):
        """f_n = stream(f*_n) with the lattice's boundaries."""
        if self.cfg["open_x"]:
            return stream_open(self.fstar, self.v, self.courant, self.win.solid, self.opp, self.f_in, self.wall_rows)
        return stream(self.fstar, self.v, self.courant, self.win.solid, self.opp)

    def force_field(self, n):
        c = self.cfg
        F = np.zeros(self.win.X.shape + (2,))
        F[..., 0] += c["body_force"][0]
        F[..., 1] += c["body_force"][1]
        if self.modes:
            a, phi, psi = mode_draws(c["seed"], n, len(self.modes), c["force_amp"])
            if c["mode_scale"] is not None:  # amplitude multipliers sigma_m (parameters of the adjoint)
                a = a * np.asarray(c["mode_scale"], np.float64)
            F += stirring_force(self.win.X, self.win.Y, c["nx"], c["ny"], self.modes, a, phi, psi)
        return F

    def macroscopic(self, f):
        """eps, u^mu (Landau frame) and T^{mu nu} of f at the fluid cells."""
        fluid = ~self.win.solid
        T = moments(f[:, fluid], self.v)
        eps, u = landau(T)
        return fluid, T, eps, u

    def step(self):
        c = self.cfg
        f = self.streamed()
        fluid, T, eps, u = self.macroscopic(f)
        Tloc = temperature(eps, c["vset"])
        ff = f[:, fluid]
        new = ff + collision(ff, eps, u, Tloc, c["eta_over_s"], c["dt"], self.v, self.w, c["vset"])
        needs_force = self.modes or c["body_force"][0] != 0.0 or c["body_force"][1] != 0.0
        if needs_force:
            F = self.force_field(self.step_index)[fluid]
            new = new + c["dt"] * force_source(ff, F, self.v, self.w, self.T0)
        self.fstar = np.zeros_like(self.fstar)
        self.fstar[:, fluid] = new
        self.step_index += 1

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    def crop(self, k=1):
        """Drop the outer k rings of cells of the window.  After a step, a cell within k
        cells of the window's edge may have pulled values across the window's own periodic
        wrap, which the lattice does not have; the cells further in are exact."""
        if self.cfg["open_x"]:
            raise ValueError("an open channel is run on the whole lattice width")
        self.fstar = self.fstar[:, k:-k, k:-k]
        self.win.X = self.win.X[k:-k, k:-k]
        self.win.Y = self.win.Y[k:-k, k:-k]
        self.win.solid = self.win.solid[k:-k, k:-k]
        return self

    def fields(self):
        """eps, u^x, u^y of the current state f_n = stream(f*_n) (zero at solid
        cells) and the totals (sum T^00, sum T^0x, sum T^0y, sum 1/2 |v|^2) over
        fluid cells."""
        f = self.streamed()
        fluid, T, eps, u = self.macroscopic(f)
        E = np.zeros(self.win.X.shape)
        UX = np.zeros(self.win.X.shape)
        UY = np.zeros(self.win.X.shape)
        E[fluid], UX[fluid], UY[fluid] = eps, u[:, 1], u[:, 2]
        vx, vy = u[:, 1] / u[:, 0], u[:, 2] / u[:, 0]
        totals = np.array([T[:, 0, 0].sum(), T[:, 0, 1].sum(), T[:, 0, 2].sum(),
                           0.5 * (vx * vx + vy * vy).sum()])
        return E, UX, UY, totals


def run(cfg, nsteps):
    """Full-lattice run; returns eps, u^x, u^y (N_y x N_x) and totals after nsteps."""
    o = Oracle(cfg).run(nsteps)
    E, UX, UY, tot = o.fields()
    if o.cfg["walls_y"]:
        E, UX, UY = E[1:-1], UX[1:-1], UY[1:-1]
    return E, UX, UY, tot


def window_populations(cfg, fstar, x, y, r):
    """The populations of the window of radius r around cell (x, y), taken from a state
    fstar (Q, N_y, N_x) of the whole lattice: x wraps; y wraps unless the lattice has
    walls, whose ghost rows (and anything beyond them) hold zero, as solid cells do."""
    c = dict(DEFAULTS)
    c.update(cfg)
    nx, ny = c["nx"], c["ny"]
    xs = np.arange(x - r, x + r + 1) % nx
    ys = np.arange(y - r, y + r + 1)
    out = np.zeros((fstar.shape[0], len(ys), len(xs)))
    if c["walls_y"]:
        inside = (ys >= 0) & (ys < ny)
        out[:, inside, :] = fstar[:, ys[inside]][:, :, xs]
    else:
        out[:] = fstar[:, ys % ny][:, :, xs]
    return out


def sample_block(cfg, x, y, nsteps, half=0, fstar_window=None, step0=0):
    """eps, u^x, u^y after nsteps steps of the (2 half + 1) x (2 half + 1) block of cells
    centred on (x, y), computed on a window of radius nsteps + half + 1 around it (the
    update's domain of dependence grows by one cell per step).  The window starts from
    the initial fields of cfg, or from the post-collision populations fstar_window of step
    step0 (as window_populations returns them); after every step it drops its outer ring,
    whose cells are no longer exact (Oracle.crop), and ends at radius half + 1: the block
    and the ring the final stream reads."""
    r = nsteps + half + 1
    o = Oracle(cfg, np.arange(x - r, x + r + 1), np.arange(y - r, y + r + 1))
    if fstar_window is not None:
        o.fstar = np.array(fstar_window, dtype=np.float64)
        o.fstar[:, o.win.solid] = 0.0
        o.step_index = step0
    for _ in range(nsteps):
        o.step()
        o.crop(1)
    E, UX, UY, _ = o.fields()
    return E[1:-1, 1:-1], UX[1:-1, 1:-1], UY[1:-1, 1:-1]


def run_sampled(cfg, nsteps, points, fstar=None, step0=0):
    """eps, u^x, u^y after nsteps steps at the cells `points` [(x, y), ...] of a lattice of
    any size, each computed on its own shrinking window (sample_block with half = 0).
    With fstar (the post-collision populations (Q, N_y, N_x) of the whole lattice at step
    step0) the run starts from that state instead of the initial fields."""
    out = []
    for (x, y) in points:
        fw = None if fstar is None else window_populations(cfg, fstar, x, y, nsteps + 1)
        E, UX, UY = sample_block(cfg, x, y, nsteps, 0, fw, step0)
        out.append((E[0, 0], UX[0, 0], UY[0, 0]))
    return np.array(out)
