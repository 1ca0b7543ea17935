"""Seeded synthetic inputs shared by the CUDA path and its checks.

This module holds input generators only (initial macroscopic fields, impurity
masks, workload shapes); none of the update's arithmetic lives here.  Every
generator is deterministic in its seed.

Workload shapes follow the paper's runs: square periodic lattices stirred in a
shell of wave numbers (Part I, "Model and Methods"), and a wide sample with
circular impurities (Part II, "Model and Methods"), with dt = 0.05.
"""
import numpy as np


def shear_wave(nx, ny, amp=0.01):
    """u^x = amp sin(2 pi y / N_y), u^y = 0, eps = 1: a decaying transverse shear wave."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    return np.ones((ny, nx)), amp * np.sin(2.0 * np.pi * y / ny), np.zeros((ny, nx))


def _real_field_from_rows(rows, coef, nx, ny):
    """The inverse real 2-D DFT (numpy's irfft2 convention) of a half spectrum whose only
    non-zero rows are `rows` (k_y mod N_y) with columns k_x = 0 .. coef.shape[1] - 1:
        g(x, y) = Re sum_{k_x} h_{k_x} / N_x  C(y, k_x) e^{2 pi i k_x x / N_x},
        C(y, k_x) = (1 / N_y) sum_rows S(row, k_x) e^{2 pi i row y / N_y},
    with h = 1 at k_x = 0 and at the Nyquist column, 2 elsewhere.  A product of a
    (N_y x rows) and a (columns x N_x) factor: no transform of the whole lattice."""
    y = np.arange(ny, dtype=np.int64)
    Ey = np.exp(2j * np.pi * (np.outer(y, rows) % ny) / ny) / ny
    C = Ey @ coef
    kx = np.arange(coef.shape[1], dtype=np.int64)
    h = np.where((kx == 0) | ((nx % 2 == 0) & (kx == nx // 2)), 1.0, 2.0) / nx
    ang = 2.0 * np.pi * (np.outer(kx, np.arange(nx, dtype=np.int64)) % nx) / nx
    Cr, Ci = np.ascontiguousarray(C.real), np.ascontiguousarray(C.imag)  # BLAS wants contiguous factors
    g = Cr @ (h[:, None] * np.cos(ang))
    g -= Ci @ (h[:, None] * np.sin(ang))
    return g


def smooth_random_fields(nx, ny, seed, eps_amp=0.05, u_amp=0.05, kmax=4):
    """eps = 1 + eps_amp * g1, u^x = u_amp * g2, u^y = u_amp * g3, where each g is a real
    periodic field with Gaussian random Fourier coefficients on the wave numbers
    |k_x|, |k_y| <= kmax (k != 0), normalised to unit maximum modulus.  Each g is the
    inverse real DFT of its half spectrum (k_y taken mod N_y; a later draw replaces an
    earlier one at the same index), evaluated from the non-zero rows only."""
    rng = np.random.default_rng(seed)
    ncols = min(kmax + 1, nx // 2 + 1)
    out = []
    for _ in range(3):
        spec = {}
        for ky in range(-kmax, kmax + 1):
            for kx in range(0, kmax + 1):
                if kx == 0 and ky <= 0:
                    continue
                v = rng.standard_normal() + 1j * rng.standard_normal()
                spec.setdefault(ky % ny, np.zeros(ncols, dtype=np.complex128))[kx] = v
        rows = np.array(sorted(spec), dtype=np.int64)
        g = _real_field_from_rows(rows, np.array([spec[r] for r in rows]), nx, ny)
        g /= max(g.max(), -g.min())
        out.append(g)
    eps, ux, uy = out
    eps *= eps_amp
    eps += 1.0
    ux *= u_amp
    uy *= u_amp
    return eps, ux, uy


def disc_mask(nx, ny, radius, fraction, seed, walls_y=True, max_trials=1_000_000):
    """Solid mask (N_y x N_x, uint8) of non-overlapping discs of the given radius at
    seeded random integer centres: a cell is solid when (x - cx)^2 + (y - cy)^2 <= r^2
    (x periodic).  The disc count is round(fraction * N_x N_y / cells_per_disc);
    centres keep a distance >= 2r + 2 from each other and >= r + 1 from the walls."""
    r = int(radius)
    offs = [(dx, dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if dx * dx + dy * dy <= r * r]
    ndisc = int(round(fraction * nx * ny / len(offs)))
    rng = np.random.default_rng(seed)
    centres = []
    trials = 0
    lo = r + 1 if walls_y else 0
    hi = ny - r - 1 if walls_y else ny - 1
    while len(centres) < ndisc:
        trials += 1
        if trials > max_trials:
            raise RuntimeError("disc placement did not converge")
        cx = int(rng.integers(0, nx))
        cy = int(rng.integers(lo, hi + 1))
        ok = True
        for (px, py) in centres:
            dx = abs(cx - px)
            dx = min(dx, nx - dx)
            dy = abs(cy - py)
            if not walls_y:
                dy = min(dy, ny - dy)
            if dx * dx + dy * dy < (2 * r + 2) ** 2:
                ok = False
                break
        if ok:
            centres.append((cx, cy))
    mask = np.zeros((ny, nx), np.uint8)
    for (cx, cy) in centres:
        for (dx, dy) in offs:
            mask[(cy + dy) % ny, (cx + dx) % nx] = 1
    return mask, centres


def ensemble_sides(nmembers, seed, choices=(256, 512, 768, 1024)):
    """Lattice side of each ensemble member, uniform over `choices`."""
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=nmembers)]


# Workload shapes (dt = 0.05 everywhere, spacing a = 0.1 so dt/a = 0.5).
SHEAR_WAVE_64 = dict(nx=64, ny=64, precision="f64", eta_over_s=0.1, steps=200)
STIRRED_1024 = dict(nx=1024, ny=1024, precision="f32", eta_over_s=0.05, kmin=8, kmax=10,
                    force_amp=1e-4, seed=2, steps=20000, spectrum_every=500)
STIRRED_4096 = dict(STIRRED_1024, nx=4096, ny=4096, steps=200)
GRAPHENE_2048x512 = dict(nx=2048, ny=512, precision="f16", walls_y=1, body_force=(1e-6, 0.0),
                         eta_over_s=0.05, radius=6, fractions=(0.01, 0.05, 0.15),
                         geometry_seeds=(31, 35, 315), steps=50000)
ENSEMBLE_64 = dict(nmembers=64, side_seed=4, member_seed0=1000, precision="bf16",
                   eta_over_s=0.05, kmin=8, kmax=10, force_amp=1e-4, steps=5000)
ADJOINT_512 = dict(nx=512, ny=512, precision="f32", eta_over_s=0.05, kmin=4, kmax=6,
                   force_amp=1e-4, seed=5, steps=2000)


def channel_impurities(nx, ny, diameter_nodes, count=1, separation_nodes=89):
    """Solid mask of the Part II sample: one disc of the given (odd) diameter in the
    obstruction region near the inflow border (centre at x = nx / 8, y = ny / 2); a second
    one, when count = 2, next to it and slightly behind it with respect to the flow, at
    the given centre-to-centre distance (offset 20 nodes downstream, the rest across)."""
    r = diameter_nodes // 2
    Y, X = np.mgrid[0:ny, 0:nx]
    cx, cy = nx // 8, ny // 2
    mask = (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
    if count == 2:
        dx = 20
        dy = int(round(np.sqrt(max(separation_nodes ** 2 - dx * dx, 0))))
        cy2 = (cy + dy) % ny
        mask |= (X - (cx + dx)) ** 2 + (np.minimum(np.abs(Y - cy2), ny - np.abs(Y - cy2))) ** 2 <= r * r
    return mask.astype(np.uint8)


# Part II sample: 1024 x 256 nodes at 0.038 um (a 40 um x 10 um graphene sheet), impurity
# diameter 0.5 um = 13 nodes, inflow 0.1 v_F, periodic sides; eta/s set for Re = 6.37.
CHANNEL_1024x256 = dict(nx=1024, ny=256, open_x=1, inflow_ux=0.1, diameter_nodes=13, reynolds=6.37)
