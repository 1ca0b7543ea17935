"""Pins of the oracle's energy spectrum (Sec. "Turbulence": E(k) as the shell
density of 1/2 |v(k)|^2)."""
import numpy as np
import pytest

from oracle import rlbm_oracle as O
from paper_2205_04658_gb300 import inputs


def test_parseval():
    ex, ux, uy = inputs.smooth_random_fields(24, 16, seed=1, u_amp=0.2)
    E = O.spectrum(ux, uy, nbins=40)
    u0 = np.sqrt(1.0 + ux * ux + uy * uy)
    assert abs(E.sum() - 0.5 * np.mean((ux / u0) ** 2 + (uy / u0) ** 2)) < 1e-15


def test_single_mode_lands_in_its_bin():
    nx = ny = 32
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    vx = 0.01 * np.cos(2 * np.pi * (3 * X / nx + 4 * Y / ny))   # |k| = 5
    u0 = 1.0 / np.sqrt(1.0 - vx * vx)
    E = O.spectrum(u0 * vx, 0 * vx, nbins=20)
    assert abs(E[5] - 0.5 * np.mean(vx * vx)) < 1e-18
    assert np.abs(np.delete(E, 5)).max() < 1e-20


def test_matches_direct_dft_8x8():
    rng = np.random.default_rng(3)
    ux, uy = 0.1 * rng.standard_normal((2, 8, 8))
    E = O.spectrum(ux, uy, nbins=7)
    u0 = np.sqrt(1 + ux ** 2 + uy ** 2)
    vx, vy = ux / u0, uy / u0
    ref = np.zeros(7)
    for qy in range(8):
        for qx in range(8):
            kx = qx if qx < 4 else qx - 8
            ky = qy if qy < 4 else qy - 8
            zx = zy = 0.0
            for y in range(8):
                for x in range(8):
                    e = np.exp(-2j * np.pi * (qx * x + qy * y) / 8)
                    zx += vx[y, x] * e
                    zy += vy[y, x] * e
            n = int(round(np.sqrt(kx * kx + ky * ky)))
            ref[n] += 0.5 * (abs(zx) ** 2 + abs(zy) ** 2) / 64 ** 2
    assert np.abs(E - ref).max() < 1e-15


def test_band_energy_parseval_and_complement():
    """The unbounded band is half the mean |v|^2 (Parseval); a band and its complement add
    up to it; a single mode lands in exactly the band holding its |k|^2."""
    rng = np.random.default_rng(5)
    ux = 0.05 * rng.standard_normal((12, 20))
    uy = 0.05 * rng.standard_normal((12, 20))
    u0 = np.sqrt(1 + ux * ux + uy * uy)
    total = 0.5 * np.mean((ux / u0) ** 2 + (uy / u0) ** 2)
    assert O.band_energy(ux, uy, 0, 0) == pytest.approx(total, rel=1e-13)
    lo = O.band_energy(ux, uy, 0, 17)
    hi = O.band_energy(ux, uy, 17, 0)
    assert lo + hi == pytest.approx(total, rel=1e-13)
    # one mode (k_x, k_y) = (3, 2), |k|^2 = 13
    Y, X = np.mgrid[0:12, 0:20]
    vx = 0.01 * np.cos(2 * np.pi * (3 * X / 20 + 2 * Y / 12))
    g = 1.0 / np.sqrt(1.0 - vx * vx)  # u = gamma v with v = vx exactly
    e13 = O.band_energy(g * vx, 0 * vx, 13, 14)
    assert e13 == pytest.approx(0.5 * np.mean(vx * vx), rel=1e-12)
    assert O.band_energy(g * vx, 0 * vx, 0, 13) < 1e-30
    assert O.band_energy(g * vx, 0 * vx, 14, 0) < 1e-30
