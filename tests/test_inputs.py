"""The seeded input generators: the smooth random fields equal numpy's inverse real 2-D
FFT of the same half spectrum (the generator evaluates it from the non-zero rows only, so
that lattices of 10^8 cells are generated in seconds)."""
import numpy as np
import pytest

from paper_2205_04658_gb300 import inputs


def _fields_by_irfft2(nx, ny, seed, eps_amp, u_amp, kmax):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        S = np.zeros((ny, nx // 2 + 1), dtype=np.complex128)
        for ky in range(-kmax, kmax + 1):
            for kx in range(0, kmax + 1):
                if kx == 0 and ky <= 0:
                    continue
                S[ky % ny, kx] = rng.standard_normal() + 1j * rng.standard_normal()
        g = np.fft.irfft2(S, s=(ny, nx))
        out.append(g / np.abs(g).max())
    return 1.0 + eps_amp * out[0], u_amp * out[1], u_amp * out[2]


@pytest.mark.parametrize("nx,ny,kmax", [
    (64, 48, 4),     # plain
    (9, 13, 4),      # odd sizes
    (8, 12, 4),      # k_x = 4 is the Nyquist column
    (16, 8, 4),      # k_y = -4 and 4 alias (a later draw replaces an earlier one)
    (160, 72, 8),
    (96, 40, 3),
])
def test_smooth_fields_equal_irfft2(nx, ny, kmax):
    got = inputs.smooth_random_fields(nx, ny, seed=nx + ny, eps_amp=0.02, u_amp=0.03, kmax=kmax)
    ref = _fields_by_irfft2(nx, ny, nx + ny, 0.02, 0.03, kmax)
    for g, r in zip(got, ref):
        assert g.shape == (ny, nx) and g.dtype == np.float64 and g.flags.c_contiguous
        assert np.max(np.abs(g - r)) <= 1e-15 * max(1.0, np.abs(r).max()) * 8


def test_smooth_fields_are_deterministic_and_normalised():
    a = inputs.smooth_random_fields(40, 24, seed=7, eps_amp=0.1, u_amp=0.2, kmax=3)
    b = inputs.smooth_random_fields(40, 24, seed=7, eps_amp=0.1, u_amp=0.2, kmax=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.isclose(np.abs(a[0] - 1.0).max(), 0.1)
    assert np.isclose(np.abs(a[1]).max(), 0.2) and np.isclose(np.abs(a[2]).max(), 0.2)
    # zero mean: no k = 0 coefficient
    for g in a[1:]:
        assert abs(g.mean()) < 1e-15
