"""Pins of the oracle's stirring force (Part I, "Model and Methods": random
amplitude and in-plane direction on a shell of wave vectors, zero spatial mean)
and of its counter-based generator."""
import os

import numpy as np

from oracle import rlbm_oracle as O

KAT = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    n = 0
    for line in open(KAT):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(x, 16) for x in line.split()]
        assert O.philox4x32_10(vals[0:4], vals[4:6]) == vals[6:10]
        n += 1
    assert n == 3


def test_shell_mode_counts_and_order():
    m = O.shell_modes(8, 10)
    assert len(m) == 62 and len(O.shell_modes(4, 6)) == 34
    assert m == sorted(m, key=lambda k: (k[1], k[0]))
    assert all(k[1] > 0 or k[0] > 0 for k in m)
    assert all(64 <= k[0] ** 2 + k[1] ** 2 <= 100 for k in m)
    # the half plane holds exactly one of every +-k pair of the full shell
    full = {(kx, ky) for kx in range(-10, 11) for ky in range(-10, 11) if 64 <= kx * kx + ky * ky <= 100}
    assert {k for k in m} | {(-k[0], -k[1]) for k in m} == full


def _field(nx, ny, seed, step, kmin, kmax, amp):
    modes = O.shell_modes(kmin, kmax)
    a, phi, psi = O.mode_draws(seed, step, len(modes), amp)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    return O.stirring_force(X, Y, nx, ny, modes, a, phi, psi), modes, a, phi, psi


def test_force_field_has_zero_mean_and_shell_support():
    nx, ny = 32, 24
    F, modes, a, phi, psi = _field(nx, ny, seed=9, step=3, kmin=4, kmax=6, amp=1e-2)
    assert np.abs(F.mean(axis=(0, 1))).max() < 1e-17
    # direct DFT: non-zero exactly on +-k of the shell, with |F^(k)| = |a_m| N / 2
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    shell = {(kx % nx, ky % ny): m for m, (kx, ky) in enumerate(modes)}
    shell.update({((-kx) % nx, (-ky) % ny): m for m, (kx, ky) in enumerate(modes)})
    for qy in range(ny):
        for qx in range(nx):
            e = np.exp(-2j * np.pi * (qx * X / nx + qy * Y / ny))
            amp = np.hypot(abs((F[..., 0] * e).sum()), abs((F[..., 1] * e).sum()))
            if (qx, qy) in shell:
                assert abs(amp - abs(a[shell[(qx, qy)]]) * nx * ny / 2) < 1e-12
            else:
                assert amp < 1e-13


def test_mode_draws_statistics():
    """Amplitudes are N(0, amp^2), phases and directions uniform on [0, 2 pi)."""
    A, P, S = [], [], []
    for step in range(300):
        a, phi, psi = O.mode_draws(1234, step, 34, 2.0)
        A.append(a), P.append(phi), S.append(psi)
    A, P, S = np.concatenate(A), np.concatenate(P), np.concatenate(S)
    n = A.size
    assert abs(A.mean()) < 4 * 2.0 / np.sqrt(n)
    assert abs(A.std() / 2.0 - 1.0) < 0.03
    for x in (P, S):
        assert x.min() > 0 and x.max() < 2 * np.pi
        assert abs(x.mean() / np.pi - 1.0) < 0.02


def test_draws_depend_on_seed_step_and_mode():
    a1 = O.mode_draws(2, 0, 5, 1.0)[0]
    assert len(set(np.round(a1, 12))) == 5
    assert not np.allclose(a1, O.mode_draws(2, 1, 5, 1.0)[0])
    assert not np.allclose(a1, O.mode_draws(3, 0, 5, 1.0)[0])
    assert np.array_equal(a1, O.mode_draws(2, 0, 5, 1.0)[0])
