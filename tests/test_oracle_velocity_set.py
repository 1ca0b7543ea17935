"""Pins of the oracle's discrete momentum sets against closed-form angular
integrals (Sec. "Boltzmann to Lattice Boltzmann"; App. A, App. B)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import rlbm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_identities.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(Fraction(v))
    return vals


def dfact(n):
    return 1 if n <= 0 else n * dfact(n - 2)


def sphere_moment(a, b, c):
    """int dOmega/4pi x^a y^b z^c on the unit sphere (closed form)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    return dfact(a - 1) * dfact(b - 1) * dfact(c - 1) / dfact(a + b + c + 1)


def circle_moment(a, b):
    """int dtheta/2pi cos^a sin^b (closed form)."""
    if a % 2 or b % 2:
        return 0.0
    return dfact(a - 1) * dfact(b - 1) / dfact(a + b)


def test_weights_positive_and_normalised():
    for vs in (2, 3):
        v, w = O.velocity_set(vs)
        assert np.all(w > 0)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)


def test_paper_set_is_26_directions_of_d3q27():
    v, w = O.velocity_set(3)
    assert v.shape == (26, 3)
    dirs = np.rint(v * np.sqrt(np.count_nonzero(np.abs(v) > 1e-12, axis=1))[:, None]).astype(int)
    assert len({tuple(d) for d in dirs}) == 26


def test_sphere_quadrature_exact_to_degree_7_and_not_8():
    v, w = O.velocity_set(3)
    worst = {}
    for a in range(9):
        for b in range(9 - a):
            for c in range(9 - a - b):
                q = np.sum(w * v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c)
                d = a + b + c
                worst[d] = max(worst.get(d, 0.0), abs(q - sphere_moment(a, b, c)))
    for d in range(8):
        assert worst[d] < 1e-15, (d, worst[d])
    assert worst[8] > 1e-3  # a 26-point rule cannot be exact at degree 8


def test_circle_quadrature_exact_to_degree_7():
    v, w = O.velocity_set(2)
    for a in range(8):
        for b in range(8 - a):
            q = np.sum(w * v[:, 0] ** a * v[:, 1] ** b)
            assert abs(q - circle_moment(a, b)) < 1e-15


def test_appendix_a_orthogonality_relations():
    g = golden()
    v, w = O.velocity_set(3)
    I = np.eye(3)
    assert abs(np.sum(w) - g["P0P0"]) < 1e-15
    P1P1 = np.einsum("q,qi,qj->ij", w, v, v)
    assert np.abs(P1P1 - g["P1P1"] * I).max() < 1e-15
    P2 = np.einsum("qi,qj->qij", v, v) - I / 3.0
    P2P2 = np.einsum("q,qij,qlm->ijlm", w, P2, P2)
    exact = g["P2P2"] * (np.einsum("il,jm->ijlm", I, I) + np.einsum("im,jl->ijlm", I, I)
                         - 2.0 / 3.0 * np.einsum("ij,lm->ijlm", I, I))
    assert np.abs(P2P2 - exact).max() < 1e-15
    # P1 and P2 are mutually orthogonal, and P3 (App. A) is orthogonal to P1.
    assert np.abs(np.einsum("q,qi,qjk->ijk", w, v, P2)).max() < 1e-15
    P3 = (np.einsum("qi,qj,qk->qijk", v, v, v)
          - 0.2 * (np.einsum("ij,qk->qijk", I, v) + np.einsum("ik,qj->qijk", I, v)
                   + np.einsum("jk,qi->qijk", I, v)))
    assert np.abs(np.einsum("q,qijk,ql->ijkl", w, P3, v)).max() < 1e-15


def test_appendix_b_fourth_angular_moment():
    g = golden()
    v, w = O.velocity_set(3)
    I = np.eye(3)
    V4 = np.einsum("q,qi,qj,ql,qm->ijlm", w, v, v, v, v)
    exact = g["V4"] * (np.einsum("il,jm->ijlm", I, I) + np.einsum("im,jl->ijlm", I, I)
                       + np.einsum("ij,lm->ijlm", I, I))
    assert np.abs(V4 - exact).max() < 1e-15


@pytest.mark.parametrize("vs", [2, 3])
def test_opposite_reverses_direction(vs):
    v, _ = O.velocity_set(vs)
    opp = O.opposite(v)
    assert np.abs(v[opp] + v).max() < 1e-15
    assert np.all(opp[opp] == np.arange(len(v)))
