"""Pins of the oracle's lattice tables, anisotropy functions and equilibria.

Each check is against something the paper or the mathematics fixes, not
against the oracle's own formulas: the hand-typed Tables 1-2 (golden fixture),
the moment identities the paper states for the lattices and the equilibria
(Sec. 3.2-3.3, Appendices A-B), finite differences of a_s, and closed-form
values of a_s along the cubic axes.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lattice_tables.json")
LATS = {7: "D3Q7", 15: "D3Q15", 19: "D3Q19", 5: "D2Q5", 9: "D2Q9"}
ALL_Q = [7, 15, 19, 5, 9]


def _dims(q):
    """Spatial dimensions of the lattice: the 2D lattices are stored with e_z = 0."""
    return 2 if q in (5, 9) else 3


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


@pytest.mark.parametrize("q", ALL_Q)
def test_tables_match_paper(gold, q):
    e, w, A, B, e2, opp = oracle.lattice(q)
    t = gold[LATS[q]]
    assert e.tolist() == t["e"]
    assert e2 == float(Fraction(t["e2"]))
    np.testing.assert_array_equal(w, [float(Fraction(v)) for v in t["w"]])
    np.testing.assert_array_equal(A, [float(Fraction(v)) for v in t["A"]])
    np.testing.assert_array_equal(B, [float(Fraction(v)) for v in t["B"]])


@pytest.mark.parametrize("q", ALL_Q)
def test_lattice_identities_exact(gold, q):
    """Moment identities of Sec. 3 in exact rational arithmetic on the typed tables,
    and the same identities on the oracle's tables in floating point."""
    t = gold[LATS[q]]
    e = t["e"]
    w = [Fraction(v) for v in t["w"]]
    A = [Fraction(v) for v in t["A"]]
    B = [Fraction(v) for v in t["B"]]
    e2 = Fraction(t["e2"])
    d = _dims(q)
    assert sum(w) == 1
    assert sum(A) == 1
    assert sum(B) == 0
    for a in range(3):
        assert sum(wi * ei[a] for wi, ei in zip(w, e)) == 0
    for a in range(d):
        for b in range(d):
            assert sum(wi * ei[a] * ei[b] for wi, ei in zip(w, e)) == (e2 if a == b else 0)
            # first moment of the B-part of h^(0): sum B_i e_ia e_ib / e^2 = delta_ab (App. B)
            assert sum(Bi * ei[a] * ei[b] for Bi, ei in zip(B, e)) / e2 == (1 if a == b else 0)
    # A_i + B_i = w_i: in pure liquid (q/zeta = 1) h^(0) reduces to the standard w_i U
    assert all(Ai + Bi == wi for Ai, Bi, wi in zip(A, B, w))
    # oracle floating tables satisfy the same identities
    eo, wo, Ao, Bo, e2o, opp = oracle.lattice(q)
    assert abs(wo.sum() - 1) < 1e-15
    eye = np.diag([1.0] * d + [0.0] * (3 - d))
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", wo, eo, eo), e2o * eye, atol=1e-15)


@pytest.mark.parametrize("q", ALL_Q)
def test_opposite_map(q):
    e, w, A, B, e2, opp = oracle.lattice(q)
    for i in range(q):
        np.testing.assert_array_equal(e[opp[i]], -e[i])
        assert w[opp[i]] == w[i]
    assert sorted(opp.tolist()) == list(range(q))


def test_fourth_order_isotropy():
    """sum w e_x^4 = 3 sum w e_x^2 e_y^2 holds for D3Q15/D3Q19 and fails for D3Q7: the
    mechanism behind the paper's grid-anisotropy comparison (Sec. 4.1)."""
    for q, iso in [(7, False), (15, True), (19, True), (5, False), (9, True)]:
        e, w, *_ = oracle.lattice(q)
        m4 = float(np.sum(w * e[:, 0] ** 4))
        m22 = float(np.sum(w * e[:, 0] ** 2 * e[:, 1] ** 2))
        assert (abs(m4 - 3 * m22) < 1e-15) == iso


# ---------------------------------------------------------------- anisotropy

def _fd_grad_of_as(kind, e1, e2, g, h=1e-6):
    out = np.zeros(3)
    for a in range(3):
        gp, gm = g.copy(), g.copy()
        gp[a] += h
        gm[a] -= h
        out[a] = (oracle.aniso(kind, e1, e2, gp)[0] - oracle.aniso(kind, e1, e2, gm)[0]) / (2 * h)
    return out


@pytest.mark.parametrize("kind,e1,e2", [(0, 0.05, 0.0), (0, -0.03, 0.0), (1, -0.02, 0.015), (1, 0.03, -0.01)])
def test_aniso_derivative_vs_finite_difference(kind, e1, e2):
    """Eq. (Derivees_As) and the derived K41/K61 derivatives against central differences
    of a_s itself (Eq. Anisotropic-Function_As, Eq. As_K41-K61)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        g = rng.normal(size=3) * rng.uniform(0.1, 3.0)
        _, das = oracle.aniso(kind, e1, e2, g)
        fd = _fd_grad_of_as(kind, e1, e2, g)
        scale = max(1e-3, np.abs(fd).max())
        assert np.abs(das - fd).max() / scale < 1e-6


def test_aniso_closed_forms():
    eps = 0.05
    # n along <100>: sum n^4 = 1 -> a_s = 1 + eps; <110>: 1/2 -> 1 - eps; <111>: 1/3 -> 1 - 5 eps/3
    for g, val in [([1.3, 0, 0], 1 + eps), ([0, -2, 2], 1 - eps), ([1, 1, 1], 1 - 5 * eps / 3)]:
        a, das = oracle.aniso(0, eps, 0, np.array(g, float))
        assert abs(a - val) < 1e-14
        # N vanishes along the symmetry axes <100>, <110>, <111>
        assert np.abs(das).max() < 1e-14
    e1, d = -0.02, 0.015
    # K41/K61: <100>: S=1, P=0; <110>: S=1/2, P=0; <111>: S=1/3, P=1/27
    for g, S, P in [([0, 0, -4.0], 1.0, 0.0), ([1, 1, 0], 0.5, 0.0), ([2, 2, 2], 1 / 3, 1 / 27)]:
        a, _ = oracle.aniso(1, e1, d, np.array(g, float))
        assert abs(a - (1 + e1 * (S - 0.6) + d * (3 * S + 66 * P - 17 / 7))) < 1e-14


def test_aniso_k41k61_reduces_to_standard_derivatives():
    """With delta = 0 and eps_1 = 4 eps, d a_s / d(grad phi) of Eq. (As_K41-K61) equals
    Eq. (Derivees_As) (the two a_s differ only by a constant)."""
    rng = np.random.default_rng(5)
    for _ in range(100):
        g = rng.normal(size=3)
        a0, d0 = oracle.aniso(0, 0.05, 0.0, g)
        a1, d1 = oracle.aniso(1, 0.20, 0.0, g)
        np.testing.assert_allclose(d1, d0, rtol=1e-12, atol=1e-14)
        assert abs((a1 - a0) - (0.15 - 0.20 * 0.6)) < 1e-13


def test_aniso_symmetries():
    """a_s depends on n only: invariant under scaling, sign flips and axis permutations;
    the derivative is odd in each component and homogeneous of degree -1."""
    rng = np.random.default_rng(9)
    for kind, e1, e2 in [(0, 0.05, 0.0), (1, -0.02, 0.015)]:
        for _ in range(50):
            g = rng.normal(size=3)
            a, d = oracle.aniso(kind, e1, e2, g)
            a2, d2 = oracle.aniso(kind, e1, e2, 2.5 * g)
            assert abs(a - a2) < 1e-14
            np.testing.assert_allclose(d2, d / 2.5, rtol=1e-12, atol=1e-15)
            perm = rng.permutation(3)
            a3, d3 = oracle.aniso(kind, e1, e2, g[perm])
            assert abs(a - a3) < 1e-14
            np.testing.assert_allclose(d3, d[perm], rtol=1e-12, atol=1e-15)
            s = np.array([-1.0, 1.0, -1.0])
            a4, d4 = oracle.aniso(kind, e1, e2, g * s)
            assert abs(a - a4) < 1e-14
            np.testing.assert_allclose(d4, d * s, rtol=1e-12, atol=1e-15)
            # Euler: a_s homogeneous of degree 0 -> g . grad(a_s) = 0
            assert abs(np.dot(g, d)) < 1e-13 * max(1.0, np.abs(d).max() * np.abs(g).max())


# ---------------------------------------------------------------- equilibria

@pytest.mark.parametrize("q", ALL_Q)
def test_phase_equilibrium_moments(q):
    """Sec. 3.2 / App. A: sum g0 = phi, sum g0 e = -N dt W0^2/(tau0 dx), sum g0 ee = e^2 phi I
    (I restricted to the lattice's plane in 2D, where N has no z component)."""
    e, w, A, B, e2, opp = oracle.lattice(q)
    d = _dims(q)
    eye = np.diag([1.0] * d + [0.0] * (3 - d))
    rng = np.random.default_rng(q)
    for _ in range(20):
        phi = rng.uniform(-1, 1)
        N = rng.normal(size=3)
        N[d:] = 0
        c = rng.uniform(0.001, 0.1)  # dt/dx W0^2/tau0
        g0 = oracle.geq(q, phi, N, c)
        assert abs(g0.sum() - phi) < 1e-14
        np.testing.assert_allclose(g0 @ e, -N * c, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", g0, e, e), e2 * phi * eye, atol=1e-14)


@pytest.mark.parametrize("q", ALL_Q)
def test_solute_equilibrium_moments(q):
    """Sec. 3.3 / App. B: sum h0 = U, sum h0 e = J dt/dx, sum h0 ee = e^2 (q/zeta) U I."""
    e, w, A, B, e2, opp = oracle.lattice(q)
    d = _dims(q)
    eye = np.diag([1.0] * d + [0.0] * (3 - d))
    rng = np.random.default_rng(100 + q)
    for _ in range(20):
        U = rng.uniform(-1, 0.5)
        qz = rng.uniform(0, 1)
        J = rng.normal(size=3)
        J[d:] = 0
        c = rng.uniform(0.001, 0.1)  # dt/dx
        h0 = oracle.heq(q, U, qz, J, c)
        assert abs(h0.sum() - U) < 1e-14
        np.testing.assert_allclose(h0 @ e, J * c, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", h0, e, e), e2 * qz * U * eye, atol=1e-14)


def test_paper_parameter_relations():
    """Eq. (Capillary-Length) and the lambda* of Sec. 4.1/4.2 reproduce the printed numbers."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")) as f:
        g = json.load(f)
    a1 = 5 * np.sqrt(2) / 8
    assert abs(a1 - g["a1"]) < 1e-15
    assert abs(1 / g["a2"] - g["lambda_star_per_kappa"]) < 1e-5
    lam = g["sec41"]["kappa"] / g["a2"]
    assert abs(lam - g["sec41"]["lambda_star"]) < 1e-4
    assert abs(a1 / lam - g["sec41"]["d0"]) < 1e-4           # d0 = a1 W0 / lambda
    assert abs(a1 / g["sec42"]["lambda_star"] - g["sec42"]["d0"]) < 1e-4
