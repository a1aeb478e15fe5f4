"""Pins of the oracle's diagnostics: the tip radius and the total-solute sum.

The tip position and radius follow the tip definition of the method's readings (the
first phi = 0 crossing along +x from the seed centre, linearly interpolated; the radius
from a least-squares parabola x(j) = x_tip - j^2/(2 rho) through the crossings of rows
j = +-1..+-4 in the xy and xz planes, averaged).  The total solute is
sum zeta(phi) (1 + (1-k) U) with zeta = ((1+k) - (1-k) phi)/2, the quantity whose
integral Eq. (Concentration_Echebarria) conserves with zero-flux walls (c / c_inf of
Sec. 2).  Each test checks the oracle against a result fixed without its code: an exact
parabola, a closed-form band for a sphere, the values at uniform phases, and the
conservation law of the PDE.
"""
import numpy as np
import pytest

import oracle

ROWS = np.array([j for j in range(-4, 5) if j != 0], dtype=np.float64)


def _sim_with_phi(phi, k=0.15, U=None, lattices=(19, 19, 0)):
    """An oracle simulation whose moments are the given phi (and U) fields: populations
    g = w phi and h = (A + B q/zeta) U, whose zeroth moments are phi and U."""
    nz, ny, nx = phi.shape
    qp, qu, _ = lattices
    s = oracle.Sim((nx, ny, nz), lattices, params=oracle.make_params(k=k))
    _, wp, *_ = oracle.lattice(qp)
    _, _, Au, Bu, _, _ = oracle.lattice(qu)
    if U is None:
        U = np.zeros_like(phi)
    q = 0.5 * (1 - phi)
    zeta = 0.5 * ((1 + k) - (1 - k) * phi)
    g = wp[:, None, None, None] * phi[None]
    h = (Au[:, None, None, None] + Bu[:, None, None, None] * (q / zeta)[None]) * U[None]
    s.set_state(g, h, None)
    return s


def _linear_crossing_field(shape, centre, X):
    """phi = s (X(y, z) - x): linear along x, so the interpolated phi = 0 crossing of every
    row is exactly X(y, z)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return 0.37 * (X(y - centre[1], z - centre[2]) - x)


def test_tip_radius_of_exact_parabola():
    """Crossings on x = x_t - j^2/(2 rho_a) + beta j in the xy plane and
    x = x_t - j^2/(2 rho_b) in the xz plane: the least-squares parabola recovers rho_a and
    rho_b exactly (the odd tilt beta cancels over the symmetric rows), and the radius is
    their mean.  A factor-2 slip in 1/(2 rho), a sign flip of one row, a missing row or a
    wrong plane average all miss the closed form by far more than rounding."""
    shape, c = (40, 13, 13), (6, 6, 6)
    xt, ra, rb, beta = 29.3, 6.5, 11.0, 0.21

    def X(dy, dz):
        return xt - dy * dy / (2 * ra) + beta * dy - dz * dz / (2 * rb)

    s = _sim_with_phi(_linear_crossing_field(shape, c, X))
    x_tip, rho = s.tip(c)
    assert abs(x_tip - xt) < 1e-12
    assert abs(rho - 0.5 * (ra + rb)) < 1e-10 * ra


@pytest.mark.parametrize("axis", [1, 2])
def test_tip_along_other_axes_of_exact_parabola(axis):
    """The same exact-parabola pin for a scan along +y or +z: the crossings lie on
    t = t_tip - j^2/(2 rho_b) in the plane of the scan axis and each other axis b."""
    n, c = (13, 13, 13), [6, 6, 6]
    shape = list(n)
    shape[axis] = 40
    others = [b for b in range(3) if b != axis]
    rb = {others[0]: 6.5, others[1]: 11.0}
    tt = 29.3
    Z, Y, X = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
    P = (X, Y, Z)
    T = tt - sum((P[b] - c[b]) ** 2 / (2 * rb[b]) for b in others)
    s = _sim_with_phi(0.37 * (T - P[axis]))
    t_tip, rho = s.tip(c, axis=axis)
    assert abs(t_tip - tt) < 1e-12
    assert abs(rho - 0.5 * (rb[others[0]] + rb[others[1]])) < 1e-10 * 6.5


def test_tip_radius_of_exact_parabola_2d():
    """On an nz = 1 grid only the xy plane exists: the radius is that plane's fit alone."""
    shape, c = (36, 11, 1), (5, 5, 0)
    xt, ra = 24.75, 4.25
    s = _sim_with_phi(_linear_crossing_field(shape, c, lambda dy, dz: xt - dy * dy / (2 * ra)),
                      lattices=(9, 5, 0))
    x_tip, rho = s.tip(c)
    assert abs(x_tip - xt) < 1e-12
    assert abs(rho - ra) < 1e-10 * ra
    # along the grid's y axis: the plane is the same, the roles of the axes swap
    yt, ry = 7.5, 3.0
    Y, X = np.meshgrid(np.arange(24), np.arange(17), indexing="ij")
    s2 = _sim_with_phi((0.37 * (yt - (X - 8) ** 2 / (2 * ry) - Y))[None], lattices=(9, 5, 0))
    y_tip, rho2 = s2.tip((8, 0, 0), axis=1)
    assert abs(y_tip - yt) < 1e-12
    assert abs(rho2 - ry) < 1e-10 * ry


@pytest.mark.parametrize("R", [20.0, 40.0])
def test_tip_radius_of_diffuse_sphere(R):
    """Seed profile phi = tanh((R - r) dx/(sqrt2 W0)) of a sphere of radius R (the initial
    condition of Sec. 4).  Two derived parts:
      - the parabola fitted to the exact circle crossings sqrt(R^2 - j^2) gives
        rho_c = R / (1 + S6/(4 R^2 S4) + S8/(8 R^4 S4) + ...) with S_m = sum_j j^m (series of
        R - sqrt(R^2 - j^2)); the first two terms bound it within 1e-5 R here;
      - linear interpolation of the tanh profile moves each crossing by at most
        e = cosh^2(a)/8 (j^2/(r^2 x) + 2 a tanh a), a = dx/(sqrt2 W0) (interpolation remainder
        |f''/(2 f')| |(x - x_i)(x - x_{i+1})| with the row's f = tanh(a (R - r(x)))), so rho
        moves by at most rho sum_j j^2 (e_0 + e_j) / sum_j j^2 (x_t - x_j).
    dx = 0.1 W0 resolves the profile over 14 nodes."""
    dx, W0 = 0.1, 1.0
    a = dx / (np.sqrt(2) * W0)
    cx, c = 3, 6
    nx, ny = int(cx + R + 6), 2 * c + 1
    z, y, x = np.meshgrid(np.arange(ny), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - cx) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi = np.tanh((R - r) * a)
    s = _sim_with_phi(phi)
    x_tip, rho = s.tip((cx, c, c))
    S4, S6, S8 = (np.sum(ROWS ** m) for m in (4, 6, 8))
    rho_c = R / (1 + S6 / (4 * R * R * S4) + S8 / (8 * R ** 4 * S4))
    xj = np.sqrt(R * R - ROWS ** 2)
    e = np.cosh(a) ** 2 / 8 * (ROWS ** 2 / (R * R * xj) + 2 * a * np.tanh(a))
    e0 = np.cosh(a) ** 2 / 8 * 2 * a * np.tanh(a)
    num = np.sum(ROWS ** 2 * (R - xj))
    tol = rho_c * np.sum(ROWS ** 2 * (e0 + e)) / (num - np.sum(ROWS ** 2 * (e0 + e))) + 1e-5 * R
    assert abs(x_tip - (cx + R)) <= e0 + 1e-12
    assert abs(rho - rho_c) <= tol, (rho, rho_c, tol)
    assert tol < 0.02 * R  # the band is narrow enough to see a wrong factor or sign


@pytest.mark.parametrize("phi0", [-1.0, 0.0, 1.0])
def test_total_solute_of_uniform_states(phi0):
    """zeta(phi) = ((1+k) - (1-k) phi)/2 is 1 in the liquid, k in the solid and (1+k)/2 at
    phi = 0, and the solute of a uniform state is n zeta (1 + (1-k) U): with two values of
    U this fixes both the phase factor and the (1-k) U factor of the sum."""
    k, n = 0.15, (9, 7, 5)
    zeta = {-1.0: 1.0, 0.0: 0.5 * (1 + k), 1.0: k}[phi0]
    for U0 in (-0.55, 0.3):
        phi = np.full(n[::-1], phi0)
        s = _sim_with_phi(phi, k=k, U=np.full(n[::-1], U0))
        tot = s.sums()[3]
        expect = np.prod(n) * zeta * (1 + (1 - k) * U0)
        assert abs(tot - expect) < 1e-12 * np.prod(n), (phi0, U0, tot, expect)


def _solute_drift(n, antitrapping=1, L=9.6, R=3.2, T=1.6):
    """Relative drift of the total solute over a growing seed's run to time T on an n^3 box
    at fixed dt/dx^2, with the moving interface (lambda != 0, anti-trapping on)."""
    dx = L / n
    dt = 0.06 * dx * dx
    p = oracle.make_params(eps1=0.02, dx=dx, dt=dt, D=1.0, lam=1.0 / 0.6267, antitrapping=antitrapping)
    s = oracle.Sim((n, n, n), (19, 19, 0), params=p)
    s.init_seed([[(n - 1) / 2] * 3], [R / dx], U0=-0.5)
    a0 = s.sums()
    s.step(int(round(T / dt)))
    a1 = s.sums()
    return (a1[3] - a0[3]) / a0[3], (a1[0] - a0[0]) / n ** 3


def test_total_solute_drift_shrinks_under_refinement():
    """Eq. (Concentration_Echebarria) is a conservation law: d/dt of the integral of
    zeta(phi) (1 + (1-k) U) is the flux through zero-flux walls, 0, for any interface motion.
    The LB scheme advances the reformulated U equation, so the total solute drifts only by
    its truncation error, which must fall under refinement while the solid fraction changes
    by O(1).  A wrong phase factor zeta or a wrong (1-k) U factor in the sum breaks this:
    the summed quantity then follows the growth of the solid instead."""
    d12, grow12 = _solute_drift(12)
    d24, grow24 = _solute_drift(24)
    assert abs(grow12) > 0.05 and abs(grow24) > 0.05      # the seed did grow
    assert abs(d12) < 0.1 * abs(grow12)
    assert abs(d12) / abs(d24) > 3.0, (d12, d24)          # measured ratio 3.6 (between 2 and 4)
