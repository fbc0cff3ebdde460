"""Pins for the oracle's Neumann path (Eq. 3.19, Sec. 3.2.6): the interior
normal derivative extracted from the 6x6 Taylor system, and the Neumann
boundary value problem solved through the BIE of Eq. 3.19 with the
interface problem of Eq. 3.30 (Phi = 0, Psi = psi).

* The extraction is exact for quadratics: U = q1 on Omega-side stencil
  points and q2 elsewhere, with the jumps of q1 - q2 at the node, gives
  d_n q1 exactly (the Taylor system holds without remainder).
* The BVP: Delta u - kappa u = f in Omega, d_n u = g_N on Gamma, with a
  manufactured u, converges at second order on average (errors measured at
  the grid nodes inside Omega), the observed order band of the paper's
  Neumann heat example (its Table 2: ratios 3.96, 3.49, 4.03).
"""

import math

import numpy as np

import oracle
from paper_2404_14864_gb300 import workloads as W


def _quad(c):
    def q(x, y):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y

    def grad(x, y):
        return c[1] + 2 * c[3] * x + c[4] * y, c[2] + c[4] * x + 2 * c[5] * y

    return q, grad


def test_normal_extraction_exact_for_quadratics():
    desc = W.domain_desc(48, W.star())
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    rng = np.random.default_rng(3)
    q1, g1 = _quad(rng.standard_normal(6))
    q2, g2 = _quad(rng.standard_normal(6))
    inside = d.inside[1:-1, 1:-1]
    U = np.where(inside, q1(X, Y), q2(X, Y))
    # jumps of q1 - q2 at the boundary nodes: value, gradient, Hessian
    zx, zy = d.zx, d.zy
    dq = q1(zx, zy) - q2(zx, zy)
    gx1, gy1 = g1(zx, zy)
    gx2, gy2 = g2(zx, zy)
    q1c = _coeffs(q1)
    q2c = _coeffs(q2)
    J = np.stack([dq, gx1 - gx2, gy1 - gy2,
                  np.full(d.nb, 2 * (q1c[3] - q2c[3])), np.full(d.nb, q1c[4] - q2c[4]),
                  np.full(d.nb, 2 * (q1c[5] - q2c[5]))], axis=1)
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    dn = oracle.extraction(d, U, J, normal=True)
    assert np.abs(dn - (gx1 * t2 - gy1 * t1)).max() <= 1e-11
    # and the value extraction from the same system
    assert np.abs(oracle.extraction(d, U, J) - q1(zx, zy)).max() <= 1e-12


def _coeffs(q):
    # recover the six coefficients of a quadratic from its values
    pts = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    A = np.array([[1, x, y, x * x, x * y, y * y] for x, y in pts], dtype=float)
    b = np.array([q(x, y) for x, y in pts], dtype=float)
    return np.linalg.solve(A, b)


def _neumann_err(M, kappa=10.0):
    desc = W.domain_desc(M, W.star())
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    m = d.interior_inside()
    u = lambda x, y: np.sin(0.6 * x + 0.8 * y)
    Ft = np.where(m, -(1.0 + kappa) * u(X, Y), 0.0)
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    cz = np.cos(0.6 * d.zx + 0.8 * d.zy)
    gN = 0.6 * cz * t2 - 0.8 * cz * t1
    b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb), Ft)
    psi, it, res, ok = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), b, None, 1e-12,
                                    50, 500)
    assert ok
    up, U = oracle.interface_solve(d, kappa, np.zeros(d.nb), Ft, psi, normal=True)
    # the extracted normal derivative of the solution is the Neumann data
    assert np.abs(up - gN).max() <= 1e-9 * np.abs(gN).max()
    return np.abs(U - u(X, Y))[m].max()


def test_neumann_bvp_second_order():
    e = [_neumann_err(M) for M in (32, 64, 128, 256)]
    order = math.log2(e[0] / e[-1]) / 3.0
    assert order > 1.8, (e, order)
    assert all(e[i + 1] < e[i] for i in range(3)), e
    assert e[-1] < 3e-4, e


def _heat_neumann_err(M):
    """Neumann heat steps on the paper's Ex. 2 solution
    u = exp(-t) sin(0.6 x + 0.8 y) (u_t = Delta u), star r = 1 + 0.2 sin 5t in
    [-1.5, 1.5]^2, tau = 16 / M as its Table 2, T = 1."""
    desc = W.domain_desc(M, W.star(1.0, 0.2, 5), lo=-1.5, hi=1.5)
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    u = lambda t: math.exp(-t) * np.sin(0.6 * X + 0.8 * Y)
    gN = lambda t: math.exp(-t) * np.cos(0.6 * d.zx + 0.8 * d.zy) * (0.6 * t2 - 0.8 * t1)
    tau = 16.0 / M
    n = int(round(1.0 / tau))
    st = oracle.HeatStepper(d, tau, 1e-11, bc="neumann")
    st.init(u(0), -u(0))
    for k in range(n):
        U = st.step(gN((k + 1) * tau))
    return np.abs(U - u(n * tau))[d.interior_inside()].max()


def test_neumann_heat_stepper_converges():
    # the paper prints 8.60e-3 and 2.17e-3 at 64 and 128 on its heart domain
    e = [_heat_neumann_err(M) for M in (32, 64, 128)]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e
    assert e[2] < 2.2e-3, e


def test_neumann_bvp_complex_kappa_converges():
    """Complex kappa (the Schroedinger steps' kappa = 2i/tau is complex):
    u = (1 + 0.5i) sin(0.6 x + 0.8 y), kappa = 10 + 20i."""
    kappa = 10.0 + 20.0j
    e = []
    for M in (32, 64, 128):
        desc = W.domain_desc(M, W.star())
        d = oracle.make_domain(desc)
        X, Y = W.grid_xy(desc)
        m = d.interior_inside()
        c = 1.0 + 0.5j
        u = c * np.sin(0.6 * X + 0.8 * Y)
        Ft = np.where(m, -(1.0 + kappa) * u, 0.0)
        t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
        cz = c * np.cos(0.6 * d.zx + 0.8 * d.zy)
        gN = 0.6 * cz * t2 - 0.8 * cz * t1
        b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb, dtype=complex), Ft)
        psi, it, res, ok = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), b, None,
                                        1e-12, 50, 500)
        assert ok
        _, U = oracle.interface_solve(d, kappa, np.zeros(d.nb, dtype=complex), Ft, psi)
        e.append(np.abs(U - u)[m].max())
    assert e[0] / e[1] > 2.5 and e[1] / e[2] > 1.5, e
    assert e[2] < 2e-3, e
