"""Pins of the oracle Richardson iteration (Eq. 3.21).

Eq. 3.21 is phi_{k+1} = phi_k + gamma (b - A phi_k) with A = 1/2 I + W.
For a normal A and b along one eigenvector (eigenvalue lam), every
residual is (1 - gamma lam)^k b exactly, so the iteration count is a closed
form; on the assembled KFBI operator the fixed point must be the solution
of the linear system and the count must sit between the bounds that the
spectral radius of I - gamma A sets.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _normal_matrix(n, lams, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(lams) @ Q.T, Q


@pytest.mark.parametrize("gamma", [0.5, 0.9, 1.0])
def test_richardson_count_is_the_closed_form_on_an_eigenvector(gamma):
    n = 40
    lams = np.linspace(0.4, 0.6, n)
    A, Q = _normal_matrix(n, lams, 1)
    for idx in (0, n - 1):
        b = Q[:, idx]
        lam = lams[idx]
        tol = 1e-10
        x, it, rel, ok = oracle.richardson(lambda v: A @ v, b, gamma=gamma, tol=tol)
        assert ok
        expected = math.ceil(math.log(tol) / math.log(abs(1.0 - gamma * lam)))
        assert it == expected, (it, expected)
        np.testing.assert_allclose(x, b / lam, rtol=0, atol=2 * tol / lam)


def test_richardson_solves_the_assembled_kfbi_system():
    desc = W.domain_desc(32, W.star(), nb=64)
    d = oracle.make_domain(desc)
    kappa = 2.0 / d.h
    nb = d.nb
    A = np.zeros((nb, nb))
    for j in range(nb):
        e = np.zeros(nb)
        e[j] = 1.0
        A[:, j] = oracle.apply_operator(d, kappa, e)
    b = np.cos(2 * d.theta) + 0.3 * np.sin(3 * d.theta)
    gamma, tol = 0.9, 1e-11
    x, it, rel, ok = oracle.richardson(lambda v: oracle.apply_operator(d, kappa, v), b, gamma=gamma,
                                       tol=tol)
    assert ok and rel <= tol
    x_lu = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.abs(x - x_lu).max() <= 10 * cond * tol * np.abs(x_lu).max()
    # the count is bounded by the spectral radius rho of I - gamma A:
    # ||r_k|| <= ||V|| ||V^-1|| rho^k ||r_0|| (eigenvector matrix V), and at
    # least the slowest component's decay is needed
    ev, V = np.linalg.eig(A)
    rho = np.abs(1.0 - gamma * ev).max()
    kv = np.linalg.cond(V)
    upper = math.ceil(math.log(tol / kv) / math.log(rho))
    assert it <= upper
    # agrees with GMRES on the same system
    x_g, it_g, rel_g, ok_g = oracle.gmres(lambda v: A @ v, b, tol=1e-13)
    assert ok_g and it_g < it
    assert np.abs(x - x_g).max() <= 10 * cond * tol * np.abs(x_g).max()


def test_richardson_zero_rhs_and_divergence():
    A = np.diag([0.5, 1.5])
    x, it, rel, ok = oracle.richardson(lambda v: A @ v, np.zeros(2), gamma=0.9)
    assert ok and it == 0 and not np.any(x)
    # gamma beyond 2 / lam_max diverges: the iteration stops unconverged
    x, it, rel, ok = oracle.richardson(lambda v: A @ v, np.ones(2), gamma=1.9, tol=1e-10, maxit=200)
    assert not ok and it == 200


def test_richardson_stepper_matches_gmres_stepper():
    # heat steps on a circle: either solver of the density equation gives the
    # same fields (to the solver tolerance), and the Richardson counts follow
    # the spectral radius (more iterations for smaller gamma)
    desc = W.domain_desc(32, W.star(1.0, 0.0, 1), lo=-1.5, hi=1.5)
    d = oracle.make_domain(desc)
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    out = {}
    for solver, gamma in (("gmres", 0.0), ("richardson", 0.5), ("richardson", 1.5)):
        orc = oracle.HeatStepper(d, d.h, 1e-12, solver=solver, gamma=gamma, maxit=5000)
        orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.src(X, Y, 0) + ex.src(X, Y, d.h))
        for k in range(3):
            t1 = (k + 1) * d.h
            U = orc.step(ex.u(zx, zy, t1), ex.src(X, Y, t1) + ex.src(X, Y, t1 + d.h))
        out[(solver, gamma)] = (U, orc.iters)
    m = d.interior_inside()
    Ug = out[("gmres", 0.0)][0]
    for key in (("richardson", 0.5), ("richardson", 1.5)):
        assert np.abs(out[key][0] - Ug)[m].max() <= 1e-9 * np.abs(Ug[m]).max()
    assert all(a > b for a, b in zip(out[("richardson", 0.5)][1], out[("richardson", 1.5)][1]))
