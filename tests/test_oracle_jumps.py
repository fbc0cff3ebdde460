"""Pins for the oracle's jump calculation (Sec. 3.2.5), correction (Sec. 3.2.4)
and boundary extraction (Sec. 3.2.6, Eq. 3.36), against analytic functions."""

import math

import numpy as np
import pytest

import oracle
from oracle.interface import tangent_data

STAR = {"kind": "polar", "cx": 0.0, "cy": 0.0, "r0": 0.5, "eps": 0.1, "k": 5, "phase": 0.0}
ELLIPSE = {"kind": "ellipse", "cx": 0.02, "cy": -0.01, "a": 0.7, "b": 0.4, "alpha": math.pi / 6}
FLOWER = {"kind": "polar", "cx": 0.0, "cy": 0.0, "r0": 0.6, "eps": 0.15, "k": 4, "phase": math.pi / 2}


def _dom(M, curve, nb=None):
    return oracle.make_domain({"M": M, "lo": -1.0, "hi": 1.0, "nb": nb or 2 * M, "curve": curve})


# w(x, y) = sin(1.3 x + 0.4) exp(0.7 y) + x^2 y / 2 and its derivatives
def w_all(x, y):
    s, c, e = np.sin(1.3 * x + 0.4), np.cos(1.3 * x + 0.4), np.exp(0.7 * y)
    return (s * e + 0.5 * x * x * y, 1.3 * c * e + x * y, 0.7 * s * e + 0.5 * x * x,
            -1.69 * s * e + y, 0.91 * c * e + x, 0.49 * s * e)


# v(x, y) = cos(x) y + 0.3 (an unrelated smooth exterior function)
def v_all(x, y):
    return (np.cos(x) * y + 0.3, -np.sin(x) * y, np.cos(x),
            -np.cos(x) * y, -np.sin(x), 0.0 * x)


def test_lagrange6_exact_for_quintics():
    rng = np.random.default_rng(7)
    s = rng.uniform(0.0, 1.0, 25)
    w0, w1, w2 = oracle.lagrange6_weights(s)
    nodes = np.arange(-2, 4, dtype=float)
    for deg in range(6):
        c = rng.standard_normal(deg + 1)
        p = np.polynomial.Polynomial(c)
        assert np.allclose(w0 @ p(nodes), p(s), atol=1e-12)
        assert np.allclose(w1 @ p(nodes), p.deriv(1)(s), atol=1e-11)
        assert np.allclose(w2 @ p(nodes), p.deriv(2)(s), atol=1e-10)
    # at s = 0 the value weights are the unit vector on local node 0
    w0, _, _ = oracle.lagrange6_weights(np.zeros(1))
    assert np.allclose(w0[0], [0, 0, 1, 0, 0, 0], atol=1e-15)


@pytest.mark.parametrize("curve", [STAR, ELLIPSE])
def test_density_derivatives_along_arc_length(curve):
    """phi = w restricted to Gamma: phi_s = grad w . t, phi_ss = t^T H t + grad w . t_s."""
    errs = []
    for nb in (256, 512, 1024):
        d = _dom(64, curve, nb)
        zx, zy = d.zx, d.zy
        W = w_all(zx, zy)
        phi = W[0]
        th = np.random.default_rng(3).uniform(0, 2 * math.pi, 40)
        g, g_s, g_ss = oracle.density_derivatives(d, phi, th)
        px, py = d.curve.z(th)
        Wt = w_all(px, py)
        t1, t2, t1p, t2p = tangent_data(d, th)
        ex_s = Wt[1] * t1 + Wt[2] * t2
        ex_ss = t1 * t1 * Wt[3] + 2 * t1 * t2 * Wt[4] + t2 * t2 * Wt[5] + Wt[1] * t1p + Wt[2] * t2p
        errs.append((np.abs(g - Wt[0]).max(), np.abs(g_s - ex_s).max(), np.abs(g_ss - ex_ss).max()))
    e = np.array(errs)
    assert e[-1, 0] < 1e-10 and e[-1, 1] < 1e-8 and e[-1, 2] < 5e-6
    # orders in the node spacing: value 6, first derivative 5, second derivative 4
    assert e[1, 0] / e[2, 0] > 40.0
    assert e[1, 1] / e[2, 1] > 20.0
    assert e[1, 2] / e[2, 2] > 10.0


def test_jump_matrix_determinant_is_minus_one():
    ang = np.random.default_rng(11).uniform(0, 2 * math.pi, 200)
    A = oracle.jump_matrix3(np.cos(ang), np.sin(ang))
    assert np.allclose(np.linalg.det(A), -1.0, atol=1e-13)


@pytest.mark.parametrize("curve", [STAR, ELLIPSE, FLOWER])
@pytest.mark.parametrize("kappa", [0.0, 7.5, 2.0 + 3.0j])
def test_jumps_reproduce_analytic_jumps(curve, kappa):
    """u+ = w in Omega, u- = 0 outside: [u] = w, [u_n] = dw/dn, [f] = (Delta - kappa) w;
    the computed jumps equal w's derivatives on Gamma."""
    d = _dom(64, curve, 1024)
    Wn = w_all(d.zx, d.zy)
    t1, t2, _, _ = tangent_data(d, d.theta)
    phi = Wn[0] * (1.0 + 0j if isinstance(kappa, complex) else 1.0)
    psi = Wn[1] * t2 - Wn[2] * t1
    # at the boundary nodes
    fg = (Wn[3] + Wn[5]) - kappa * Wn[0]
    J = oracle.jumps_at(d, None, phi, fg, kappa, psi, node_k=np.arange(d.nb))
    for c in range(6):
        tol = (1e-14, 1e-8, 1e-8, 5e-5, 5e-5, 5e-5)[c]
        assert np.abs(J[:, c] - Wn[c]).max() < tol, c
    # at the cut-edge intersections
    px, py = d.curve.z(d.edge_theta)
    We = w_all(px, py)
    fe = (We[3] + We[5]) - kappa * We[0]
    Je = oracle.jumps_at(d, d.edge_theta, phi, fe, kappa, psi)
    for c in range(6):
        tol = (1e-10, 1e-8, 1e-8, 5e-5, 5e-5, 5e-5)[c]
        assert np.abs(Je[:, c] - We[c]).max() < tol, c


def _exact_edge_jumps(d):
    px, py = d.curve.z(d.edge_theta)
    # exact intersection points (use the stored coordinate on the grid line)
    ex = np.where(d.edge_dir == 0, d.edge_coord, d.x[d.edge_i])
    ey = np.where(d.edge_dir == 0, d.x[d.edge_j], d.edge_coord)
    W, V = w_all(ex, ey), v_all(ex, ey)
    return np.stack([W[c] - V[c] for c in range(6)], axis=1)


@pytest.mark.parametrize("curve", [STAR, ELLIPSE])
def test_corrected_truncation_error_orders(curve):
    """Corrected five-point residual of a piecewise-smooth u: O(h) at irregular
    nodes, O(h^2) at regular nodes (Sec. 3.2.4)."""
    kappa = 3.0
    rows = []
    for M in (64, 128, 256):
        d = _dom(M, curve)
        X, Y = np.meshgrid(d.x, d.x)
        W, V = w_all(X, Y), v_all(X, Y)
        u = np.where(d.inside, W[0], V[0])
        Fg = np.where(d.inside, W[3] + W[5] - kappa * W[0], V[3] + V[5] - kappa * V[0])[1:-1, 1:-1]
        R = oracle.correction_rhs(d, Fg, _exact_edge_jumps(d))
        h = d.h
        lap = (u[1:-1, 2:] + u[1:-1, :-2] + u[2:, 1:-1] + u[:-2, 1:-1] - 4 * u[1:-1, 1:-1]) / h ** 2
        r = lap - kappa * u[1:-1, 1:-1] - R
        irr = d.irregular[1:-1, 1:-1]
        rows.append((np.abs(r[irr]).max(), np.abs(r[~irr]).max()))
        # uncorrected residual at irregular nodes is O(1/h^2)
        r0 = lap - kappa * u[1:-1, 1:-1] - Fg
        assert np.abs(r0[irr]).max() > 50.0 * np.abs(r[irr]).max()
    rows = np.array(rows)
    assert rows[0, 0] / rows[1, 0] > 1.6 and rows[1, 0] / rows[2, 0] > 1.6
    assert rows[0, 1] / rows[1, 1] > 3.2 and rows[1, 1] / rows[2, 1] > 3.2


@pytest.mark.parametrize("curve", [STAR, ELLIPSE, FLOWER])
def test_extraction_exact_for_quadratics(curve):
    def q1(x, y):
        return (1 + 2 * x - y + 0.5 * x * x + 0.3 * x * y - 0.7 * y * y,
                2 + x + 0.3 * y, -1 + 0.3 * x - 1.4 * y, 1.0, 0.3, -1.4)

    def q2(x, y):
        return (-0.5 + x + 3 * y - x * x + 0.2 * x * y + 0.1 * y * y,
                1 - 2 * x + 0.2 * y, 3 + 0.2 * x + 0.2 * y, -2.0, 0.2, 0.2)

    d = _dom(48, curve)
    X, Y = np.meshgrid(d.x, d.x)
    U = np.where(d.inside, q1(X, Y)[0], q2(X, Y)[0])[1:-1, 1:-1]
    A, B = q1(d.zx, d.zy), q2(d.zx, d.zy)
    jumps = np.stack([np.broadcast_to(np.asarray(A[c]) - np.asarray(B[c]), d.zx.shape)
                      for c in range(6)], axis=1)
    up = oracle.extraction(d, U, jumps)
    assert np.abs(up - A[0]).max() < 1e-12


def test_extraction_stencil_shape():
    d = _dom(64, STAR)
    si, sj = oracle.extraction_stencil(d)
    for k in range(d.nb):
        pts = set(zip(si[k].tolist(), sj[k].tolist()))
        assert len(pts) == 6
        # nearest node first, within half a cell
        assert abs(d.x[si[k, 0]] - d.zx[k]) <= 0.5 * d.h + 1e-15
        assert abs(d.x[sj[k, 0]] - d.zy[k]) <= 0.5 * d.h + 1e-15
