"""Pins of the oracle's values of f on Gamma (the third row of the 3x3
jump system, Sec. 3.2.5, with the reading of f on Gamma the paper leaves
open: linear extrapolation along the cut edge at intersections, the
nearest Omega-side extraction-stencil point at boundary nodes).

- edge_f_gamma reproduces a linear f exactly at every intersection whose
  extrapolation node lies in Omega (a sign or offset error in the
  extrapolation breaks this), and is within |grad f| h elsewhere;
- node_f_gamma returns a constant f exactly (it never reads a point
  outside Omega, where f-tilde is zero), is within 1.6 |grad f| h of a
  linear f at the node, and converges at first order for a smooth f.
"""

import numpy as np

import oracle
from oracle.interface import edge_f_gamma, node_f_gamma, extraction_stencil
from paper_2404_14864_gb300 import workloads as W


def _linear(d, a=0.3, b=1.0, c=2.0):
    f = lambda x, y: a + b * x + c * y
    X, Y = np.meshgrid(d.x[1:-1], d.x[1:-1])
    Ft = np.where(d.interior_inside(), f(X, Y), 0.0)
    return f, Ft, np.hypot(b, c)


def _intersections(d):
    horiz = d.edge_dir == 0
    ex = np.where(horiz, d.edge_coord, d.x[d.edge_i])
    ey = np.where(horiz, d.x[d.edge_j], d.edge_coord)
    return ex, ey


def test_edge_f_gamma_exact_for_linear_f():
    for desc in (W.domain_desc(64, W.star()), W.domain_desc(96, W.ellipse()),
                 W.domain_desc(80, W.flower())):
        d = oracle.make_domain(desc)
        f, Ft, g = _linear(d)
        got = edge_f_gamma(d, Ft)
        ex, ey = _intersections(d)
        want = f(ex, ey)
        # which intersections had their second node p2 in Omega
        horiz = d.edge_dir == 0
        p_in = d.inside[d.edge_j, d.edge_i]
        pi_ = np.where(p_in, d.edge_i, d.edge_i + horiz)
        pj = np.where(p_in, d.edge_j, d.edge_j + (~horiz))
        step = np.where(p_in, -1, 1)
        ok = d.inside[np.where(horiz, pj, pj + step), np.where(horiz, pi_ + step, pi_)]
        assert ok.mean() > 0.8
        assert np.abs(got - want)[ok].max() <= 1e-12
        assert np.abs(got - want)[~ok].max(initial=0.0) <= g * d.h * (1 + 1e-12)


def test_node_f_gamma_constant_and_linear():
    for desc in (W.domain_desc(64, W.star()), W.domain_desc(96, W.ellipse()),
                 W.domain_desc(80, W.flower())):
        d = oracle.make_domain(desc)
        Fc = np.where(d.interior_inside(), 7.0, 0.0)
        assert np.array_equal(node_f_gamma(d, Fc), np.full(d.nb, 7.0))
        f, Ft, g = _linear(d)
        err = np.abs(node_f_gamma(d, Ft) - f(d.zx, d.zy))
        assert err.max() <= 1.6 * g * d.h
        # the point used is one of the node's six stencil points, inside
        si, sj = extraction_stencil(d)
        X, Y = np.meshgrid(d.x, d.x)
        vals = np.where(d.inside[sj, si], f(X[sj, si], Y[sj, si]), np.nan)
        got = node_f_gamma(d, Ft)
        assert all(np.any(np.isclose(vals[k], got[k], rtol=0, atol=1e-13)) for k in range(d.nb))


def test_node_f_gamma_first_order():
    errs = []
    for M in (64, 128, 256):
        desc = W.domain_desc(M, W.star())
        d = oracle.make_domain(desc)
        f = lambda x, y: np.sin(2 * x + 1) * np.cosh(y)
        X, Y = np.meshgrid(d.x[1:-1], d.x[1:-1])
        Ft = np.where(d.interior_inside(), f(X, Y), 0.0)
        errs.append(np.abs(node_f_gamma(d, Ft) - f(d.zx, d.zy)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.4 < r1 < 3.0 and 1.4 < r2 < 3.0, errs
