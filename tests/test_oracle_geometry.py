"""Pins for the oracle's geometry (Procedure 1 of Sec. 3.3): intersections
against closed forms, node classification against a brute-force scan,
curvature against textbook formulas."""

import math

import numpy as np
import pytest

import oracle

STAR = {"kind": "polar", "cx": 0.0, "cy": 0.0, "r0": 0.5, "eps": 0.1, "k": 5, "phase": 0.0}
ELLIPSE = {"kind": "ellipse", "cx": 0.0, "cy": 0.0, "a": 0.7, "b": 0.4, "alpha": math.pi / 6}


def _dom(M, curve, nb=None, lo=-1.0, hi=1.0):
    return oracle.make_domain({"M": M, "lo": lo, "hi": hi, "nb": nb or 2 * M, "curve": curve})


@pytest.mark.parametrize("M", [32, 61])
def test_circle_intersections_closed_form(M):
    r, cx, cy = 0.55, 0.031, -0.017
    d = _dom(M, {"kind": "polar", "cx": cx, "cy": cy, "r0": r, "eps": 0.0, "k": 1, "phase": 0.0})
    assert d.n_edges > 0
    for e in range(d.n_edges):
        i, j, dr, c = d.edge_i[e], d.edge_j[e], d.edge_dir[e], d.edge_coord[e]
        if dr == 0:
            y = d.x[j]
            roots = cx + np.array([-1.0, 1.0]) * math.sqrt(r * r - (y - cy) ** 2)
            lo_, hi_ = d.x[i], d.x[i + 1]
        else:
            x = d.x[i]
            roots = cy + np.array([-1.0, 1.0]) * math.sqrt(r * r - (x - cx) ** 2)
            lo_, hi_ = d.x[j], d.x[j + 1]
        root = roots[(roots >= lo_ - 1e-15) & (roots <= hi_ + 1e-15)]
        assert len(root) == 1
        assert abs(c - root[0]) < 1e-14
        px, py = (c, d.x[j]) if dr == 0 else (d.x[i], c)
        assert abs(d.edge_theta[e] - (math.atan2(py - cy, px - cx) % (2 * math.pi))) < 1e-14


@pytest.mark.parametrize("curve", [STAR, ELLIPSE])
def test_intersection_points_lie_on_curve_and_edge(curve):
    d = _dom(64, curve)
    zx, zy = d.curve.z(d.edge_theta)
    for e in range(d.n_edges):
        i, j, dr, c = d.edge_i[e], d.edge_j[e], d.edge_dir[e], d.edge_coord[e]
        if dr == 0:
            assert d.x[i] <= c <= d.x[i + 1]
            assert abs(zx[e] - c) < 1e-13 and abs(zy[e] - d.x[j]) < 1e-13
        else:
            assert d.x[j] <= c <= d.x[j + 1]
            assert abs(zy[e] - c) < 1e-13 and abs(zx[e] - d.x[i]) < 1e-13


@pytest.mark.parametrize("curve", [STAR, ELLIPSE])
def test_classification_brute_force(curve):
    M = 40
    d = _dom(M, curve)
    for j in range(M + 1):
        for i in range(M + 1):
            x, y = d.x[i], d.x[j]
            ins = bool(d.curve.level(x, y) < 0.0)
            assert ins == bool(d.inside[j, i])
    for j in range(1, M):
        for i in range(1, M):
            irr = any(d.inside[j + dj, i + di] != d.inside[j, i]
                      for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)))
            assert irr == bool(d.irregular[j, i])
    # every cut edge joins two irregular nodes; edge count = status changes
    n_h = sum(d.inside[j, i] != d.inside[j, i + 1] for j in range(M + 1) for i in range(M))
    n_v = sum(d.inside[j, i] != d.inside[j + 1, i] for j in range(M) for i in range(M + 1))
    assert d.n_edges == n_h + n_v


def test_inside_area():
    d = _dom(256, ELLIPSE)
    area = d.inside.sum() * d.h ** 2
    assert abs(area - math.pi * 0.7 * 0.4) < 0.01


def _curvature_polar(c, t):
    r = c["r0"] + c["eps"] * np.sin(c["k"] * t + c["phase"])
    dr = c["eps"] * c["k"] * np.cos(c["k"] * t + c["phase"])
    d2r = -c["eps"] * c["k"] ** 2 * np.sin(c["k"] * t + c["phase"])
    return (r * r + 2 * dr * dr - r * d2r) / (r * r + dr * dr) ** 1.5


def _curvature_ellipse(c, t):
    a, b = c["a"], c["b"]
    return a * b / (a * a * np.sin(t) ** 2 + b * b * np.cos(t) ** 2) ** 1.5


@pytest.mark.parametrize("curve,kfun", [(STAR, _curvature_polar), (ELLIPSE, _curvature_ellipse)])
def test_tangent_derivative_is_curvature_normal(curve, kfun):
    from oracle.interface import tangent_data
    d = _dom(64, curve)
    t = np.linspace(0.0, 2 * math.pi, 97)
    t1, t2, t1p, t2p = tangent_data(d, t)
    assert np.allclose(t1 ** 2 + t2 ** 2, 1.0, atol=1e-14)
    kap = kfun(curve, t)
    # CCW curve: d tau / ds = curvature * (-tau2, tau1)
    assert np.abs(t1p - kap * (-t2)).max() < 1e-12
    assert np.abs(t2p - kap * t1).max() < 1e-12
