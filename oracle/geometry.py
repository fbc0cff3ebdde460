"""Oracle geometry: Procedure 1 of Sec. 3.3 (arXiv 2404.14864).

  (a) quasi-uniform points z_k on the interface Gamma,
  (b) a uniform Cartesian grid on the box B = [lo, hi]^2 (Sec. 3.2.4:
      x_i = lo + i h, h = (hi - lo) / M, i = 0..M),
  (c) regular / irregular node classification (Sec. 3.2.4: a node is
      irregular when one of its four stencil neighbours lies on the other
      side of Gamma),
  (d) intersections of Gamma with the grid lines.

Readings where the paper is silent (it fits its curves with cubic splines,
Sec. 4.1, and gives no node-classification tie rule):

* Curves are analytic.  ``polar``: z(t) = c + r(t) (cos t, sin t) with
  r(t) = r0 + eps * sin(k t + phase) (a star; phase = pi/2 gives the
  cos-flower; eps = 0 a circle).  ``ellipse``: z(t) = c + Rot(alpha)
  (a cos t, b sin t).  Both are traversed counter-clockwise, so the outward
  normal is n = (tau_2, -tau_1) as in Sec. 3.2.5.
* Boundary nodes are z_k = z(2 pi k / nb), k = 0..nb-1.
* A grid node p is inside Omega iff the level function L(p) < 0 strictly
  (L = |p - c| - r(angle of p - c) for polar curves, (x'/a)^2 + (y'/b)^2 - 1
  in the ellipse frame); L = 0 counts as outside.
* The intersection on a cut edge is found by bisection of L along the edge
  until the bracket cannot shrink further in float64.  Its curve parameter
  t* is recovered from the point (angle about c for polar curves,
  atan2(y'/b, x'/a) for the ellipse).
"""

import math

import numpy as np

TWO_PI = 2.0 * math.pi


class PolarCurve:
    """z(t) = c + r(t)(cos t, sin t),  r(t) = r0 + eps sin(k t + phase)."""

    def __init__(self, cx, cy, r0, eps, k, phase):
        self.cx, self.cy = float(cx), float(cy)
        self.r0, self.eps, self.k, self.phase = float(r0), float(eps), float(k), float(phase)

    def _r(self, t):
        return self.r0 + self.eps * np.sin(self.k * t + self.phase)

    def _dr(self, t):
        return self.eps * self.k * np.cos(self.k * t + self.phase)

    def _d2r(self, t):
        return -self.eps * self.k * self.k * np.sin(self.k * t + self.phase)

    def z(self, t):
        r = self._r(t)
        return self.cx + r * np.cos(t), self.cy + r * np.sin(t)

    def dz(self, t):
        r, dr = self._r(t), self._dr(t)
        c, s = np.cos(t), np.sin(t)
        return dr * c - r * s, dr * s + r * c

    def d2z(self, t):
        r, dr, d2r = self._r(t), self._dr(t), self._d2r(t)
        c, s = np.cos(t), np.sin(t)
        return d2r * c - 2.0 * dr * s - r * c, d2r * s + 2.0 * dr * c - r * s

    def level(self, x, y):
        dx, dy = x - self.cx, y - self.cy
        return np.hypot(dx, dy) - self._r(np.arctan2(dy, dx))

    def param_of(self, x, y):
        t = np.arctan2(y - self.cy, x - self.cx)
        return np.where(t < 0.0, t + TWO_PI, t)


class EllipseCurve:
    """z(t) = c + Rot(alpha) (a cos t, b sin t)."""

    def __init__(self, cx, cy, a, b, alpha):
        self.cx, self.cy = float(cx), float(cy)
        self.a, self.b, self.alpha = float(a), float(b), float(alpha)
        self.ca, self.sa = math.cos(self.alpha), math.sin(self.alpha)

    def _rot(self, u, v):
        return self.ca * u - self.sa * v, self.sa * u + self.ca * v

    def _unrot(self, x, y):
        dx, dy = x - self.cx, y - self.cy
        return self.ca * dx + self.sa * dy, -self.sa * dx + self.ca * dy

    def z(self, t):
        u, v = self._rot(self.a * np.cos(t), self.b * np.sin(t))
        return self.cx + u, self.cy + v

    def dz(self, t):
        return self._rot(-self.a * np.sin(t), self.b * np.cos(t))

    def d2z(self, t):
        return self._rot(-self.a * np.cos(t), -self.b * np.sin(t))

    def level(self, x, y):
        u, v = self._unrot(x, y)
        return (u / self.a) ** 2 + (v / self.b) ** 2 - 1.0

    def param_of(self, x, y):
        u, v = self._unrot(x, y)
        t = np.arctan2(v / self.b, u / self.a)
        return np.where(t < 0.0, t + TWO_PI, t)


def curve_from_desc(c):
    kind = c["kind"]
    if kind == "polar":
        return PolarCurve(c["cx"], c["cy"], c["r0"], c["eps"], c["k"], c.get("phase", 0.0))
    if kind == "ellipse":
        return EllipseCurve(c["cx"], c["cy"], c["a"], c["b"], c["alpha"])
    raise ValueError("unknown curve kind %r" % (kind,))


def _param(curve, x, y):
    """Curve parameter of a point on the curve, in [0, 2 pi)."""
    return float(curve.param_of(np.float64(x), np.float64(y)))


def _bisect_edge(curve, px, py, qx, qy, p_inside):
    """Root of L along the segment p -> q; returns the fraction t in (0, 1)."""
    t_in, t_out = (0.0, 1.0) if p_inside else (1.0, 0.0)
    for _ in range(200):
        tm = 0.5 * (t_in + t_out)
        if tm == t_in or tm == t_out:
            break
        if curve.level(px + tm * (qx - px), py + tm * (qy - py)) < 0.0:
            t_in = tm
        else:
            t_out = tm
    return 0.5 * (t_in + t_out)


class Domain:
    """Grid, interface discretisation and cut-edge data (Procedure 1)."""

    def __init__(self, desc):
        self.desc = desc
        self.M = int(desc["M"])
        self.lo, self.hi = float(desc["lo"]), float(desc["hi"])
        self.nb = int(desc["nb"])
        self.curve = curve_from_desc(desc["curve"])
        M = self.M
        self.h = (self.hi - self.lo) / M
        # (b) grid nodes x_i = lo + i h, i = 0..M (same along y).
        self.x = self.lo + self.h * np.arange(M + 1)
        # (a) boundary nodes, uniform in the curve parameter.
        self.dtheta = TWO_PI / self.nb
        self.theta = self.dtheta * np.arange(self.nb)
        self.zx, self.zy = self.curve.z(self.theta)
        # (c) inside mask over all (M+1)^2 nodes, indexed [j, i] (y, x).
        X, Y = np.meshgrid(self.x, self.x)  # X[j, i] = x_i, Y[j, i] = y_j
        self.inside = self.curve.level(X, Y) < 0.0
        if self.inside[0, :].any() or self.inside[-1, :].any() or \
                self.inside[:, 0].any() or self.inside[:, -1].any():
            raise ValueError("interface touches the box boundary")
        irr = np.zeros_like(self.inside)
        c = self.inside[1:-1, 1:-1]
        for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            nb_ = self.inside[1 + dj:M + dj, 1 + di:M + di]
            irr[1:-1, 1:-1] |= (c != nb_)
        self.irregular = irr
        # Stencils (correction and extraction) must stay on interior nodes:
        # inside nodes and boundary nodes keep two cells from the box edge.
        lim_lo, lim_hi = self.lo + 2.0 * self.h, self.hi - 2.0 * self.h
        if self.inside[:2, :].any() or self.inside[-2:, :].any() or \
                self.inside[:, :2].any() or self.inside[:, -2:].any() or \
                self.zx.min() < lim_lo or self.zx.max() > lim_hi or \
                self.zy.min() < lim_lo or self.zy.max() > lim_hi:
            raise ValueError("interface closer than 2h to the box boundary")
        # (d) cut edges.  Each record: (i, j) of the lower/left endpoint p,
        # direction 0 (edge along x, q = (i+1, j)) or 1 (along y, q = (i, j+1)),
        # the intersection coordinate along the edge's line, and t*.
        ei, ej, ed, ec, et = [], [], [], [], []
        hj, hi_ = np.nonzero(self.inside[:, :-1] != self.inside[:, 1:])
        for j, i in zip(hj.tolist(), hi_.tolist()):
            t = _bisect_edge(self.curve, self.x[i], self.x[j], self.x[i + 1], self.x[j],
                             bool(self.inside[j, i]))
            xi = self.x[i] + t * self.h
            ei.append(i); ej.append(j); ed.append(0); ec.append(xi)
            et.append(_param(self.curve, xi, self.x[j]))
        vj, vi = np.nonzero(self.inside[:-1, :] != self.inside[1:, :])
        for j, i in zip(vj.tolist(), vi.tolist()):
            t = _bisect_edge(self.curve, self.x[i], self.x[j], self.x[i], self.x[j + 1],
                             bool(self.inside[j, i]))
            eta = self.x[j] + t * self.h
            ei.append(i); ej.append(j); ed.append(1); ec.append(eta)
            et.append(_param(self.curve, self.x[i], eta))
        self.edge_i = np.array(ei, dtype=np.int64)
        self.edge_j = np.array(ej, dtype=np.int64)
        self.edge_dir = np.array(ed, dtype=np.int64)
        self.edge_coord = np.array(ec, dtype=np.float64)
        self.edge_theta = np.array(et, dtype=np.float64)

    @property
    def n_edges(self):
        return len(self.edge_i)

    def interior_inside(self):
        """Inside mask over the (M-1)^2 unknowns, indexed [j-1, i-1]."""
        return self.inside[1:-1, 1:-1]


def make_domain(desc):
    return Domain(desc)
