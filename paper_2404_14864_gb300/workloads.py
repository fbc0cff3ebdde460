"""Seeded synthetic workloads: domain descriptors and manufactured solutions.

This module holds inputs only (curve parameters, exact solutions used as
initial and boundary data, seeded random domains); it contains none of the
KFBI method's arithmetic.  Both the CUDA path's tests and the oracle's
tests draw their inputs from here.

The paper's own domains (cubic-spline bullet and heart, stars whose
parameter c is not given; Sec. 4.1) cannot be rebuilt, so every workload is
an analytic curve in the box [-1, 1]^2 with a manufactured solution that
supplies the Dirichlet data, the source and the initial data.
"""

import math

import numpy as np

SQRT2PI = math.sqrt(2.0) * math.pi


# ----------------------------------------------------------------------------
# Domains
# ----------------------------------------------------------------------------


def star(r0=0.5, eps=0.1, k=5, phase=0.0, cx=0.0, cy=0.0):
    """r(t) = r0 + eps sin(k t + phase) about (cx, cy)."""
    return {"kind": "polar", "cx": cx, "cy": cy, "r0": r0, "eps": eps, "k": k, "phase": phase}


def flower(r0=0.6, eps=0.15, k=4):
    """r(t) = r0 + eps cos(k t), written as a star with phase pi/2."""
    return star(r0, eps, k, math.pi / 2)


def ellipse(a=0.7, b=0.4, alpha_deg=30.0, cx=0.0, cy=0.0):
    return {"kind": "ellipse", "cx": cx, "cy": cy, "a": a, "b": b,
            "alpha": math.radians(alpha_deg)}


def domain_desc(M, curve, nb=None, lo=-1.0, hi=1.0):
    """Grid label M (intervals per side), nb boundary nodes (default M, the
    paper's choice; the 64^2 heat configuration states 128)."""
    return {"M": int(M), "lo": float(lo), "hi": float(hi),
            "nb": int(nb if nb is not None else M), "curve": dict(curve)}


def grid_xy(desc):
    """Interior node coordinates X[j-1, i-1] = x_i, Y[j-1, i-1] = y_j."""
    M, lo, hi = desc["M"], desc["lo"], desc["hi"]
    h = (hi - lo) / M
    x = lo + h * np.arange(1, M)
    return np.meshgrid(x, x)


def boundary_xy(desc):
    """Boundary node coordinates z(2 pi k / nb), k = 0..nb-1."""
    c = desc["curve"]
    t = (2.0 * math.pi / desc["nb"]) * np.arange(desc["nb"])
    if c["kind"] == "polar":
        r = c["r0"] + c["eps"] * np.sin(c["k"] * t + c["phase"])
        return c["cx"] + r * np.cos(t), c["cy"] + r * np.sin(t)
    ca, sa = math.cos(c["alpha"]), math.sin(c["alpha"])
    u, v = c["a"] * np.cos(t), c["b"] * np.sin(t)
    return c["cx"] + ca * u - sa * v, c["cy"] + sa * u + ca * v


def boundary_normal(desc):
    """Outward unit normal (n_x, n_y) = (y', -x') / |z'| at the boundary nodes
    (the curves run counter-clockwise), for Neumann data d_n u = grad u . n."""
    c = desc["curve"]
    t = (2.0 * math.pi / desc["nb"]) * np.arange(desc["nb"])
    if c["kind"] == "polar":
        r = c["r0"] + c["eps"] * np.sin(c["k"] * t + c["phase"])
        dr = c["eps"] * c["k"] * np.cos(c["k"] * t + c["phase"])
        dx = dr * np.cos(t) - r * np.sin(t)
        dy = dr * np.sin(t) + r * np.cos(t)
    else:
        ca, sa = math.cos(c["alpha"]), math.sin(c["alpha"])
        du, dv = -c["a"] * np.sin(t), c["b"] * np.cos(t)
        dx, dy = ca * du - sa * dv, sa * du + ca * dv
    s = np.hypot(dx, dy)
    return dy / s, -dx / s


# ----------------------------------------------------------------------------
# Manufactured solutions (value, Laplacian, source)
# ----------------------------------------------------------------------------


class HeatExact:
    """u = exp(-t) sin(pi x) cos(pi y); u_t = Delta u + s, s = (2 pi^2 - 1) u."""

    def u(self, x, y, t):
        return math.exp(-t) * np.sin(math.pi * x) * np.cos(math.pi * y)

    def lap(self, x, y, t):
        return -2.0 * math.pi ** 2 * self.u(x, y, t)

    def src(self, x, y, t):
        return (2.0 * math.pi ** 2 - 1.0) * self.u(x, y, t)


class WaveExact:
    """u = cos(sqrt(2) pi t) sin(pi x) sin(pi y); u_tt = Delta u (source-free)."""

    def u(self, x, y, t):
        return math.cos(SQRT2PI * t) * np.sin(math.pi * x) * np.sin(math.pi * y)

    def grad(self, x, y, t):
        c = math.cos(SQRT2PI * t) * math.pi
        return (c * np.cos(math.pi * x) * np.sin(math.pi * y),
                c * np.sin(math.pi * x) * np.cos(math.pi * y))

    def lap(self, x, y, t):
        return -2.0 * math.pi ** 2 * self.u(x, y, t)


class PlaneWaveExact:
    """u = exp(i (k . x + |k|^2 t)) solves u_t = -i Delta u (V = 0, w = 0)."""

    def __init__(self, kx=5.0, ky=0.0):
        self.kx, self.ky = float(kx), float(ky)
        self.k2 = self.kx ** 2 + self.ky ** 2

    def u(self, x, y, t):
        return np.exp(1j * (self.kx * x + self.ky * y + self.k2 * t))

    def lap(self, x, y, t):
        return -self.k2 * self.u(x, y, t)


def ex5_star(c=0.2):
    """The star of the paper's nonlinear Schroedinger example (Sec. 4, Ex. 5):
    r = 1.5 ((1 - c) + c cos 3 theta) about the origin.  The paper does not
    state c."""
    return star(1.5 * (1.0 - c), 1.5 * c, 3, 0.5 * math.pi)


class NonlinearSchrodingerExact:
    """u = exp(i t) cos x cos y solves i u_t = Delta u + (v + w |u|^2) u with
    w = 1 and v = 1 - cos^2 x cos^2 y (Sec. 4, Eqs. 4.3-4.4)."""

    w = 1.0

    def u(self, x, y, t):
        return np.exp(1j * t) * np.cos(x) * np.cos(y)

    def lap(self, x, y, t):
        return -2.0 * self.u(x, y, t)

    def v(self, x, y):
        return 1.0 - (np.cos(x) * np.cos(y)) ** 2


class GaussianPacket:
    """u0 = A exp(-|x - x0|^2 / (2 s^2)) exp(i k . x), normalised so that the
    discrete L2 norm over the grid is 1 (A computed by the caller)."""

    def __init__(self, x0=0.1, y0=0.0, width=0.1, kx=5.0, ky=0.0, amp=1.0):
        self.x0, self.y0, self.s = x0, y0, width
        self.kx, self.ky, self.amp = kx, ky, amp

    def u(self, x, y):
        dx, dy = x - self.x0, y - self.y0
        return self.amp * np.exp(-(dx * dx + dy * dy) / (2 * self.s ** 2)) * \
            np.exp(1j * (self.kx * x + self.ky * y))

    def lap(self, x, y):
        dx, dy = x - self.x0, y - self.y0
        s2 = self.s ** 2
        gx = -dx / s2 + 1j * self.kx
        gy = -dy / s2 + 1j * self.ky
        return self.u(x, y) * (gx * gx + gy * gy - 2.0 / s2)


def harmonic_potential(x, y):
    return 0.5 * (x * x + y * y)


# ----------------------------------------------------------------------------
# Benchmark configurations
# ----------------------------------------------------------------------------

CONFIG_HEAT_64 = dict(name="heat-star-64", M=64, curve=star(), nb=128, dt_over_h=1.0,
                      steps=31, tol=1e-10)
CONFIG_WAVE = dict(name="wave-ellipse", curve=ellipse(), dt_over_h=1.0, T=0.5, theta=0.25,
                   tol=1e-10)
CONFIG_SCHR = dict(name="schrodinger-flower", M=1024, curve=flower(), dt_over_h=0.5,
                   steps=400, tol=1e-10)


def random_star(rng):
    """Star r = 0.5 + eps sin(k t + phase), k in 3..7, eps in [0.05, 0.15]."""
    k = int(rng.integers(3, 8))
    eps = float(rng.uniform(0.05, 0.15))
    phase = float(rng.uniform(0.0, 2.0 * math.pi))
    return star(0.5, eps, k, phase)


def batched_instances(n=256, sizes=(128, 192, 256, 384, 512), seed=0):
    """Seeded list of (M, curve) pairs for the batched heat workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        M = int(sizes[int(rng.integers(0, len(sizes)))])
        out.append((M, random_star(rng)))
    return out


def served_requests(n=1000, rate=200.0, sizes=(128, 256, 512, 1024, 2048),
                    steps=(20, 200), seed=0):
    """Seeded Poisson request stream: (arrival_s, kind, M, curve, steps)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    kinds = ("heat", "wave", "schrodinger")
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        kind = kinds[int(rng.integers(0, 3))]
        M = int(sizes[int(rng.integers(0, len(sizes)))])
        st = int(rng.integers(steps[0], steps[1] + 1))
        out.append((t, kind, M, random_star(rng), st))
    return out


# ----------------------------------------------------------------------------
# Served requests: host inputs of one time-stepping request
# ----------------------------------------------------------------------------

KINDS = {"heat": 0, "wave": 1, "schrodinger": 2}   # kfbi_equation values
STEP_OVER_H = {"heat": 1.0, "wave": 4.0, "schrodinger": 0.5}


def request_inputs(kind, desc, steps, theta=0.5):
    """Host inputs of a manufactured-solution request (the arguments of
    ``kfbi.Server.submit`` besides the descriptor, arrival and tolerance).

    heat: u = exp(-t) sin(pi x) cos(pi y) with its source, whose step sums
    are src_coef[n] * profile (the source is exp(-t) times a profile);
    wave: u = cos(sqrt 2 pi t) sin(pi x) sin(pi y), theta = 1/2 by default
    (second order like 1/4; its roots stay away from the double root at -1
    where theta = 1/4 lets a few random-star domains grow over 20-200 steps);
    Schroedinger: plane wave k = (5, 0), V = 0.  "exact" gives the solution
    at the request's final time on the interior grid."""
    X, Y = grid_xy(desc)
    zx, zy = boundary_xy(desc)
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    dt = STEP_OVER_H[kind] * h
    out = {"equation": KINDS[kind], "dt": dt, "steps": int(steps)}
    if kind == "heat":
        ex = HeatExact()
        prof = ex.src(X, Y, 0.0)
        out.update(u0=ex.u(X, Y, 0.0), lap_u0=ex.lap(X, Y, 0.0),
                   src_init=ex.src(X, Y, 0.0) + ex.src(X, Y, dt), src_profile=prof,
                   src_coef=np.array([math.exp(-(n + 1) * dt) + math.exp(-(n + 2) * dt)
                                      for n in range(steps)]),
                   g=np.stack([ex.u(zx, zy, (n + 1) * dt) for n in range(steps)]))
        t_end = steps * dt
    elif kind == "wave":
        ex = WaveExact()
        out.update(theta=float(theta), u0=ex.u(X, Y, 0.0), lap_u0=ex.lap(X, Y, 0.0), u1=ex.u(X, Y, dt),
                   lap_u1=ex.lap(X, Y, dt),
                   g=np.stack([ex.u(zx, zy, (n + 2) * dt) for n in range(steps)]))
        t_end = (steps + 1) * dt
    else:
        ex = PlaneWaveExact(5.0, 0.0)
        out.update(u0=ex.u(X, Y, 0.0), lap_u0=ex.lap(X, Y, 0.0), potential=np.zeros_like(X),
                   g=np.stack([ex.u(zx, zy, (n + 1) * dt) for n in range(steps)]))
        t_end = steps * dt
    out["exact"] = lambda: ex.u(X, Y, t_end)
    return out
