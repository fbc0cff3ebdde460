"""Pins for the oracle's time steppers (Sec. 3.1, Procedure 3): observed
second-order convergence on manufactured solutions (the paper's Tables 1
and 4 show error ratios near 4 per halving of h and tau), and L2-norm
conservation of the Strang-split Schroedinger step."""

import math
import os

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_convergence_tables.txt")


def _paper_orders():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, g, e = line.split()
        rows.setdefault(t, []).append((int(g), float(e)))
    out = {}
    for t, r in rows.items():
        r.sort()
        out[t] = [math.log2(r[i][1] / r[i + 1][1]) for i in range(len(r) - 1)]
    return out


def _heat_err(M, T=0.125):
    # the 64^2 heat configuration's node density: 128 boundary nodes at 64^2
    desc = W.domain_desc(M, W.star(), nb=2 * M)
    d = oracle.make_domain(desc)
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = d.h
    n = int(round(T / tau))
    st = oracle.HeatStepper(d, tau, 1e-11)
    st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.src(X, Y, 0) + ex.src(X, Y, tau))
    for k in range(n):
        t1 = (k + 1) * tau
        U = st.step(ex.u(zx, zy, t1), ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau))
    return np.abs(U - ex.u(X, Y, n * tau))[d.interior_inside()].max()


def _wave_err(M, T=0.5, ratio=4.0):
    desc = W.domain_desc(M, W.ellipse())
    d = oracle.make_domain(desc)
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = ratio * d.h
    n = int(round(T / tau))
    st = oracle.WaveStepper(d, tau, 1e-11)
    st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    for k in range(1, n):
        U = st.step(ex.u(zx, zy, (k + 1) * tau))
    return np.abs(U - ex.u(X, Y, n * tau))[d.interior_inside()].max()


def _schr_err(M, T=0.125):
    desc = W.domain_desc(M, W.flower())
    d = oracle.make_domain(desc)
    ex = W.PlaneWaveExact(2.0, 1.0)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 0.5 * d.h
    n = int(round(T / tau))
    st = oracle.SchrodingerStepper(d, tau, 1e-11)
    st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0))
    V = np.zeros_like(X)
    for k in range(n):
        U = st.step(ex.u(zx, zy, (k + 1) * tau), V)
    return np.abs(U - ex.u(X, Y, n * tau))[d.interior_inside()].max()


def test_golden_paper_orders_are_second_order():
    orders = _paper_orders()
    # the fixture itself: the paper's observed orders lie in [1.8, 2.9]
    for t, o in orders.items():
        assert all(1.8 < v < 2.9 for v in o), (t, o)


@pytest.mark.parametrize("fn,limit", [(_heat_err, 1e-3), (_wave_err, 5e-3), (_schr_err, 1e-3)])
def test_second_order_in_h_and_tau(fn, limit):
    e = [fn(M) for M in (32, 64, 128)]
    order = math.log2(e[0] / e[2]) / 2.0
    band = _paper_orders()
    lo_ = min(min(v) for v in band.values()) - 0.3
    hi_ = max(max(v) for v in band.values()) + 0.3
    assert e[-1] < limit, e
    assert lo_ < order < hi_, (e, order, lo_, hi_)
    assert e[0] / e[1] > 2.5 and e[1] / e[2] > 2.5, e


def test_schrodinger_norm_conservation():
    """w = 0, g = 0 and a packet far from Gamma: the Strang step composes the
    unitary pointwise B step with the Cayley (Crank-Nicolson) map of the A
    part, so the discrete L2 norm drifts only at discretisation level."""
    M = 128
    desc = W.domain_desc(M, W.flower())
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    pk = W.GaussianPacket(0.1, 0.0, 0.1, 5.0, 0.0)
    mask = d.interior_inside()
    u0 = np.where(mask, pk.u(X, Y), 0.0)
    lap0 = np.where(mask, pk.lap(X, Y), 0.0)
    norm0 = math.sqrt(np.sum(np.abs(u0[mask]) ** 2) * d.h ** 2)
    st = oracle.SchrodingerStepper(d, 0.5 * d.h, 1e-12)
    st.init(u0 / norm0, lap0 / norm0)
    V = W.harmonic_potential(X, Y)
    g = np.zeros(d.nb, dtype=np.complex128)
    norms = []
    for _ in range(8):
        U = st.step(g, V)
        norms.append(math.sqrt(np.sum(np.abs(U[mask]) ** 2) * d.h ** 2))
    drift = np.abs(np.array(norms) - 1.0).max()
    assert drift < 2e-3, norms
    # the B step alone is exactly unitary pointwise
    z = (np.random.default_rng(1).standard_normal(50) + 1j) * 0.3
    vv = np.random.default_rng(2).uniform(0, 3, 50)
    assert np.allclose(np.abs(st.b_step(z, vv)), np.abs(z), atol=1e-15)


def test_nonlinear_b_step_newton_root():
    """Eq. 3.10 with w != 0, solved by Newton: the root satisfies the
    printed equation, keeps |u| (the two sides of Eq. 3.10 then have equal
    moduli), and so equals the closed form u* (1 - i b)/(1 + i b) with
    b = tau/2 (v + w |u*|^2)."""
    rng = np.random.default_rng(7)
    z = (rng.standard_normal(400) + 1j * rng.standard_normal(400)) * 0.8
    v = rng.uniform(-1.0, 3.0, 400)
    d = oracle.make_domain(W.domain_desc(16, W.star()))
    for tau, w in ((0.25, 1.0), (0.05, -2.0), (0.125, 3.0)):
        st = oracle.SchrodingerStepper(d, tau)
        u = st.b_step(z, v, w)
        c = 0.5 * tau
        lhs = u + 1j * c * (v + w * np.abs(u) ** 2) * u
        rhs = z - 1j * c * (v + w * np.abs(z) ** 2) * z
        assert np.abs(lhs - rhs).max() <= 1e-14 * np.abs(z).max()
        assert np.allclose(np.abs(u), np.abs(z), rtol=1e-14, atol=0)
        b = c * (v + w * np.abs(z) ** 2)
        assert np.abs(u - z * (1 - 1j * b) / (1 + 1j * b)).max() <= 1e-14
    # w = 0: the linear Cayley factor
    st = oracle.SchrodingerStepper(d, 0.1)
    assert np.allclose(st.b_step(z, v, 0.0), z * (1 - 0.05j * v) / (1 + 0.05j * v), rtol=1e-15)


def _nls_err(M, c=0.2):
    """The paper's nonlinear example (Sec. 4, Ex. 5): w = 1,
    v = 1 - cos^2 x cos^2 y, u = exp(i t) cos x cos y, star
    r = 1.5((1 - c) + c cos 3 theta), box [-pi, pi]^2, N_b = M,
    tau = 8 / M (Table 4's time steps), T = 1."""
    ex = W.NonlinearSchrodingerExact()
    desc = W.domain_desc(M, W.ex5_star(c), lo=-math.pi, hi=math.pi)
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 8.0 / M
    n = int(round(1.0 / tau))
    st = oracle.SchrodingerStepper(d, tau, 1e-11)
    st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0))
    V = ex.v(X, Y)
    for k in range(n):
        U = st.step(ex.u(zx, zy, (k + 1) * tau), V, ex.w)
    return np.abs(U - ex.u(X, Y, n * tau))[d.interior_inside()].max()


def test_nonlinear_schrodinger_matches_paper_table4():
    """The whole Strang step with the nonlinear B step against the errors the
    paper prints for this example (Table 4, grids 32, 64, 128): the paper's
    c is not stated; with c = 0.2 the errors agree within 10 % (they are
    dominated by the time step: c in [0.1, 0.25] stays within 20 %)."""
    paper = {}
    for line in open(GOLDEN):
        if line.startswith("table4"):
            _, g, e = line.split()
            paper[int(g)] = float(e)
    for M in (32, 64, 128):
        e = _nls_err(M)
        assert abs(e / paper[M] - 1.0) < 0.1, (M, e, paper[M])
