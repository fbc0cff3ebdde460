"""GPU parity of the mixed-precision path (KFBI_MIXED_TF32: tcgen05 TF32x3
DST passes with FP32 accumulation drained per K-block, FP32 correction and
extraction, FP64 GMRES and steppers) against the float64 oracle.

Stated bound for the fast operator (one application, what GMRES iterates
with): 2e-5 relative L-infinity for u+ and the grid solution.  Arithmetic
behind it: operands are TF32 pairs (2^-22 relative) and all four products
are formed; each group of 64 K-terms is accumulated by the tensor core (16
MMA accumulations, <= ~2e-6 relative of the group's partial sum) and groups
(and the two K halves of a split pass) are summed in FP32 with
round-to-nearest (< 2e-7 relative at K = 2048); four passes plus the FP32
correction and extraction stay below ~1e-5.  Observed maximum: 2.5e-6 for
M <= 1024.  The bound is below the discretisation
error of every workload here (5.6e-5 for the 1024^2 wave, 4e-4 for the
64^2 heat problem).  For time steps the test also requires the mixed
path's error against the exact solution to be at most 1.1x the float64
path's.

Time steps and kfbi_solve_density on a mixed domain use iterative
refinement: the density residual, the volume term b and the final grid come
from the accurate operator (two TF32x3 box solves with an FP64 five-point
residual between them, error ~delta^2 with delta ~2e-6), so step results
must match the oracle to STEP_BOUND = 1e-8 relative.
"""

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
BOUND = 2e-5
STEP_BOUND = 1e-8

CASES = [
    ("star-64", W.domain_desc(64, W.star())),
    ("flower-130", W.domain_desc(130, W.flower(), nb=260)),
    ("ellipse-1024", W.domain_desc(1024, W.ellipse())),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _inputs(desc, cplx, seed=5):
    d = oracle.make_domain(desc)
    rng = np.random.default_rng(seed)
    phi = np.cos(3 * d.theta) + 0.2 * np.sin(5 * d.theta) + 0.05 * rng.standard_normal(d.nb)
    X, Y = W.grid_xy(desc)
    f = 30.0 * np.sin(2 * X + 1) * np.cosh(Y) + rng.standard_normal(X.shape)
    if cplx:
        phi = phi + 1j * np.sin(2 * d.theta)
        f = f * (1 - 0.5j)
    return d, phi, f


@pytest.mark.parametrize("name,desc", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["heat", "wave", "schr"])
def test_mixed_operator_within_bound(name, desc, kind):
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = {"heat": 2.0 / h, "wave": 4.0 / (4 * h) ** 2, "schr": 2.0j / (0.5 * h)}[kind]
    d, phi, f = _inputs(desc, isinstance(kappa, complex))
    Ft = np.where(d.interior_inside(), f, 0.0)
    up_or, U_or = oracle.interface_solve(d, kappa, phi, Ft)
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32)
    up, U = dom.interface_solve(kappa, dev(phi), dev(f))
    assert rel_linf(host(up), up_or) <= BOUND
    assert rel_linf(host(U), U_or) <= BOUND
    # f = 0: the sparse route GMRES iterates with
    a_or = oracle.apply_operator(d, kappa, phi)
    a = dom.apply_operator(kappa, dev(phi))
    assert rel_linf(host(a), a_or) <= BOUND
    up0 = host(dom.apply_operator(kappa, dev(phi)))
    assert rel_linf(up0, oracle.apply_operator(d, kappa, phi)) <= BOUND
    # deterministic: the same call gives the same bits
    up1 = host(dom.apply_operator(kappa, dev(phi)))
    assert np.array_equal(up0, up1)
    dom.close()


def _run_heat(desc, prec, steps, d):
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = d.h
    dom = kfbi.Domain(desc, prec, tol=1e-12)
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    st.init_heat(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)),
                 dev(ex.src(X, Y, 0) + ex.src(X, Y, tau)))
    for k in range(steps):
        t1 = (k + 1) * tau
        st.step_heat(dev(ex.u(zx, zy, t1)), dev(ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau)))
    return host(st.get_u()), ex.u(X, Y, steps * tau)


def test_mixed_heat_steps():
    desc = W.domain_desc(64, W.star(), nb=128)
    d = oracle.make_domain(desc)
    m = d.interior_inside()
    u32, exact = _run_heat(desc, kfbi.KFBI_MIXED_TF32, 4, d)
    u64, _ = _run_heat(desc, kfbi.KFBI_FP64, 4, d)
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    orc = oracle.HeatStepper(d, d.h, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.src(X, Y, 0) + ex.src(X, Y, d.h))
    for k in range(4):
        t1 = (k + 1) * d.h
        U = orc.step(ex.u(zx, zy, t1), ex.src(X, Y, t1) + ex.src(X, Y, t1 + d.h))
    assert rel_linf(u32[m], U[m]) <= STEP_BOUND
    e32 = np.abs(u32 - exact)[m].max()
    e64 = np.abs(u64 - exact)[m].max()
    assert e32 <= 1.1 * e64


def _run_wave(desc, prec, steps):
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 4.0 * (desc["hi"] - desc["lo"]) / desc["M"]
    dom = kfbi.Domain(desc, prec, tol=1e-12, maxit=1000)
    st = kfbi.State(dom, kfbi.KFBI_WAVE)
    st.init_wave(tau, 0.25, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)), dev(ex.u(X, Y, tau)),
                 dev(ex.lap(X, Y, tau)))
    for k in range(1, steps + 1):
        st.step_wave(dev(ex.u(zx, zy, (k + 1) * tau)))
    return host(st.get_u()), ex.u(X, Y, (steps + 1) * tau), tau


@pytest.mark.parametrize("M", [128, 1024])
def test_mixed_wave_steps(M):
    desc = W.domain_desc(M, W.ellipse())
    d = oracle.make_domain(desc)
    m = d.interior_inside()
    steps = 3 if M == 1024 else 4
    u32, exact, tau = _run_wave(desc, kfbi.KFBI_MIXED_TF32, steps)
    u64, _, _ = _run_wave(desc, kfbi.KFBI_FP64, steps)
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    orc = oracle.WaveStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    for k in range(1, steps + 1):
        U = orc.step(ex.u(zx, zy, (k + 1) * tau))
    assert rel_linf(u32[m], U[m]) <= STEP_BOUND
    assert rel_linf(u64[m], U[m]) <= 1e-10
    e32 = np.abs(u32 - exact)[m].max()
    e64 = np.abs(u64 - exact)[m].max()
    assert e32 <= 1.1 * e64


def test_mixed_schrodinger_steps():
    desc = W.domain_desc(64, W.flower())
    d = oracle.make_domain(desc)
    ex = W.PlaneWaveExact(2.0, 1.0)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 0.5 * d.h
    V = np.zeros_like(X)
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, tol=1e-12)
    st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
    st.init_schrodinger(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
    orc = oracle.SchrodingerStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0))
    m = d.interior_inside()
    for k in range(4):
        g = ex.u(zx, zy, (k + 1) * tau)
        st.step_schrodinger(dev(V), dev(g))
        U = orc.step(g, V)
    assert rel_linf(host(st.get_u())[m], U[m]) <= STEP_BOUND


@pytest.mark.parametrize("kappa", [64.0, 128.0j])
def test_mixed_solve_density_refined(kappa):
    desc = W.domain_desc(64, W.star())
    d = oracle.make_domain(desc)
    b = np.cos(2 * d.theta) + 0.3 * np.sin(d.theta)
    if isinstance(kappa, complex):
        b = b + 0.5j * np.cos(d.theta)
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, tol=1e-12, maxit=400)
    phi = dev(np.zeros_like(b))
    info = dom.solve_density(kappa, dev(b), phi)
    assert info["converged"]
    x_or, it, res, ok = oracle.gmres(lambda v: oracle.apply_operator(d, kappa, v), b, None,
                                     1e-13, 50, 400)
    assert rel_linf(host(phi), x_or) <= STEP_BOUND


def test_mixed_operator_full_size_2048():
    """The largest served grid (2048^2, 4096 boundary nodes) at the wave's
    kappa (the largest kappa h^2 of the steppers): fast operator against the
    oracle."""
    rng = np.random.Generator(np.random.PCG64(7))
    desc = W.domain_desc(2048, W.random_star(rng))
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = 4.0 / (4 * h) ** 2
    d, phi, f = _inputs(desc, False, seed=3)
    Ft = np.where(d.interior_inside(), f, 0.0)
    up_or, U_or = oracle.interface_solve(d, kappa, phi, Ft)
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32)
    up, U = dom.interface_solve(kappa, dev(phi), dev(f))
    assert rel_linf(host(up), up_or) <= BOUND
    assert rel_linf(host(U), U_or) <= BOUND
    # f = 0: the sparse route GMRES iterates with
    a_or = oracle.apply_operator(d, kappa, phi)
    a = dom.apply_operator(kappa, dev(phi))
    assert rel_linf(host(a), a_or) <= BOUND
