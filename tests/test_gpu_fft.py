"""GPU parity of KFBI_MIXED_FFT32 domains (DST-I passes by FP32 FFT on the
CUDA cores; correction, extraction, GMRES and refinement as for
KFBI_MIXED_TF32) against the float64 oracle.

Stated bound for the fast operator: 2e-5 relative L-infinity, the same as
the TF32 path.  Arithmetic behind it: each row transform is a complex FFT
of length M in FP32 (log2 M radix-2 stages, or one radix-3 stage and
radix-2 stages, twiddles correctly rounded from float64: a few units of
2^-24 per stage, ~1.3e-7 of the largest output measured on the host
prototype at M = 1024) plus an O(1)-operation untangling; four row
transforms (the middle two in one pass), the FP32 eigenvalue division and
the FP32 correction and extraction stay well below 1e-5.  Sizes: powers of
two and three times powers of two from 64 to 2048, each several 128-wide
tiles with a ragged tail (M - 1 unknowns per row on Mp padded columns).
Steps use the refined (accurate) operator and must match the oracle to
1e-8, with the error against the exact solution at most 1.1x the float64
path's.
"""

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
BOUND = 2e-5
STEP_BOUND = 1e-8
FFT = kfbi.KFBI_MIXED_FFT32

CASES = [
    ("star-64", W.domain_desc(64, W.star())),
    ("star-192", W.domain_desc(192, W.star())),
    ("ellipse-256", W.domain_desc(256, W.ellipse())),
    ("flower-384", W.domain_desc(384, W.flower())),
    ("flower-768", W.domain_desc(768, W.flower())),
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
def test_fft_operator_within_bound(name, desc, kind):
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = {"heat": 2.0 / h, "wave": 4.0 / (4 * h) ** 2, "schr": 2.0j / (0.5 * h)}[kind]
    d, phi, f = _inputs(desc, isinstance(kappa, complex))
    Ft = np.where(d.interior_inside(), f, 0.0)
    up_or, U_or = oracle.interface_solve(d, kappa, phi, Ft)
    dom = kfbi.Domain(desc, FFT)
    up, U = dom.interface_solve(kappa, dev(phi), dev(f))
    assert rel_linf(host(up), up_or) <= BOUND
    assert rel_linf(host(U), U_or) <= BOUND
    # f = 0: the fast application GMRES iterates with
    a0 = host(dom.apply_operator(kappa, dev(phi)))
    assert rel_linf(a0, oracle.apply_operator(d, kappa, phi)) <= BOUND
    # deterministic: the same call gives the same bits
    a1 = host(dom.apply_operator(kappa, dev(phi)))
    assert np.array_equal(a0, a1)
    # and the dense route after the fast one still sees a clean right-hand side
    up2, U2 = dom.interface_solve(kappa, dev(phi), dev(f))
    assert np.array_equal(host(up2), host(up))
    dom.close()


def test_fft_pure_box_solve_matches_dst():
    """phi = 0, f = one grid point inside the domain away from the
    interface: the grid solution is one column of the discrete solution
    operator, against the oracle's float64 box solve."""
    desc = W.domain_desc(256, W.ellipse())
    d = oracle.make_domain(desc)
    M = desc["M"]
    h = (desc["hi"] - desc["lo"]) / M
    kappa = 2.0 / h
    f = np.zeros((M - 1, M - 1))
    f[127, 120] = 1.0
    # the point lies inside the ellipse, away from the interface, so the
    # correction adds nothing there
    assert d.interior_inside()[127, 120]
    up_or, U_or = oracle.interface_solve(d, kappa, np.zeros(d.nb), np.where(d.interior_inside(), f, 0.0))
    dom = kfbi.Domain(desc, FFT)
    up, U = dom.interface_solve(kappa, dev(np.zeros(d.nb)), dev(f))
    assert rel_linf(host(U), U_or) <= BOUND
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


def test_fft_heat_steps():
    desc = W.domain_desc(64, W.star(), nb=128)
    d = oracle.make_domain(desc)
    m = d.interior_inside()
    u32, exact = _run_heat(desc, FFT, 4, d)
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
    assert np.abs(u32 - exact)[m].max() <= 1.1 * np.abs(u64 - exact)[m].max()


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


@pytest.mark.parametrize("M", [128, 192, 1024])
def test_fft_wave_steps(M):
    desc = W.domain_desc(M, W.ellipse())
    d = oracle.make_domain(desc)
    m = d.interior_inside()
    steps = 3 if M == 1024 else 4
    u32, exact, tau = _run_wave(desc, FFT, steps)
    u64, _, _ = _run_wave(desc, kfbi.KFBI_FP64, steps)
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    orc = oracle.WaveStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    for k in range(1, steps + 1):
        U = orc.step(ex.u(zx, zy, (k + 1) * tau))
    assert rel_linf(u32[m], U[m]) <= STEP_BOUND
    assert np.abs(u32 - exact)[m].max() <= 1.1 * np.abs(u64 - exact)[m].max()


def test_fft_schrodinger_steps():
    desc = W.domain_desc(64, W.flower())
    d = oracle.make_domain(desc)
    ex = W.PlaneWaveExact(2.0, 1.0)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 0.5 * d.h
    V = np.zeros_like(X)
    dom = kfbi.Domain(desc, FFT, tol=1e-12)
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
def test_fft_solve_density_refined(kappa):
    desc = W.domain_desc(64, W.star())
    d = oracle.make_domain(desc)
    b = np.cos(2 * d.theta) + 0.3 * np.sin(d.theta)
    if isinstance(kappa, complex):
        b = b + 0.5j * np.cos(d.theta)
    dom = kfbi.Domain(desc, FFT, tol=1e-12, maxit=400)
    phi = dev(np.zeros_like(b))
    info = dom.solve_density(kappa, dev(b), phi)
    assert info["converged"]
    x_or, it, res, ok = oracle.gmres(lambda v: oracle.apply_operator(d, kappa, v), b, None,
                                     1e-13, 50, 400)
    assert rel_linf(host(phi), x_or) <= STEP_BOUND


def test_fft_operator_2048():
    """The largest transform (M = 2048, N1 = 64: two 32-point DFTs per lane),
    real and complex kappa, against the oracle."""
    desc = W.domain_desc(2048, W.ellipse())
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    dom = kfbi.Domain(desc, FFT)
    for kappa in (2.0 / h, 2.0j / (0.5 * h)):
        d, phi, f = _inputs(desc, isinstance(kappa, complex))
        a = host(dom.apply_operator(kappa, dev(phi)))
        assert rel_linf(a, oracle.apply_operator(d, kappa, phi)) <= BOUND
    dom.close()


@pytest.mark.parametrize("M", [96, 130, 160, 4096])
def test_fft_unsupported_sizes_are_refused(M):
    desc = W.domain_desc(M, W.star())
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Domain(desc, FFT)
    assert e.value.status == 8  # KFBI_ERR_UNSUPPORTED
