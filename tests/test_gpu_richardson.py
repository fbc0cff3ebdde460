"""GPU parity of the Richardson solver (Eq. 3.21, KFBI_RICHARDSON) against
the float64 oracle.

On a KFBI_FP64 domain the GPU runs the same iteration as
``oracle.richardson`` (same gamma, same stop test), so the iterate and the
iteration count must agree: the iterates differ only by the rounding of the
operator (below 1e-12 relative), and the count may differ by one only when
the last residual sits within that rounding of the threshold.  On mixed
domains the Richardson iteration is the inner solver of the refinement, and
the result must match the solution of the system (oracle GMRES) to 1e-8,
as every refined solve does.
"""

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
R = kfbi.KFBI_RICHARDSON
STEP_BOUND = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _rhs(d, cplx):
    b = np.cos(2 * d.theta) + 0.3 * np.sin(d.theta)
    if cplx:
        b = b + 0.5j * np.cos(d.theta)
    return b


@pytest.mark.parametrize("kappa", [64.0, 256.0, 128.0j])
@pytest.mark.parametrize("gamma", [0.9, 1.5])
def test_richardson_fp64_matches_oracle_iteration(kappa, gamma):
    desc = W.domain_desc(64, W.star())
    d = oracle.make_domain(desc)
    b = _rhs(d, isinstance(kappa, complex))
    tol = 1e-10
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=tol, maxit=2000, solver=R, gamma=gamma)
    phi = dev(np.zeros_like(b))
    info = dom.solve_density(kappa, dev(b), phi)
    x_or, it_or, rel_or, ok = oracle.richardson(lambda v: oracle.apply_operator(d, kappa, v), b,
                                                gamma=gamma, tol=tol)
    assert ok and info["converged"]
    assert abs(info["iters"] - it_or) <= 1, (info["iters"], it_or)
    assert info["applications"] == info["iters"] + 1  # the initial guess is applied
    assert info["rel_residual"] <= tol
    if info["iters"] == it_or:
        assert rel_linf(host(phi), x_or) <= 1e-9
    # and the fixed point is the solution of the system
    x_g, _, _, _ = oracle.gmres(lambda v: oracle.apply_operator(d, kappa, v), b, None, 1e-13,
                                50, 400)
    assert rel_linf(host(phi), x_g) <= 1e-7
    dom.close()


def test_richardson_fp64_initial_guess_and_zero_rhs():
    desc = W.domain_desc(64, W.ellipse())
    d = oracle.make_domain(desc)
    kappa = 2.0 / d.h
    b = _rhs(d, False)
    x0 = 0.7 * np.sin(3 * d.theta)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=1e-10, maxit=2000, solver=R, gamma=0.9)
    phi = dev(x0)
    info = dom.solve_density(kappa, dev(b), phi)
    x_or, it_or, _, _ = oracle.richardson(lambda v: oracle.apply_operator(d, kappa, v), b, x0=x0,
                                          gamma=0.9, tol=1e-10)
    assert abs(info["iters"] - it_or) <= 1
    if info["iters"] == it_or:
        assert rel_linf(host(phi), x_or) <= 1e-9
    # b = 0: phi = 0 at once, whatever the initial guess
    phi = dev(x0)
    info = dom.solve_density(kappa, dev(np.zeros_like(b)), phi)
    assert info["converged"] and info["iters"] == 0
    assert not np.any(host(phi))
    dom.close()


def test_richardson_reports_maxit():
    desc = W.domain_desc(64, W.star())
    d = oracle.make_domain(desc)
    kappa = 2.0 / d.h
    b = _rhs(d, False)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=1e-10, maxit=7, solver=R, gamma=0.9)
    phi = dev(np.zeros_like(b))
    with pytest.raises(kfbi.KfbiError) as e:
        dom.solve_density(kappa, dev(b), phi)
    assert e.value.status == 4  # KFBI_ERR_NOT_CONVERGED
    # exactly maxit updates were made: the iterate is the oracle's 7th
    x7, it7, _, ok7 = oracle.richardson(lambda v: oracle.apply_operator(d, kappa, v), b, gamma=0.9,
                                        tol=1e-10, maxit=7)
    assert not ok7 and it7 == 7
    assert rel_linf(host(phi), x7) <= 1e-11
    dom.close()


@pytest.mark.parametrize("prec", [kfbi.KFBI_MIXED_TF32, kfbi.KFBI_MIXED_FFT32])
@pytest.mark.parametrize("kappa", [64.0, 128.0j])
def test_richardson_mixed_refined_solution(prec, kappa):
    desc = W.domain_desc(64, W.star())
    d = oracle.make_domain(desc)
    b = _rhs(d, isinstance(kappa, complex))
    dom = kfbi.Domain(desc, prec, tol=1e-12, maxit=4000, solver=R, gamma=0.9)
    phi = dev(np.zeros_like(b))
    info = dom.solve_density(kappa, dev(b), phi)
    assert info["converged"]
    x_g, _, _, _ = oracle.gmres(lambda v: oracle.apply_operator(d, kappa, v), b, None, 1e-13,
                                50, 400)
    assert rel_linf(host(phi), x_g) <= STEP_BOUND
    dom.close()


def _heat(desc, prec, steps, gamma, c=1.0):
    """Heat steps of c u_t = Delta u + s (time step h / c in u_t = Delta u +
    s), GPU with the Richardson solver and the oracle stepper with the
    same iteration; returns both fields and per-step iteration counts."""
    d = oracle.make_domain(desc)
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = d.h / c
    dom = kfbi.Domain(desc, prec, tol=1e-12, maxit=4000, solver=R, gamma=gamma)
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    st.init_heat(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)),
                 dev(ex.src(X, Y, 0) + ex.src(X, Y, tau)))
    orc = oracle.HeatStepper(d, tau, 1e-12, solver="richardson", gamma=gamma, maxit=4000)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.src(X, Y, 0) + ex.src(X, Y, tau))
    its = []
    for k in range(steps):
        t1 = (k + 1) * tau
        g, s = ex.u(zx, zy, t1), ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau)
        its.append(st.step_heat(dev(g), dev(s))["iters"])
        U = orc.step(g, s)
    u = host(st.get_u())
    dom.close()
    return u, U, its, orc.iters, d.interior_inside()


@pytest.mark.parametrize("c,gamma", [(1.0, 0.5), (16.0, 1.5)])
def test_richardson_fp64_heat_steps_match_oracle_counts(c, gamma):
    # the circle of the paper's scale-factor example, box [-1.5, 1.5]^2
    desc = W.domain_desc(64, W.star(1.0, 0.0, 1), lo=-1.5, hi=1.5)
    u, U, its, its_or, m = _heat(desc, kfbi.KFBI_FP64, 4, gamma, c)
    assert rel_linf(u[m], U[m]) <= STEP_BOUND
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_or)), (its, its_or)
    assert all(i > 0 for i in its)


def test_richardson_fft_heat_steps_match_oracle():
    desc = W.domain_desc(64, W.star(), nb=128)
    u, U, its, _, m = _heat(desc, kfbi.KFBI_MIXED_FFT32, 4, 0.9)
    assert rel_linf(u[m], U[m]) <= STEP_BOUND
    assert all(i > 0 for i in its)


def test_richardson_wave_1024_steps_match_oracle():
    desc = W.domain_desc(1024, W.ellipse())
    d = oracle.make_domain(desc)
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 4.0 * d.h
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_FFT32, tol=1e-12, maxit=4000, solver=R, gamma=0.9)
    st = kfbi.State(dom, kfbi.KFBI_WAVE)
    st.init_wave(tau, 0.25, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)), dev(ex.u(X, Y, tau)),
                 dev(ex.lap(X, Y, tau)))
    orc = oracle.WaveStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    for k in range(1, 3):
        g = ex.u(zx, zy, (k + 1) * tau)
        info = st.step_wave(dev(g))
        U = orc.step(g)
        assert info["converged"]
    m = d.interior_inside()
    assert rel_linf(host(st.get_u())[m], U[m]) <= STEP_BOUND


def test_batches_refuse_richardson_domains():
    desc = W.domain_desc(64, W.star())
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, solver=R, gamma=0.9)
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Batch([dom])
    assert e.value.status == 1
    dom.close()
