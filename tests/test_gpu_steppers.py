"""GPU parity of the float64 time steppers (kfbi_step_heat / _wave /
_schrodinger) against the oracle steppers on the same seeded inputs, plus
the manufactured-solution error of the GPU path itself."""

import math

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _setup(desc, tol):
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, restart=50, tol=tol, maxit=600)
    return d, X, Y, zx, zy, dom


def test_heat_steps_match_oracle():
    """Heat, star r = 0.5 + 0.1 sin 5t, 64^2, 128 nodes, dt = h."""
    desc = W.domain_desc(64, W.star(), nb=128)
    d, X, Y, zx, zy, dom = _setup(desc, 1e-12)
    ex = W.HeatExact()
    tau = d.h
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    s01 = ex.src(X, Y, 0) + ex.src(X, Y, tau)
    st.init_heat(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)), dev(s01))
    orc = oracle.HeatStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), s01)
    mask = d.interior_inside()
    for k in range(4):
        t1 = (k + 1) * tau
        g = ex.u(zx, zy, t1)
        s = ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau)
        info = st.step_heat(dev(g), dev(s))
        U_or = orc.step(g, s)
        assert info["converged"]
        u = host(st.get_u())
        assert rel_linf(u[mask], U_or[mask]) <= TOL
        assert abs(info["iters"] - orc.iters[-1]) <= 2
    err = np.abs(u - ex.u(X, Y, 4 * tau))[mask].max()
    assert err < 2e-3


def test_wave_steps_match_oracle():
    """Wave, ellipse a=0.7 b=0.4 rotated 30 deg, 64^2, dt = 4h, theta = 1/4."""
    desc = W.domain_desc(64, W.ellipse())
    d, X, Y, zx, zy, dom = _setup(desc, 1e-12)
    ex = W.WaveExact()
    tau = 4 * d.h
    st = kfbi.State(dom, kfbi.KFBI_WAVE)
    st.init_wave(tau, 0.25, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)), dev(ex.u(X, Y, tau)),
                 dev(ex.lap(X, Y, tau)))
    orc = oracle.WaveStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    mask = d.interior_inside()
    for k in range(1, 5):
        g = ex.u(zx, zy, (k + 1) * tau)
        st.step_wave(dev(g))
        U_or = orc.step(g)
        assert rel_linf(host(st.get_u())[mask], U_or[mask]) <= TOL


def test_schrodinger_steps_match_oracle():
    """Strang Schroedinger, flower r = 0.6 + 0.15 cos 4t, 64^2, dt = h/2,
    plane wave k = (2, 1), V = 0."""
    desc = W.domain_desc(64, W.flower())
    d, X, Y, zx, zy, dom = _setup(desc, 1e-12)
    ex = W.PlaneWaveExact(2.0, 1.0)
    tau = 0.5 * d.h
    st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
    st.init_schrodinger(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
    orc = oracle.SchrodingerStepper(d, tau, 1e-12)
    orc.init(ex.u(X, Y, 0), ex.lap(X, Y, 0))
    V = 0.5 * (X ** 2 + Y ** 2)
    mask = d.interior_inside()
    for k in range(4):
        g = ex.u(zx, zy, (k + 1) * tau)
        st.step_schrodinger(dev(V), dev(g))
        U_or = orc.step(g, V)
        assert rel_linf(host(st.get_u())[mask], U_or[mask]) <= TOL
    # density too
    assert rel_linf(host(st.get_phi()), orc.phi) <= 1e-9


def test_nonfinite_w_is_refused():
    desc = W.domain_desc(64, W.flower())
    dom = kfbi.Domain(desc)
    st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
    X, Y = W.grid_xy(desc)
    ex = W.PlaneWaveExact(2.0, 1.0)
    st.init_schrodinger(0.01, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
    g = dev(np.zeros(desc["nb"], dtype=np.complex128))
    with pytest.raises(kfbi.KfbiError) as e:
        st.step_schrodinger(dev(np.zeros_like(X)), g, w=float("nan"))
    assert e.value.status == 1  # KFBI_ERR_ARG
