"""GPU parity of the Neumann path (Eqs. 3.19, 3.20, 3.22) on float64
domains against the float64 oracle.

Bars: the operator psi -> d_n u+ (with and without a volume source) within
1e-10 relative L-infinity, as every float64 operator; the solved density
and grid solution of a Neumann BVP within 1e-9 (GMRES at tol 1e-12 on both
sides); the Richardson iteration of Eq. 3.22 with the oracle's count (+-1).
"""

import math

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
CASES = [
    ("star-64", W.domain_desc(64, W.star())),
    ("ellipse-256", W.domain_desc(256, W.ellipse())),
    ("flower-1024", W.domain_desc(1024, W.flower())),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _psi(d, cplx, seed=3):
    rng = np.random.default_rng(seed)
    psi = np.sin(2 * d.theta) + 0.4 * np.cos(5 * d.theta) + 0.05 * rng.standard_normal(d.nb)
    return psi + 0.3j * np.cos(3 * d.theta) if cplx else psi


@pytest.mark.parametrize("name,desc", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["heat", "wave", "schr"])
def test_neumann_operator_matches_oracle(name, desc, kind):
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = {"heat": 2.0 / h, "wave": 4.0 / (4 * h) ** 2, "schr": 2.0j / (0.5 * h)}[kind]
    cplx = isinstance(kappa, complex)
    d = oracle.make_domain(desc)
    psi = _psi(d, cplx)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64)
    out = host(dom.apply_neumann(kappa, dev(psi)))
    assert rel_linf(out, oracle.apply_neumann(d, kappa, psi)) <= 1e-10
    if desc["M"] <= 256:
        X, Y = W.grid_xy(desc)
        f = 20.0 * np.sin(2 * X + 1) * np.cosh(Y)
        if cplx:
            f = f * (1 - 0.5j)
        Ft = np.where(d.interior_inside(), f, 0.0)
        out = host(dom.apply_neumann(kappa, dev(psi), dev(f)))
        assert rel_linf(out, oracle.apply_neumann(d, kappa, psi, Ft)) <= 1e-10
    dom.close()


def _bvp(M, kappa=10.0):
    desc = W.domain_desc(M, W.star())
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    u = np.sin(0.6 * X + 0.8 * Y)
    f = -(1.0 + kappa) * u
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    cz = np.cos(0.6 * d.zx + 0.8 * d.zy)
    gN = 0.6 * cz * t2 - 0.8 * cz * t1
    return desc, d, u, f, gN


@pytest.mark.parametrize("M", [64, 128])
def test_neumann_bvp_matches_oracle(M):
    kappa = 10.0
    desc, d, u, f, gN = _bvp(M, kappa)
    m = d.interior_inside()
    Ft = np.where(m, f, 0.0)
    b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb), Ft)
    psi_or, it, _, ok = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), b, None,
                                     1e-13, 50, 500)
    _, U_or = oracle.interface_solve(d, kappa, np.zeros(d.nb), Ft, psi_or)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=1e-12, maxit=500)
    psi = dev(np.zeros(d.nb))
    import torch
    ug = torch.empty((M - 1) ** 2, dtype=torch.float64, device="cuda")
    info = dom.solve_neumann(kappa, dev(gN), psi, dev(f), ug)
    assert info["converged"]
    assert rel_linf(host(psi), psi_or) <= 1e-9
    Ug = host(ug).reshape(M - 1, M - 1)
    assert rel_linf(Ug[m], U_or[m]) <= 1e-9
    # the same error against the exact solution as the oracle
    e_gpu, e_or = np.abs(Ug - u)[m].max(), np.abs(U_or - u)[m].max()
    assert abs(e_gpu - e_or) <= 1e-8 * np.abs(u).max()
    # and the extracted normal derivative of the solution is the data
    dn = host(dom.apply_neumann(kappa, psi, dev(f)))
    assert np.abs(dn - gN).max() <= 1e-8 * np.abs(gN).max()
    dom.close()


@pytest.mark.parametrize("gamma", [0.5, 1.2])
def test_neumann_richardson_matches_oracle(gamma):
    """Eq. 3.22: psi <- psi + gamma (b - A_N psi), the same iteration and
    stop test on both sides."""
    kappa = 10.0
    desc, d, u, f, gN = _bvp(64, kappa)
    m = d.interior_inside()
    Ft = np.where(m, f, 0.0)
    b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb), Ft)
    tol = 1e-10
    x_or, it_or, _, ok = oracle.richardson(lambda v: oracle.apply_neumann(d, kappa, v), b,
                                           gamma=gamma, tol=tol, maxit=5000)
    assert ok
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=tol, maxit=5000, solver=kfbi.KFBI_RICHARDSON,
                      gamma=gamma)
    psi = dev(np.zeros(d.nb))
    info = dom.solve_neumann(kappa, dev(gN), psi, dev(f))
    assert info["converged"] and abs(info["iters"] - it_or) <= 1, (info["iters"], it_or)
    if info["iters"] == it_or:
        assert rel_linf(host(psi), x_or) <= 1e-9
    dom.close()


def test_neumann_complex_kappa_solve():
    # kappa = 2i/tau of the Schroedinger step: the BVP with complex data
    desc = W.domain_desc(64, W.flower())
    d = oracle.make_domain(desc)
    kappa = 2.0j / (0.5 * d.h)
    gN = _psi(d, True, 9)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=1e-12, maxit=500)
    psi = dev(np.zeros(d.nb, dtype=np.complex128))
    info = dom.solve_neumann(kappa, dev(gN), psi)
    assert info["converged"]
    x_or, _, _, _ = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), gN, None, 1e-13,
                                 50, 500)
    assert rel_linf(host(psi), x_or) <= 1e-9
    dom.close()


MIXED = [kfbi.KFBI_MIXED_TF32, kfbi.KFBI_MIXED_FFT32]


@pytest.mark.parametrize("prec", MIXED, ids=["tf32", "fft32"])
@pytest.mark.parametrize("name,desc", [CASES[0], ("ellipse-1024", W.domain_desc(1024, W.ellipse()))],
                         ids=["star-64", "ellipse-1024"])
@pytest.mark.parametrize("kind", ["heat", "schr"])
def test_neumann_fast_operator_within_bound(prec, name, desc, kind):
    """The fast (FP32 / TF32x3) Neumann operator within 2e-5 relative, the
    bound of the Dirichlet fast operator (same passes, same FP32 tables)."""
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = {"heat": 2.0 / h, "schr": 2.0j / (0.5 * h)}[kind]
    cplx = isinstance(kappa, complex)
    d = oracle.make_domain(desc)
    psi = _psi(d, cplx)
    dom = kfbi.Domain(desc, prec)
    out = host(dom.apply_neumann(kappa, dev(psi)))
    assert rel_linf(out, oracle.apply_neumann(d, kappa, psi)) <= 2e-5
    # with a volume source (dense route)
    X, Y = W.grid_xy(desc)
    f = 20.0 * np.sin(2 * X + 1) * np.cosh(Y) * ((1 - 0.5j) if cplx else 1.0)
    out = host(dom.apply_neumann(kappa, dev(psi), dev(f)))
    Ft = np.where(d.interior_inside(), f, 0.0)
    assert rel_linf(out, oracle.apply_neumann(d, kappa, psi, Ft)) <= 2e-5
    dom.close()


@pytest.mark.parametrize("prec", MIXED, ids=["tf32", "fft32"])
def test_neumann_mixed_bvp_refined(prec):
    """Refined solves on mixed domains: density and grid within 1e-8.  The
    solve stops at 1e-10: the normal derivative amplifies the refined grid's
    relative error (~1e-13 after two sweeps) by O(1/h), which bounds the
    outer residual a little above 1e-12 at this size."""
    kappa = 10.0
    desc, d, u, f, gN = _bvp(128, kappa)
    m = d.interior_inside()
    Ft = np.where(m, f, 0.0)
    b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb), Ft)
    psi_or, _, _, _ = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), b, None, 1e-13,
                                   50, 500)
    _, U_or = oracle.interface_solve(d, kappa, np.zeros(d.nb), Ft, psi_or)
    dom = kfbi.Domain(desc, prec, tol=1e-10, maxit=1000)
    psi = dev(np.zeros(d.nb))
    import torch
    ug = torch.empty(127 ** 2, dtype=torch.float64, device="cuda")
    info = dom.solve_neumann(kappa, dev(gN), psi, dev(f), ug)
    assert info["converged"]
    assert rel_linf(host(psi), psi_or) <= 1e-8
    assert rel_linf(host(ug).reshape(127, 127)[m], U_or[m]) <= 1e-8
    dom.close()


def _heat_neumann_data(M):
    """The paper's Neumann heat solution (Sec. 4, Ex. 2):
    u = exp(-t) sin(0.6 x + 0.8 y), u_t = Delta u, on a star in
    [-1.5, 1.5]^2, tau = 16 / M (its Table 2 steps)."""
    desc = W.domain_desc(M, W.star(1.0, 0.2, 5), lo=-1.5, hi=1.5)
    d = oracle.make_domain(desc)
    X, Y = W.grid_xy(desc)
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    u = lambda t: math.exp(-t) * np.sin(0.6 * X + 0.8 * Y)
    gN = lambda t: math.exp(-t) * np.cos(0.6 * d.zx + 0.8 * d.zy) * (0.6 * t2 - 0.8 * t1)
    return desc, d, u, gN, 16.0 / M


@pytest.mark.parametrize("M", [64, 128])
def test_neumann_heat_steps_match_oracle(M):
    desc, d, u, gN, tau = _heat_neumann_data(M)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64, tol=1e-12, maxit=500)
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    st.set_neumann(True)
    st.init_heat(tau, dev(u(0)), dev(-u(0)))
    orc = oracle.HeatStepper(d, tau, 1e-12, bc="neumann")
    orc.init(u(0), -u(0))
    m = d.interior_inside()
    n = int(round(1.0 / tau))
    for k in range(n):
        info = st.step_heat(dev(gN((k + 1) * tau)))
        U = orc.step(gN((k + 1) * tau))
        assert info["converged"]
        assert rel_linf(host(st.get_u())[m], U[m]) <= 1e-10, k
    e = np.abs(host(st.get_u()) - u(n * tau))[m].max()
    assert e <= 1.01 * np.abs(U - u(n * tau))[m].max() + 1e-12
    dom.close()


@pytest.mark.parametrize("M", [64, 256])
def test_neumann_heat_steps_fft32(M):
    desc, d, u, gN, tau = _heat_neumann_data(M)
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_FFT32, tol=1e-10, maxit=1000)
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    st.set_neumann(True)
    st.init_heat(tau, dev(u(0)), dev(-u(0)))
    orc = oracle.HeatStepper(d, tau, 1e-12, bc="neumann")
    orc.init(u(0), -u(0))
    m = d.interior_inside()
    for k in range(4):
        info = st.step_heat(dev(gN((k + 1) * tau)))
        U = orc.step(gN((k + 1) * tau))
        assert info["converged"]
    assert rel_linf(host(st.get_u())[m], U[m]) <= 1e-8
    dom.close()


def test_batches_refuse_neumann_states():
    desc = W.domain_desc(64, W.star())
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32)
    st = kfbi.State(dom, kfbi.KFBI_HEAT)
    X, Y = W.grid_xy(desc)
    st.init_heat(0.01, dev(np.sin(X)), dev(-np.sin(X)))
    st.set_neumann(True)
    b = kfbi.Batch([dom])
    with pytest.raises(kfbi.KfbiError) as e:
        b.step([st], [dev(np.zeros(desc["nb"]))])
    assert e.value.status == 1
    b.close()
    dom.close()


def test_neumann_zero_data_gives_zero_density():
    desc = W.domain_desc(64, W.star())
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_FFT32, tol=1e-10)
    psi = dev(np.full(desc["nb"], 0.3))  # a nonzero initial guess
    info = dom.solve_neumann(10.0, dev(np.zeros(desc["nb"])), psi)
    assert info["converged"] and info["iters"] == 0
    assert not np.any(host(psi))
    dom.close()


@pytest.mark.parametrize("prec", [kfbi.KFBI_FP64, kfbi.KFBI_MIXED_FFT32], ids=["fp64", "fft32"])
def test_neumann_richardson_on_every_precision(prec):
    kappa = 10.0
    desc, d, u, f, gN = _bvp(64, kappa)
    m = d.interior_inside()
    Ft = np.where(m, f, 0.0)
    b = gN - oracle.apply_neumann(d, kappa, np.zeros(d.nb), Ft)
    x_g, _, _, _ = oracle.gmres(lambda v: oracle.apply_neumann(d, kappa, v), b, None, 1e-13,
                                50, 500)
    dom = kfbi.Domain(desc, prec, tol=1e-10, maxit=5000, solver=kfbi.KFBI_RICHARDSON, gamma=1.2)
    psi = dev(np.zeros(d.nb))
    info = dom.solve_neumann(kappa, dev(gN), psi, dev(f))
    assert info["converged"]
    assert rel_linf(host(psi), x_g) <= 1e-8
    dom.close()
