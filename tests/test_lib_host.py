"""Host-side tests of the C-ABI library (no GPU): the shared library loads
and exports every entry point of include/kfbi.h, and the host-built plan
(geometry and coefficient tables) agrees with the oracle."""

import math
import os
import re

import numpy as np
import pytest

import oracle
from oracle.interface import edge_f_gamma, node_f_gamma
from paper_2404_14864_gb300 import kfbi, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DOMAINS = [
    W.domain_desc(64, W.star()),
    W.domain_desc(48, W.ellipse(), nb=80),
    W.domain_desc(96, W.flower(), nb=150),
    W.domain_desc(40, W.star(0.45, 0.12, 3, 1.1, 0.05, -0.03)),
    # near-tie nodes that once classified differently on an aarch64 host
    W.domain_desc(192, W.star()),
    W.domain_desc(384, W.flower()),
]


@pytest.fixture(scope="module")
def built():
    from paper_2404_14864_gb300 import build
    build.build()
    return kfbi.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "kfbi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kfbi_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(built):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(built, n), n
    # and the binding declares the same set
    import ctypes
    for n in names:
        assert isinstance(getattr(built, n), ctypes._CFuncPtr)


def test_create_domain_errors_without_touching_the_gpu(built):
    bad = W.domain_desc(64, W.star(0.95, 0.1, 5, 0.0))  # touches the box
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Plan(bad)
    assert e.value.status == 2
    d = kfbi.make_desc(W.domain_desc(64, W.star()))
    d.M = 3
    import ctypes
    h = ctypes.c_void_p()
    assert built.kfbi_create_domain(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert not h.value
    d = kfbi.make_desc(W.domain_desc(64, W.star()))
    d.gmres_restart = 0
    assert built.kfbi_create_domain(ctypes.byref(d), None, ctypes.byref(h)) == 1
    # solver: unknown kinds and Richardson steps outside (0, 2) are refused
    # before any device work
    for solver, gamma in ((2, 0.9), (-1, 0.9), (kfbi.KFBI_RICHARDSON, 0.0),
                          (kfbi.KFBI_RICHARDSON, 2.0), (kfbi.KFBI_RICHARDSON, float("nan"))):
        d = kfbi.make_desc(W.domain_desc(64, W.star()), solver=solver, gamma=gamma)
        assert built.kfbi_create_domain(ctypes.byref(d), None, ctypes.byref(h)) == 1
        assert not h.value


@pytest.mark.parametrize("desc", DOMAINS, ids=lambda d: "%s-%d" % (d["curve"]["kind"], d["M"]))
def test_plan_geometry_matches_oracle(built, desc):
    p = kfbi.Plan(desc)
    d = oracle.make_domain(desc)
    M = desc["M"]
    assert np.array_equal(p.field("inside").reshape(M + 1, M + 1).astype(bool), d.inside)
    irr = np.flatnonzero(d.irregular[1:-1, 1:-1].ravel())
    assert np.array_equal(p.field("irregular"), irr)
    assert p.n_edges == d.n_edges and p.n_arms == 2 * d.n_edges
    assert np.array_equal(p.field("edge_i"), d.edge_i)
    assert np.array_equal(p.field("edge_j"), d.edge_j)
    assert np.array_equal(p.field("edge_dir"), d.edge_dir)
    assert np.abs(p.field("edge_coord") - d.edge_coord).max() <= 1e-13
    assert np.abs(p.field("edge_theta") - d.edge_theta).max() <= 1e-13


def _plan_rhs(p, desc, phi, kappa, Ft):
    """Apply the plan's arm tables as the correction kernel does (test-only)."""
    nb = desc["nb"]
    n1 = desc["M"] - 1
    f = Ft.ravel()
    R = f.astype(np.result_type(f, phi, kappa)).copy()
    irr = p.field("irregular")
    node = p.field("arm_node"); k0 = p.field("arm_k0")
    al = p.field("arm_alpha").reshape(-1, 6); be = p.field("arm_beta").reshape(-1, 6)
    fi = p.field("arm_fidx").reshape(-1, 2); fc = p.field("arm_fcoef").reshape(-1, 2)
    idx = (k0[:, None] + np.arange(6)[None, :]) % nb
    contrib = ((al + kappa * be) * phi[idx]).sum(axis=1) + (fc * f[fi]).sum(axis=1)
    acc = np.zeros(len(irr), dtype=R.dtype)
    np.add.at(acc, node, contrib)
    R[irr] = f[irr] + acc
    return R.reshape(n1, n1)


def _plan_extract(p, desc, U, phi, kappa, Ft):
    nb = desc["nb"]
    u = U.ravel(); f = Ft.ravel()
    g = p.field("node_gidx").reshape(nb, 6); w = p.field("node_w").reshape(nb, 6)
    a = p.field("node_a").reshape(nb, 6); b = p.field("node_b").reshape(nb, 6)
    idx = (np.arange(nb)[:, None] - 2 + np.arange(6)[None, :]) % nb
    return (w * u[g]).sum(1) + ((a + kappa * b) * phi[idx]).sum(1) + \
        p.field("node_fcoef") * f[p.field("node_fidx")]


@pytest.mark.parametrize("desc", DOMAINS, ids=lambda d: "%s-%d" % (d["curve"]["kind"], d["M"]))
@pytest.mark.parametrize("kappa", [17.0, 3.5e4, 40.0j])
def test_plan_tables_reproduce_oracle_correction_and_extraction(built, desc, kappa):
    p = kfbi.Plan(desc)
    d = oracle.make_domain(desc)
    rng = np.random.default_rng(21)
    n1 = desc["M"] - 1
    cplx = isinstance(kappa, complex)
    phi = np.cos(3 * d.theta) + 0.3 * np.sin(7 * d.theta) + 0.1 * rng.standard_normal(d.nb)
    X, Y = W.grid_xy(desc)
    Ft = np.where(d.interior_inside(), np.sin(2 * X + 1) * np.cosh(Y) * 50.0, 0.0)
    if cplx:
        phi = phi + 1j * np.sin(2 * d.theta)
        Ft = Ft * (1 - 0.5j)
    ej = oracle.jumps_at(d, d.edge_theta, phi, edge_f_gamma(d, Ft), kappa)
    R_or = oracle.correction_rhs(d, Ft, ej)
    R_pl = _plan_rhs(p, desc, phi, kappa, Ft)
    scale = np.abs(R_or).max()
    assert np.abs(R_pl - R_or).max() <= 1e-12 * scale
    U = rng.standard_normal((n1, n1)) + (1j * rng.standard_normal((n1, n1)) if cplx else 0)
    nj = oracle.jumps_at(d, None, phi, node_f_gamma(d, Ft), kappa, node_k=np.arange(d.nb))
    up_or = oracle.extraction(d, U, nj)
    up_pl = _plan_extract(p, desc, U, phi, kappa, Ft)
    assert np.abs(up_pl - up_or).max() <= 1e-11 * max(1.0, np.abs(up_or).max())


@pytest.mark.parametrize("desc", DOMAINS, ids=lambda d: "%s-%d" % (d["curve"]["kind"], d["M"]))
@pytest.mark.parametrize("kappa", [17.0, 40.0j])
def test_plan_neumann_tables_reproduce_oracle(built, desc, kappa):
    """Psi = psi, Phi = 0: the arm weights of psi give the oracle's corrected
    right-hand side, and the normal-derivative tables its d_n u+ (Eq. 3.36
    rows U_x, U_y with the psi and f jump terms)."""
    p = kfbi.Plan(desc)
    d = oracle.make_domain(desc)
    rng = np.random.default_rng(5)
    n1, nb = desc["M"] - 1, desc["nb"]
    cplx = isinstance(kappa, complex)
    psi = np.sin(2 * d.theta) + 0.4 * np.cos(5 * d.theta) + 0.1 * rng.standard_normal(nb)
    X, Y = W.grid_xy(desc)
    Ft = np.where(d.interior_inside(), np.sin(2 * X + 1) * np.cosh(Y) * 50.0, 0.0)
    if cplx:
        psi = psi + 0.5j * np.cos(3 * d.theta)
        Ft = Ft * (1 - 0.5j)
    zero = np.zeros(nb, dtype=psi.dtype)
    ej = oracle.jumps_at(d, d.edge_theta, zero, edge_f_gamma(d, Ft), kappa, psi)
    R_or = oracle.correction_rhs(d, Ft, ej)
    irr = p.field("irregular")
    node = p.field("arm_node"); k0 = p.field("arm_k0")
    de = p.field("arm_delta").reshape(-1, 6)
    fi = p.field("arm_fidx").reshape(-1, 2); fc = p.field("arm_fcoef").reshape(-1, 2)
    idx = (k0[:, None] + np.arange(6)[None, :]) % nb
    f = Ft.ravel()
    contrib = (de * psi[idx]).sum(axis=1) + (fc * f[fi]).sum(axis=1)
    acc = np.zeros(len(irr), dtype=R_or.dtype)
    np.add.at(acc, node, contrib)
    R_pl = Ft.ravel().astype(R_or.dtype).copy()
    R_pl[irr] = f[irr] + acc
    assert np.abs(R_pl.reshape(n1, n1) - R_or).max() <= 1e-12 * np.abs(R_or).max()
    U = rng.standard_normal((n1, n1)) + (1j * rng.standard_normal((n1, n1)) if cplx else 0)
    nj = oracle.jumps_at(d, None, zero, node_f_gamma(d, Ft), kappa, psi, node_k=np.arange(nb))
    dn_or = oracle.extraction(d, U, nj, normal=True)
    g = p.field("node_gidx").reshape(nb, 6)
    wn = p.field("node_wn").reshape(nb, 6); e = p.field("node_e").reshape(nb, 6)
    jdx = (np.arange(nb)[:, None] - 2 + np.arange(6)[None, :]) % nb
    dn_pl = (wn * U.ravel()[g]).sum(1) + (e * psi[jdx]).sum(1) + \
        p.field("node_fcoef_n") * f[p.field("node_fidx")]
    assert np.abs(dn_pl - dn_or).max() <= 1e-10 * max(1.0, np.abs(dn_or).max())


def test_plan_device_bytes_on_the_host(built):
    """The exact admission count is host-only: it grows with the padded grid
    and the equation's fields, and rejects bad arguments."""
    d = W.domain_desc(128, W.star())
    p = kfbi.Plan(d, kfbi.KFBI_MIXED_TF32, 50)
    heat, wave, schr = (p.device_bytes(e) for e in (kfbi.KFBI_HEAT, kfbi.KFBI_WAVE,
                                                   kfbi.KFBI_SCHRODINGER))
    Mp = 128
    assert 0 < heat < wave < schr
    assert wave - heat == Mp * Mp * 8           # F^n plane of the wave state
    # complex u, F, ft, u** and Y f-tilde (10 planes) against real u, F, ft, Y f-tilde (4)
    assert schr - heat == 6 * Mp * Mp * 8
    assert p.device_bytes(7) == -1
    p.close()
    p64 = kfbi.Plan(d, kfbi.KFBI_FP64, 50)
    # the FP64 domain keeps a second FP64 work grid but no tensor-core planes
    assert p64.device_bytes(kfbi.KFBI_HEAT) < heat
    p64.close()
    big = kfbi.Plan(W.domain_desc(512, W.star()), kfbi.KFBI_MIXED_TF32, 50)
    ratio = big.device_bytes(kfbi.KFBI_HEAT) / heat
    big.close()
    assert 12.0 < ratio < 16.0                  # planes dominate: below (512/128)^2


def test_served_request_stream_is_poisson_and_balanced():
    reqs = W.served_requests(4000, rate=200.0, seed=0)
    t = np.array([r[0] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1   # exponential: cv = 1
    kinds = [r[1] for r in reqs]
    for k in ("heat", "wave", "schrodinger"):
        assert abs(kinds.count(k) / len(kinds) - 1 / 3) < 0.04
    assert set(r[2] for r in reqs) == {128, 256, 512, 1024, 2048}
    steps = [r[4] for r in reqs]
    assert min(steps) >= 20 and max(steps) <= 200
    assert reqs[:3] == W.served_requests(3, rate=200.0, seed=0)  # seeded


def test_request_inputs_shapes():
    desc = W.domain_desc(64, W.star())
    for kind in ("heat", "wave", "schrodinger"):
        x = W.request_inputs(kind, desc, 5)
        assert x["g"].shape == (5, 64)
        assert x["u0"].shape == (63, 63)
        assert x["exact"]().shape == (63, 63)
    h = W.request_inputs("heat", desc, 5)
    # the source sums are coefficient times profile (source = exp(-t) * profile)
    ex = W.HeatExact()
    X, Y = W.grid_xy(desc)
    s2 = ex.src(X, Y, 2 * h["dt"]) + ex.src(X, Y, 3 * h["dt"])
    assert np.allclose(h["src_coef"][1] * h["src_profile"], s2, rtol=1e-14, atol=1e-14)


def test_binding_wrappers_expose_the_entry_points():
    for cls, names in [(kfbi.Domain, ["apply_operator", "interface_solve", "solve_density",
                                      "device_bytes"]),
                       (kfbi.State, ["init_heat", "init_wave", "init_schrodinger", "step_heat",
                                     "step_wave", "step_schrodinger", "get_u", "get_phi",
                                     "device_bytes"]),
                       (kfbi.Batch, ["step", "tuning"]),
                       (kfbi.Server, ["submit", "tick", "run", "info", "result", "stats"]),
                       (kfbi.Plan, ["field", "device_bytes"])]:
        for n in names:
            assert callable(getattr(cls, n, None)), (cls.__name__, n)
    assert callable(kfbi.table_cache_bytes)


def test_self_checks_refuse_bad_arguments_without_touching_the_gpu(built):
    """The device self-checks validate their arguments before any CUDA call."""
    import ctypes
    m = ctypes.c_longlong(-1)
    assert built.kfbi_check_conversions(0, 0, ctypes.byref(m), None) == kfbi.KFBI_ERR_ARG
    assert built.kfbi_check_conversions(0, 16, None, None) == kfbi.KFBI_ERR_ARG
    for seconds in (0.0, -1.0, 1.5, float("nan")):
        assert built.kfbi_check_wait_timeout(seconds, None) == kfbi.KFBI_ERR_ARG
