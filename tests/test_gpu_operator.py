"""GPU parity of the float64 operator application (kfbi_apply_operator,
kfbi_interface_solve, kfbi_solve_density) against the oracle, through the
C ABI.  Bar: 1e-10 relative L-infinity."""

import math

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
TOL = 1e-10

CASES = [
    ("star-64", W.domain_desc(64, W.star())),
    ("ellipse-48", W.domain_desc(48, W.ellipse(), nb=80)),
    ("flower-130", W.domain_desc(130, W.flower(), nb=260)),   # two 128-tiles + ragged tail
]


def _inputs(desc, cplx, seed=3):
    d = oracle.make_domain(desc)
    rng = np.random.default_rng(seed)
    phi = np.cos(3 * d.theta) + 0.2 * np.sin(5 * d.theta) + 0.05 * rng.standard_normal(d.nb)
    X, Y = W.grid_xy(desc)
    f = 30.0 * np.sin(2 * X + 1) * np.cosh(Y) + rng.standard_normal(X.shape)
    if cplx:
        phi = phi + 1j * (np.sin(2 * d.theta) + 0.05 * rng.standard_normal(d.nb))
        f = f * (1 - 0.5j)
    return d, phi, f


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("name,desc", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["heat", "wave", "schr"])
def test_apply_operator_matches_oracle(name, desc, kind):
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    kappa = {"heat": 2.0 / h, "wave": 4.0 / (4 * h) ** 2, "schr": 2.0j / (0.5 * h)}[kind]
    cplx = isinstance(kappa, complex)
    d, phi, f = _inputs(desc, cplx)
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64)
    Ft = np.where(d.interior_inside(), f, 0.0)
    up_or, U_or = oracle.interface_solve(d, kappa, phi, Ft)
    up = host(dom.apply_operator(kappa, dev(phi), dev(f)))
    assert rel_linf(up, up_or) <= TOL
    up2, U = dom.interface_solve(kappa, dev(phi), dev(f))
    assert rel_linf(host(U), U_or) <= TOL
    assert rel_linf(host(up2), up_or) <= TOL
    # without a volume source (the GMRES operator)
    up0 = host(dom.apply_operator(kappa, dev(phi)))
    assert rel_linf(up0, oracle.apply_operator(d, kappa, phi)) <= TOL
    dom.close()


def test_zero_density_zero_source_gives_zero():
    desc = CASES[0][1]
    dom = kfbi.Domain(desc)
    import torch
    z = torch.zeros(desc["nb"], dtype=torch.float64, device="cuda")
    out = dom.apply_operator(64.0, z)
    assert float(out.abs().max()) == 0.0


def test_operator_linearity_and_repeatability():
    desc = CASES[1][1]
    d, phi, _ = _inputs(desc, False)
    dom = kfbi.Domain(desc)
    a = host(dom.apply_operator(50.0, dev(phi)))
    b = host(dom.apply_operator(50.0, dev(2.0 * phi)))
    c = host(dom.apply_operator(50.0, dev(phi)))
    assert np.array_equal(a, c)
    assert rel_linf(b, 2.0 * a) <= 1e-14


@pytest.mark.parametrize("kappa", [64.0, 128.0j])
def test_solve_density_matches_oracle(kappa):
    desc = CASES[0][1]
    d = oracle.make_domain(desc)
    cplx = isinstance(kappa, complex)
    b = np.cos(2 * d.theta) + 0.3 * np.sin(d.theta)
    if cplx:
        b = b + 0.5j * np.cos(d.theta)
    dom = kfbi.Domain(desc, tol=1e-13, restart=50, maxit=400)
    phi = dev(np.zeros_like(b))
    info = dom.solve_density(kappa, dev(b), phi)
    assert info["converged"] and info["iters"] < 80
    x_or, it, res, ok = oracle.gmres(lambda v: oracle.apply_operator(d, kappa, v), b, None,
                                     1e-13, 50, 400)
    assert ok
    assert rel_linf(host(phi), x_or) <= 1e-10


@pytest.mark.parametrize("curve", [W.ellipse(), W.star()])
def test_apply_operator_full_size_1024(curve):
    """The bench's grid (1024^2): full operator against the oracle."""
    desc = W.domain_desc(1024, curve)
    kappa = 4.0 / (4 * 2.0 / 1024) ** 2
    d, phi, f = _inputs(desc, False, seed=11)
    dom = kfbi.Domain(desc)
    Ft = np.where(d.interior_inside(), f, 0.0)
    up_or, U_or = oracle.interface_solve(d, kappa, phi, Ft)
    up, U = dom.interface_solve(kappa, dev(phi), dev(f))
    assert rel_linf(host(up), up_or) <= TOL
    assert rel_linf(host(U), U_or) <= TOL


def test_launch_count_advances():
    desc = CASES[0][1]
    d, phi, _ = _inputs(desc, False)
    dom = kfbi.Domain(desc)
    n0 = kfbi.launch_count()
    dom.apply_operator(64.0, dev(phi))
    assert kfbi.launch_count() - n0 >= 6
