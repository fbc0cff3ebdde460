"""GPU test of kfbi_box_solve_noalloc, the entry point for callers that
cannot allocate device memory (its work space is a static device array).

Its output must equal the grid solution of the existing entry point
kfbi_interface_solve when that call's corrections vanish: density zero and
a source that is zero on every irregular node and on the nodes its
extrapolation of f reads, so the corrected right-hand side is the source
itself.  Two calls in a row (real, then complex kappa) are checked.  It is
also compared with the oracle's box solve (the DST-I formula of Eq. 3.31
written out in float64) at the smallest and the largest grid it takes and on
a stream of its own, and grids outside 2 <= M <= 257 and wrongly typed
tensors are rejected.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _deep_interior_source(desc, cplx):
    """Smooth source on nodes whose 5x5 neighbourhood lies inside Omega."""
    M = desc["M"]
    ins = kfbi.Plan(desc).field("inside").reshape(M + 1, M + 1).astype(bool)
    deep = np.ones_like(ins)
    for dj in range(-2, 3):
        for di in range(-2, 3):
            deep &= np.roll(np.roll(ins, dj, 0), di, 1)
    deep = deep[1:-1, 1:-1]
    X, Y = W.grid_xy(desc)
    f = 40.0 * np.sin(3 * X + 0.5) * np.cos(2 * Y) + 7.0
    if cplx:
        f = f * (0.6 - 0.8j)
    return np.where(deep, f, 0.0)


def test_box_solve_noalloc_matches_interface_solve_twice():
    ensure_built()
    desc = W.domain_desc(200, W.star(), nb=400)   # 199^2 unknowns, padded to 256
    M, lo, hi = desc["M"], desc["lo"], desc["hi"]
    h = (hi - lo) / M
    dom = kfbi.Domain(desc, kfbi.KFBI_FP64)
    for kappa in (2.0 / h, 2.0j / (0.5 * h)):
        cplx = isinstance(kappa, complex)
        f = _deep_interior_source(desc, cplx)
        phi = np.zeros(desc["nb"], dtype=np.complex128 if cplx else np.float64)
        _, U_ref = dom.interface_solve(kappa, dev(phi), dev(f))
        u = dev(np.zeros_like(f))
        kfbi.kfbi_box_solve_noalloc(M, lo, hi, kappa, dev(f), u)
        assert rel_linf(host(u), host(U_ref)) <= TOL
    dom.close()


@pytest.mark.parametrize("M", [2, 3, 130, 257])
def test_box_solve_noalloc_matches_oracle_on_own_stream(M):
    """Against the oracle's box solve, on a non-default stream: M = 2 (one
    unknown, padded to 128) through M = 257 (the largest padded size, 256)."""
    import torch
    ensure_built()
    rng = np.random.default_rng(M)
    lo, hi = -1.0, 1.0
    h = (hi - lo) / M
    n1 = M - 1
    st = torch.cuda.Stream()
    for kappa in (2.0 / h, 3.0 + 2.0j / h):
        cplx = isinstance(kappa, complex)
        R = rng.standard_normal((n1, n1))
        if cplx:
            R = R + 1j * rng.standard_normal((n1, n1))
        ref = oracle.box_solve(R, kappa, M, h)
        f = dev(R.reshape(-1))
        u = dev(np.zeros(n1 * n1, dtype=R.dtype))
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            kfbi.kfbi_box_solve_noalloc(M, lo, hi, kappa, f, u, stream=st)
        st.synchronize()
        assert rel_linf(host(u).reshape(n1, n1), ref) <= TOL


def test_box_solve_noalloc_rejects_bad_sizes_and_types():
    ensure_built()
    import torch
    f = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.kfbi_box_solve_noalloc(301, -1.0, 1.0, 10.0, f, f)
    assert e.value.status == kfbi.KFBI_ERR_ARG
    one = torch.zeros(0, dtype=torch.float64, device="cuda")
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.kfbi_box_solve_noalloc(1, -1.0, 1.0, 10.0, one, one)
    assert e.value.status == kfbi.KFBI_ERR_ARG
    g = torch.zeros(15 * 15, dtype=torch.float64, device="cuda")
    with pytest.raises(kfbi.KfbiError):   # complex kappa needs complex128 data
        kfbi.kfbi_box_solve_noalloc(16, -1.0, 1.0, 1.0 + 2.0j, g, g)
    with pytest.raises(kfbi.KfbiError):   # too few values
        kfbi.kfbi_box_solve_noalloc(17, -1.0, 1.0, 10.0, g, g)
