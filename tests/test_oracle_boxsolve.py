"""Pins for the oracle's box solve (Sec. 3.4.2, Eq. 3.31): DST-I orthogonality,
the eigen-relation of the 1-D second difference, and agreement with a
sparse direct solve of the same five-point system."""

import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle


@pytest.mark.parametrize("M", [2, 3, 8, 33, 64, 129])
def test_dst_orthogonality(M):
    S = oracle.dst_matrix(M)
    # S S = (M/2) I for the DST-I matrix sin(pi a i / M).
    err = np.abs(S @ S - 0.5 * M * np.eye(M - 1)).max()
    assert err <= 1e-13 * M


@pytest.mark.parametrize("M", [5, 16, 31])
def test_dst_entries_closed_form(M):
    S = oracle.dst_matrix(M)
    for a in (1, 2, M - 1):
        for i in (1, M // 2, M - 1):
            assert abs(S[a - 1, i - 1] - math.sin(math.pi * a * i / M)) < 1e-13


@pytest.mark.parametrize("M", [4, 17, 64])
def test_eigen_relation(M):
    h = 2.0 / M
    n = M - 1
    T = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2
    S = oracle.dst_matrix(M)
    lam = oracle.eigenvalues(M, h)
    resid = T @ S - S * lam[None, :]
    assert np.abs(resid).max() <= 1e-10 * np.abs(lam).max()


def _five_point(M, h, kappa):
    n = M - 1
    d2 = sp.diags([np.ones(n - 1), -2.0 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h ** 2
    I = sp.identity(n)
    # unknown index j*n + i (row j = y, column i = x)
    return (sp.kron(I, d2) + sp.kron(d2, I) - kappa * sp.identity(n * n)).tocsc()


@pytest.mark.parametrize("M", [8, 17, 32])
@pytest.mark.parametrize("kappa", [0.5, 64.0, 3.0 + 4.0j, 2.0e5, 1e6j])
def test_box_solve_matches_sparse_direct(M, kappa):
    rng = np.random.default_rng(1234 + M)
    h = 2.0 / M
    R = rng.standard_normal((M - 1, M - 1))
    if isinstance(kappa, complex):
        R = R + 1j * rng.standard_normal((M - 1, M - 1))
    U = oracle.box_solve(R, kappa, M, h)
    A = _five_point(M, h, kappa)
    if isinstance(kappa, complex):
        A = A.astype(np.complex128)
    Ud = spla.spsolve(A, R.ravel()).reshape(M - 1, M - 1)
    assert np.abs(U - Ud).max() <= 1e-12 * np.abs(Ud).max()
