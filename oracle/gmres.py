"""Oracle restarted GMRES for the Dirichlet boundary integral equation.

The paper solves Eq. 3.17, (1/2 I + W) phi = g_D - Y f, by the Richardson
iteration of Eq. 3.21 and names GMRES as the Krylov alternative (Sec. 5).
This is textbook GMRES(m): Arnoldi with modified Gram-Schmidt, Givens
rotations on the Hessenberg matrix, restart after m inner steps, stop when
the rotated residual |g_{j+1}| <= tol * ||b||_2.  Complex vectors use the
conjugating inner product.
"""

import numpy as np


def _givens(a, b):
    """c (real), s with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 * a
    if a == 0:
        return 0.0, 1.0 + 0.0 * a
    den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    return abs(a) / den, (a / abs(a)) * np.conj(b) / den


def gmres(apply_A, b, x0=None, tol=1e-10, restart=50, maxit=1000):
    """Solve A x = b.  Returns (x, iterations, relative residual estimate,
    converged flag)."""
    b = np.asarray(b)
    dt = np.result_type(b, np.float64) if x0 is None else np.result_type(b, x0, np.float64)
    x = np.zeros(len(b), dtype=dt) if x0 is None else np.array(x0, dtype=dt, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(len(b), dtype=dt), 0, 0.0, True
    it = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return x, it, beta / bnorm, True
        if it >= maxit:
            return x, it, beta / bnorm, False
        m = restart
        V = np.zeros((m + 1, len(b)), dtype=dt)
        H = np.zeros((m + 1, m), dtype=dt)
        cs = np.zeros(m); sn = np.zeros(m, dtype=dt)
        g = np.zeros(m + 1, dtype=dt)
        g[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(m):
            w = np.asarray(apply_A(V[j]), dtype=dt)
            it += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm:
                done = True
                break
            if it >= maxit or H[j, j] == 0.0:
                break
        # back substitution on the k x k upper-triangular system
        y = np.zeros(k, dtype=dt)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + V[:k].T @ y
        if done:
            return x, it, abs(g[k]) / bnorm, True


def richardson(apply_A, b, x0=None, gamma=0.5, tol=1e-10, maxit=10000):
    """The Richardson iteration of Eq. 3.21 for Eq. 3.17.

    With A = 1/2 I + W and b = g_D - Y f, Eq. 3.21 reads
    phi_{k+1} = (1 - gamma/2) phi_k + gamma (g_D - Y f - W phi_k)
              = phi_k + gamma (b - A phi_k),
    gamma in (0, 1) in the paper, which gives no value: 0.5 is the default
    read here.  Stops when ||b - A phi_k||_2 <= tol
    ||b||_2: Sec. 4 leaves the convergence norm open, and the relative
    2-norm of the residual (gamma^-1 times the change of phi) is the
    reading taken here, the same test GMRES uses.
    Returns (x, iterations, relative residual, converged flag): iterations
    counts the updates made, i.e. operator applications minus one for the
    final check."""
    b = np.asarray(b)
    dt = np.result_type(b, np.float64) if x0 is None else np.result_type(b, x0, np.float64)
    x = np.zeros(len(b), dtype=dt) if x0 is None else np.array(x0, dtype=dt, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(x), 0, 0.0, True
    it = 0
    while True:
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, it, rel, True
        if it >= maxit or not np.isfinite(rel):
            return x, it, rel, False
        x = x + gamma * r
        it += 1
