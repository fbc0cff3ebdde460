"""Oracle for Procedure 2 of Sec. 3.3 (arXiv 2404.14864): one application of
the KFBI boundary-integral operator.

Given the density phi at the boundary nodes, kappa and the volume source
f-tilde on the grid, it evaluates the interior limit u+ at the boundary nodes
of the solution u of the unified interface problem (Eq. 3.30)

    Delta u - kappa u = F   in B \\ Gamma,   [u] = Phi,  [u_n] = Psi,  u = 0 on dB,

with Phi = phi, Psi = psi (zero for the Dirichlet BIE) and F = f-tilde
(Eq. 3.25), in the paper's three sub-steps:

  (a) jumps of u and its first and second derivatives at the cut-edge
      intersections (Sec. 3.2.5) and the correction terms C+ / C- added to
      the five-point right-hand side at irregular nodes (Sec. 3.2.4);
  (b) the five-point system (Eq. 3.31) with u = 0 on dB, solved by a
      forward DST-I, a division by the eigenvalues and an inverse DST-I
      (Sec. 3.4.2, "procedure 2, point 2");
  (c) boundary extraction with the six-point stencil and the 6x6 Taylor
      system of Eq. 3.36 (Sec. 3.2.6).

Readings of silent or garbled passages (each also listed in the design notes):

* Eq. 3.35, second row: the right-hand side printed as psi_s is read as psi,
  because [u_n] = n . [grad u] = tau_2 [u_x] - tau_1 [u_y] = Psi (Eq. 3.34).
* Sec. 3.2.4 labels p_{i,j} exterior and p_{i+1,j} interior but the C+
  formula uses u+ at x_i and u- at x_{i+1}; the formulas are taken as
  written: a node on the Omega side of a cut arm gets
  C = -J / h^2, a node on the Omega^c side gets C = +J / h^2, with
  J = [u] + [u_d] d + 1/2 [u_dd] d^2 and d = (neighbour coordinate - xi).
* The density is only known at the nodes; phi, phi_theta, phi_thetatheta at
  a parameter t* come from the six-point Lagrange interpolant on nodes
  k0-2 .. k0+3 with k0 = floor(t* / dtheta) (k0 = k at node k), converted to
  arc length by the chain rule.
* f at an intersection (third row of the 3x3 system) is extrapolated
  linearly along the cut edge's grid line from its Omega-side endpoint and
  the next node inward (constant when that node is outside Omega): f scales
  like 1/tau in the time steppers, and a constant extrapolation would leave
  an O(1) instead of O(h) corrected truncation error.  At a boundary node it
  is f-tilde at the Omega-side point of its extraction stencil nearest to
  the node (first in stencil order on ties); there it only enters the
  extracted value through O(h^2) Taylor terms.
* Extraction stencil of node z: p0 = nearest grid node (floor(v + 1/2) per
  axis), s = sign(z - p0) per axis with 0 -> +1; points p0, p0 +- e_x,
  p0 +- e_y, p0 + s_x e_x + s_y e_y (unisolvent for quadratics).
"""

import math

import numpy as np

# ----------------------------------------------------------------------------
# (b) box solve: five-point modified Helmholtz operator, u = 0 on dB.
# ----------------------------------------------------------------------------


def dst_matrix(M):
    """S[a-1, i-1] = sin(pi a i / M), a, i = 1..M-1 (DST-I); a*i is reduced
    modulo 2M in integers before scaling so the sine argument stays in
    [0, 2 pi)."""
    a = np.arange(1, M, dtype=np.int64)
    ai = np.mod(np.outer(a, a), 2 * M)
    return np.sin(math.pi * ai.astype(np.float64) / M)


def eigenvalues(M, h):
    """Eigenvalues of the 1-D second difference (u_{i+1} - 2u_i + u_{i-1})/h^2
    with zero end values, on the DST-I eigenvectors sin(pi a i / M)."""
    a = np.arange(1, M, dtype=np.float64)
    return -(4.0 / (h * h)) * np.sin(math.pi * a / (2.0 * M)) ** 2


def box_solve(R, kappa, M, h):
    """Solve (D_xx + D_yy - kappa) U = R on the (M-1)^2 interior nodes with
    U = 0 on the box boundary (Eq. 3.31): forward DST-I in both directions,
    divide by lambda_a + lambda_b - kappa, inverse DST-I.  R[j-1, i-1]."""
    S = dst_matrix(M)
    lam = eigenvalues(M, h)
    Rhat = S @ R @ S
    Uhat = Rhat / (lam[:, None] + lam[None, :] - kappa)
    return (2.0 / M) ** 2 * (S @ Uhat @ S)


# ----------------------------------------------------------------------------
# Density derivatives along Gamma.
# ----------------------------------------------------------------------------


def lagrange6_weights(s):
    """Weights of the Lagrange interpolant on the six local abscissae
    -2, -1, 0, 1, 2, 3 for the value, first and second derivative at local
    coordinate s (array).  Returns three arrays of shape (n, 6)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    nodes = np.arange(-2, 4, dtype=np.float64)
    n = len(s)
    w0 = np.zeros((n, 6)); w1 = np.zeros((n, 6)); w2 = np.zeros((n, 6))
    for m in range(6):
        den = 1.0
        for l in range(6):
            if l != m:
                den *= nodes[m] - nodes[l]
        others = [l for l in range(6) if l != m]
        # value: prod_l (s - t_l)
        v = np.ones(n)
        for l in others:
            v = v * (s - nodes[l])
        # first derivative: sum_l prod_{q != l} (s - t_q)
        d1 = np.zeros(n)
        for l in others:
            t = np.ones(n)
            for q in others:
                if q != l:
                    t = t * (s - nodes[q])
            d1 = d1 + t
        # second derivative: sum_{l != q} prod_{r != l, q} (s - t_r)
        d2 = np.zeros(n)
        for l in others:
            for q in others:
                if q == l:
                    continue
                t = np.ones(n)
                for r in others:
                    if r != l and r != q:
                        t = t * (s - nodes[r])
                d2 = d2 + t
        w0[:, m] = v / den
        w1[:, m] = d1 / den
        w2[:, m] = d2 / den
    return w0, w1, w2


def _stencil_of_param(dom, theta, node_k=None):
    """k0 and the local coordinate of each target parameter."""
    if node_k is not None:
        k0 = np.asarray(node_k, dtype=np.int64)
        s = np.zeros(len(k0))
        return k0, s
    q = theta / dom.dtheta
    k0 = np.floor(q).astype(np.int64)
    k0 = np.minimum(k0, dom.nb - 1)
    s = q - k0
    return k0, s


def density_derivatives(dom, dens, theta, node_k=None):
    """dens, d dens/ds, d^2 dens/ds^2 at curve parameters theta (arc length s).

    Six-point Lagrange in the curve parameter, then the chain rule with
    sigma = |z'(theta)|:  g_s = g_t / sigma,
    g_ss = (g_tt - g_t sigma_t / sigma) / sigma^2."""
    k0, s = _stencil_of_param(dom, theta, node_k)
    w0, w1, w2 = lagrange6_weights(s)
    idx = np.mod(k0[:, None] + np.arange(-2, 4)[None, :], dom.nb)
    vals = dens[idx]
    g = np.sum(w0 * vals, axis=1)
    g_t = np.sum(w1 * vals, axis=1) / dom.dtheta
    g_tt = np.sum(w2 * vals, axis=1) / dom.dtheta ** 2
    th = theta if node_k is None else dom.theta[np.asarray(node_k)]
    dx, dy = dom.curve.dz(th)
    ddx, ddy = dom.curve.d2z(th)
    sigma = np.hypot(dx, dy)
    sigma_t = (dx * ddx + dy * ddy) / sigma
    g_s = g_t / sigma
    g_ss = (g_tt - g_t * sigma_t / sigma) / sigma ** 2
    return g, g_s, g_ss


def tangent_data(dom, theta):
    """Unit tangent (tau1, tau2) and its arc-length derivative (tau1', tau2')."""
    dx, dy = dom.curve.dz(theta)
    ddx, ddy = dom.curve.d2z(theta)
    sigma = np.hypot(dx, dy)
    sigma_t = (dx * ddx + dy * ddy) / sigma
    t1, t2 = dx / sigma, dy / sigma
    # d tau / ds = (z'' / sigma - z' sigma_t / sigma^2) / sigma
    t1p = (ddx / sigma - dx * sigma_t / sigma ** 2) / sigma
    t2p = (ddy / sigma - dy * sigma_t / sigma ** 2) / sigma
    return t1, t2, t1p, t2p


# ----------------------------------------------------------------------------
# (a) jumps (Sec. 3.2.5) and corrections (Sec. 3.2.4).
# ----------------------------------------------------------------------------


def jump_matrix3(t1, t2):
    """Coefficient matrix of the 3x3 system for ([u_xx], [u_xy], [u_yy])."""
    t1 = np.atleast_1d(t1); t2 = np.atleast_1d(t2)
    A = np.zeros((len(t1), 3, 3))
    A[:, 0, 0] = t1 * t1; A[:, 0, 1] = 2.0 * t1 * t2; A[:, 0, 2] = t2 * t2
    A[:, 1, 0] = t1 * t2; A[:, 1, 1] = t2 * t2 - t1 * t1; A[:, 1, 2] = -t1 * t2
    A[:, 2, 0] = 1.0; A[:, 2, 1] = 0.0; A[:, 2, 2] = 1.0
    return A


def jumps_at(dom, theta, phi, f_gamma, kappa, psi=None, node_k=None):
    """Jumps ([u], [u_x], [u_y], [u_xx], [u_xy], [u_yy]) at parameters theta.

    [u] = phi, [u_n] = psi on Gamma (Eqs. 3.33-3.34); the first derivatives
    solve the 2x2 system of Eq. 3.35 (second row read as = psi), the second
    derivatives the 3x3 system of Sec. 3.2.5 whose last row is the jump of
    the PDE: [u_xx] + [u_yy] = f + kappa [u]."""
    th = theta if node_k is None else dom.theta[np.asarray(node_k)]
    cplx = np.iscomplexobj(phi) or np.iscomplexobj(f_gamma) or np.iscomplexobj(kappa) \
        or (psi is not None and np.iscomplexobj(psi))
    dt = np.complex128 if cplx else np.float64
    phi = np.asarray(phi, dtype=dt)
    psi = np.zeros(dom.nb, dtype=dt) if psi is None else np.asarray(psi, dtype=dt)
    n = len(th)
    p0, p_s, p_ss = density_derivatives(dom, phi, theta, node_k)
    q0, q_s, _ = density_derivatives(dom, psi, theta, node_k)
    t1, t2, t1p, t2p = tangent_data(dom, th)
    # Eq. 3.35: tau1 [u_x] + tau2 [u_y] = phi_s ; tau2 [u_x] - tau1 [u_y] = psi
    A2 = np.zeros((n, 2, 2))
    A2[:, 0, 0] = t1; A2[:, 0, 1] = t2; A2[:, 1, 0] = t2; A2[:, 1, 1] = -t1
    rhs2 = np.stack([p_s, q0], axis=1).astype(dt)
    g1 = np.linalg.solve(A2.astype(dt), rhs2[:, :, None])[:, :, 0]
    ux, uy = g1[:, 0], g1[:, 1]
    # 3x3 system of Sec. 3.2.5.
    A3 = jump_matrix3(t1, t2).astype(dt)
    rhs3 = np.stack([
        p_ss - (t1p * ux + t2p * uy),
        q_s - t2p * ux + t1p * uy,
        np.asarray(f_gamma, dtype=dt) + kappa * p0,
    ], axis=1)
    g2 = np.linalg.solve(A3, rhs3[:, :, None])[:, :, 0]
    out = np.zeros((n, 6), dtype=dt)
    out[:, 0] = p0; out[:, 1] = ux; out[:, 2] = uy
    out[:, 3] = g2[:, 0]; out[:, 4] = g2[:, 1]; out[:, 5] = g2[:, 2]
    return out


def edge_f_gamma(dom, Ft):
    """f at every cut-edge intersection, extrapolated linearly along the edge's
    grid line from the Omega-side endpoint p and the next node p2 further
    inside: f(p) + (f(p) - f(p2)) delta / h, delta = |intersection - p|;
    f(p) alone when p2 is not in Omega."""
    i, j, d, c = dom.edge_i, dom.edge_j, dom.edge_dir, dom.edge_coord
    horiz = d == 0
    qi = i + horiz; qj = j + (~horiz)
    p_in = dom.inside[j, i]
    pi_ = np.where(p_in, i, qi); pj = np.where(p_in, j, qj)
    # step from p away from the intersection (into Omega): -1 if p is the
    # lower/left endpoint, +1 otherwise
    step = np.where(p_in, -1, 1)
    p2i = np.where(horiz, pi_ + step, pi_)
    p2j = np.where(horiz, pj, pj + step)
    fp = Ft[pj - 1, pi_ - 1]
    ok = dom.inside[p2j, p2i]
    fp2 = Ft[np.clip(p2j - 1, 0, dom.M - 2), np.clip(p2i - 1, 0, dom.M - 2)]
    delta = np.abs(c - np.where(horiz, dom.x[pi_], dom.x[pj]))
    return np.where(ok, fp + (fp - fp2) * (delta / dom.h), fp)


def correction_rhs(dom, Ft, edge_jumps):
    """Five-point right-hand side F-tilde + C at every interior node: every
    cut edge contributes C+ (Omega side, -J/h^2) or C- (Omega^c side,
    +J/h^2) to each of its two endpoints (Sec. 3.2.4)."""
    h = dom.h
    R = np.array(Ft, dtype=np.result_type(Ft, edge_jumps), copy=True)
    i, j, d, xi = dom.edge_i, dom.edge_j, dom.edge_dir, dom.edge_coord
    horiz = d == 0
    u0 = edge_jumps[:, 0]
    u1 = np.where(horiz, edge_jumps[:, 1], edge_jumps[:, 2])   # [u_x] or [u_y]
    u2 = np.where(horiz, edge_jumps[:, 3], edge_jumps[:, 5])   # [u_xx] or [u_yy]
    qi = i + horiz; qj = j + (~horiz)
    # endpoint p = (i, j) has neighbour q; endpoint q has neighbour p.
    for (ni, nj), (mi, mj) in (((i, j), (qi, qj)), ((qi, qj), (i, j))):
        cm = np.where(horiz, dom.x[mi], dom.x[mj])   # neighbour coordinate
        dd = cm - xi
        J = u0 + u1 * dd + 0.5 * u2 * dd * dd
        sign = np.where(dom.inside[nj, ni], -1.0, 1.0)
        np.add.at(R, (nj - 1, ni - 1), sign * J / (h * h))
    return R


# ----------------------------------------------------------------------------
# (c) boundary extraction (Sec. 3.2.6, Eq. 3.36).
# ----------------------------------------------------------------------------


def extraction_stencil(dom):
    """Six stencil points (i, j) per boundary node, arrays of shape (nb, 6)."""
    vx = (dom.zx - dom.lo) / dom.h
    vy = (dom.zy - dom.lo) / dom.h
    i0 = np.floor(vx + 0.5).astype(np.int64)
    j0 = np.floor(vy + 0.5).astype(np.int64)
    sx = np.where(dom.zx - dom.x[i0] >= 0.0, 1, -1)
    sy = np.where(dom.zy - dom.x[j0] >= 0.0, 1, -1)
    si = np.stack([i0, i0 + 1, i0 - 1, i0, i0, i0 + sx], axis=1)
    sj = np.stack([j0, j0, j0, j0 + 1, j0 - 1, j0 + sy], axis=1)
    return si, sj


def node_f_gamma(dom, Ft):
    """f-tilde at the Omega-side stencil point nearest each boundary node."""
    si, sj = extraction_stencil(dom)
    ins = dom.inside[sj, si]
    if not ins.any(axis=1).all():
        raise ValueError("an extraction stencil has no point in Omega")
    dist = (dom.x[si] - dom.zx[:, None]) ** 2 + (dom.x[sj] - dom.zy[:, None]) ** 2
    m = np.argmin(np.where(ins, dist, np.inf), axis=1)   # first minimum on ties
    k = np.arange(dom.nb)
    return Ft[sj[k, m] - 1, si[k, m] - 1]


def extraction(dom, U, node_jumps, normal=False):
    """u+ at every boundary node from the 6x6 Taylor system of Eq. 3.36:
    U(p) + J(p) [p in Omega^c] = U+ + U+_x xi + U+_y eta + U+_xx xi^2/2
    + U+_xy xi eta + U+_yy eta^2/2, (xi, eta) = p - z.  With normal=True the
    interior normal derivative d_n u+ = n_x U+_x + n_y U+_y, n = (tau2, -tau1)
    the outward normal of Sec. 3.2.5 (the data the Neumann BIE, Eq. 3.19,
    needs)."""
    si, sj = extraction_stencil(dom)
    dt = np.result_type(U, node_jumps)
    xi = dom.x[si] - dom.zx[:, None]          # (nb, 6)
    eta = dom.x[sj] - dom.zy[:, None]
    A = np.stack([np.ones_like(xi), xi, eta, 0.5 * xi * xi, xi * eta, 0.5 * eta * eta], axis=2)
    jm = node_jumps[:, None, :]               # jumps at z_k for all six points
    J = (jm[..., 0] + jm[..., 1] * xi + jm[..., 2] * eta + 0.5 * jm[..., 3] * xi * xi
         + jm[..., 4] * xi * eta + 0.5 * jm[..., 5] * eta * eta)
    b = U[sj - 1, si - 1] + np.where(dom.inside[sj, si], 0.0, J)
    c = np.linalg.solve(A.astype(dt), b.astype(dt)[:, :, None])[:, :, 0]
    if not normal:
        return c[:, 0]
    t1, t2, _, _ = tangent_data(dom, dom.theta)
    return t2 * c[:, 1] - t1 * c[:, 2]


# ----------------------------------------------------------------------------
# Procedure 2 end to end.
# ----------------------------------------------------------------------------


def interface_solve(dom, kappa, phi, Ft=None, psi=None, normal=False):
    """Grid solution U of Eq. 3.30 and the extracted u+ (or, with normal=True,
    d_n u+) at the boundary nodes.

    phi (nb,), psi (nb,) or None, Ft (M-1, M-1) f-tilde or None (zero);
    kappa real or complex.  Returns (u_plus (nb,), U (M-1, M-1))."""
    M, h = dom.M, dom.h
    cplx = np.iscomplexobj(phi) or np.iscomplexobj(kappa) or \
        (Ft is not None and np.iscomplexobj(Ft)) or (psi is not None and np.iscomplexobj(psi))
    dt = np.complex128 if cplx else np.float64
    if Ft is None:
        Ft = np.zeros((M - 1, M - 1), dtype=dt)
    Ft = np.asarray(Ft, dtype=dt)
    phi = np.asarray(phi, dtype=dt)
    # (a) jumps at the intersections, corrected right-hand side.
    ej = jumps_at(dom, dom.edge_theta, phi, edge_f_gamma(dom, Ft), kappa, psi)
    R = correction_rhs(dom, Ft, ej)
    # (b) box solve.
    U = box_solve(R, kappa, M, h)
    # (c) jumps at the boundary nodes and extraction.
    nj = jumps_at(dom, None, phi, node_f_gamma(dom, Ft), kappa, psi,
                  node_k=np.arange(dom.nb))
    return extraction(dom, U, nj, normal), U


def apply_operator(dom, kappa, phi, Ft=None, psi=None):
    """u+ at the boundary nodes (one application of the BIE operator)."""
    return interface_solve(dom, kappa, phi, Ft, psi)[0]


def apply_neumann(dom, kappa, psi, Ft=None):
    """d_n u+ at the boundary nodes of the interface solution with Phi = 0,
    Psi = psi, F = Ft (Eq. 3.30).  With Ft = None this is the Neumann BIE
    operator of Eq. 3.19: u = -V psi has [u_n] = psi (Sec. 3.2.3's table), so
    its interior normal derivative is psi/2 - d_n(V psi), the principal value
    plus half the jump; with psi = 0 it is d_n(Y f), the known term."""
    psi = np.asarray(psi)
    return interface_solve(dom, kappa, np.zeros(dom.nb, dtype=psi.dtype), Ft, psi, True)[0]
