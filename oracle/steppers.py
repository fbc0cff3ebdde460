"""Oracle time steppers: Procedure 3 of Sec. 3.3 with the semi-discretisations
of Sec. 3.1 (arXiv 2404.14864).

Each time step solves one modified-Helmholtz Dirichlet problem
Delta u - kappa u = -F in Omega, u = g on Gamma (Eq. 3.13 with f = -F) by
the boundary integral equation of Eq. 3.17:

  b = g - u+[phi = 0, f-tilde]          (Y f at the boundary nodes)
  (1/2 I + W) phi = b                    (GMRES, or the Richardson iteration
                                          of Eq. 3.21; phi_0 = 2 phi^n - phi^(n-1))
  U = interface solution for (f-tilde, phi), u^{n+1} = U on Omega nodes.

The right-hand side F is carried as its own variable (Eqs. 3.4 and the
unnumbered wave recurrence after Eq. 3.7), never by differencing u.

Readings where the paper is silent (Procedure 3(a) only says "calculate
F^1 by initial boundary condition"):

* Heat (Crank-Nicolson, kappa = 2/tau): the caller gives u^0, Delta u^0 and
  optional source sums; F^1 = (2/tau) u^0 + Delta u^0 + s^0 + s^1 and
  F^{n+2} = (4/tau) u^{n+1} - F^{n+1} + s^{n+1} + s^{n+2} (Eq. 3.4 with a
  source term added to u_t = Delta u + s).
* Wave (theta-scheme, Eq. 3.5, kappa = 1/(theta tau^2), theta = 1/4 gives
  4/tau^2): the caller gives u^0, u^1, Delta u^0, Delta u^1;
  F^1 = kappa u^1 - Delta u^1,
  F^2 = kappa (2 u^1 - u^0) + ((1 - 2 theta)/theta) Delta u^1 + Delta u^0,
  F^{n+2} = (kappa/theta) u^{n+1} - ((1 - 2 theta)/theta) F^{n+1} - F^n
  (for theta = 1/4: 16/tau^2, 2, 1 as printed).
* Schroedinger (Strang, A = -i Delta as in Eq. 2.2, B = -i (v + w|u|^2)):
  u* = u^n - i (tau/2) Delta u^n (Step 1); u** from the pointwise
  Crank-Nicolson step of Eq. 3.10, closed form for w = 0; Step 3 (Eq. 3.12)
  is Delta u - kappa u = -kappa u** with kappa = 2i/tau.  Delta u^{n+1} then
  equals kappa (u^{n+1} - u**), so the next u* = 2 u^{n+1} - u**; the first
  step uses the caller's Delta u^0.
"""

import numpy as np

from .gmres import gmres, richardson
from .interface import apply_neumann, apply_operator, interface_solve


class _Base:
    def __init__(self, dom, tau, tol=1e-10, restart=50, maxit=2000, solver="gmres", gamma=0.5,
                 bc="dirichlet"):
        self.dom, self.tau = dom, float(tau)
        self.tol, self.restart, self.maxit = tol, restart, maxit
        self.solver, self.gamma = solver, gamma
        self.bc = bc
        self.mask = dom.interior_inside()
        self.phi = None
        self.phi_prev = None
        self.iters = []

    def _solve(self, kappa, F, g):
        """u^{n+1} on the grid for Delta u - kappa u = -F with u = g on Gamma
        (Eq. 3.17), or d_n u = g on Gamma when bc == "neumann" (Eq. 3.19,
        u = Y f - V psi of Eq. 3.20; the density is then psi)."""
        dom = self.dom
        Ft = np.where(self.mask, -F, 0.0)
        op = apply_neumann if self.bc == "neumann" else apply_operator
        b = np.asarray(g) - op(dom, kappa, np.zeros(dom.nb, dtype=Ft.dtype), Ft)
        # initial density: zero, the previous density, then the linear
        # extrapolation in time 2 phi^n - phi^(n-1) (the paper leaves the
        # initial value open)
        if self.phi is None:
            x0 = np.zeros(dom.nb, dtype=b.dtype)
        elif self.phi_prev is None:
            x0 = self.phi
        else:
            x0 = 2.0 * self.phi - self.phi_prev
        self.phi_prev = self.phi
        A = lambda v: op(dom, kappa, v)
        if self.solver == "richardson":
            phi, it, res, ok = richardson(A, b, x0, self.gamma, self.tol, self.maxit)
        else:
            phi, it, res, ok = gmres(A, b, x0, self.tol, self.restart, self.maxit)
        if not ok:
            raise RuntimeError("%s did not converge (res %.3e)" % (self.solver, res))
        self.phi = phi
        self.iters.append(it)
        if self.bc == "neumann":
            _, U = interface_solve(dom, kappa, np.zeros(dom.nb, dtype=phi.dtype), Ft, phi)
        else:
            _, U = interface_solve(dom, kappa, phi, Ft)
        return U


class HeatStepper(_Base):
    """u_t = Delta u + s, Crank-Nicolson (Eqs. 3.1-3.4)."""

    def init(self, u0, lap_u0, src_sum=None):
        self.kappa = 2.0 / self.tau
        self.F = (2.0 / self.tau) * np.asarray(u0) + np.asarray(lap_u0)
        if src_sum is not None:
            self.F = self.F + src_sum
        self.u = np.array(u0, copy=True)

    def step(self, g_next, src_sum_next=None):
        """Advance one step; src_sum_next = s^{n+1} + s^{n+2} on the grid."""
        U = self._solve(self.kappa, self.F, g_next)
        self.u = U
        self.F = (4.0 / self.tau) * U - self.F
        if src_sum_next is not None:
            self.F = self.F + src_sum_next
        return U


class WaveStepper(_Base):
    """u_tt = Delta u, implicit theta-scheme (Eqs. 3.5-3.7)."""

    def init(self, u0, lap_u0, u1, lap_u1, theta=0.25):
        th = float(theta)
        self.theta = th
        self.kappa = 1.0 / (th * self.tau ** 2)
        c = (1.0 - 2.0 * th) / th
        self.F_prev = self.kappa * np.asarray(u1) - np.asarray(lap_u1)
        self.F = self.kappa * (2.0 * np.asarray(u1) - np.asarray(u0)) + c * np.asarray(lap_u1) \
            + np.asarray(lap_u0)
        self.u = np.array(u1, copy=True)

    def step(self, g_next):
        U = self._solve(self.kappa, self.F, g_next)
        self.u = U
        c = (1.0 - 2.0 * self.theta) / self.theta
        F_next = (self.kappa / self.theta) * U - c * self.F - self.F_prev
        self.F_prev, self.F = self.F, F_next
        return U


class SchrodingerStepper(_Base):
    """-i u_t + Delta u + v u + w |u|^2 u = 0 (Eq. 2.2), Strang splitting."""

    def init(self, u0, lap_u0):
        self.kappa = 2.0j / self.tau
        u0 = np.asarray(u0, dtype=np.complex128)
        self.ustar = u0 - 0.5j * self.tau * np.asarray(lap_u0, dtype=np.complex128)
        self.u = u0.copy()

    def b_step(self, ustar, v, w=0.0, tol=1e-15, maxit=50):
        """Pointwise Crank-Nicolson step of Eq. 3.10 for iu_t = (v + w|u|^2) u.

        With c = tau/2 the step is u + i c (v + w|u|^2) u = R,
        R = u* - i c (v + w|u*|^2) u*.  For w = 0 it is linear:
        u = (1 - i c v)/(1 + i c v) u*.  For w != 0 it is solved, as the
        paper says, by Newton's method, here on the real 2x2 system in
        (Re u, Im u) at every node, from u = u* until the update is below
        tol |u| (quadratic convergence; maxit bounds it)."""
        ustar = np.asarray(ustar, dtype=np.complex128)
        v = np.asarray(v, dtype=np.float64)
        c = 0.5 * self.tau
        if w == 0.0:
            a = 1j * c * v
            return (1.0 - a) / (1.0 + a) * ustar
        R = ustar - 1j * c * (v + w * np.abs(ustar) ** 2) * ustar
        x, y = ustar.real.copy(), ustar.imag.copy()
        for _ in range(maxit):
            al = c * (v + w * (x * x + y * y))
            # F(x, y) = (x - al y - Re R, y + al x - Im R), al = c (v + w (x^2 + y^2))
            f1 = x - al * y - R.real
            f2 = y + al * x - R.imag
            dx_al, dy_al = 2.0 * c * w * x, 2.0 * c * w * y
            j11, j12 = 1.0 - y * dx_al, -al - y * dy_al
            j21, j22 = al + x * dx_al, 1.0 + x * dy_al
            det = j11 * j22 - j12 * j21
            d1 = (j22 * f1 - j12 * f2) / det
            d2 = (j11 * f2 - j21 * f1) / det
            x, y = x - d1, y - d2
            if np.max(np.hypot(d1, d2) / np.maximum(np.hypot(x, y), 1e-300)) <= tol:
                break
        return x + 1j * y

    def step(self, g_next, v, w=0.0):
        uss = self.b_step(self.ustar, v, w)
        # Step 3 (Eq. 3.12): Delta u - kappa u = -kappa u**, i.e. F = kappa u**.
        U = self._solve(self.kappa, self.kappa * uss, g_next)
        self.u = U
        self.ustar = 2.0 * U - uss
        return U
