"""3D-IMEX in the Schur form: the implicit solve with BiCGstab and a polynomial preconditioner.

Test infrastructure (oracle).  The paper's 3D-IMEX treats the whole linear operator L of
Set2NC implicitly (Sec. "Equation Set2NC", Eqs. imex2nc, 2ncp, utteqn, helm2nc):

    u_a = A^-1 (u_e + lam g z_hat H0 theta_e / (G0 rho0)),        A = I + lam^2 (g / theta0) z_hat (grad theta0)^T
    u_p(P) = A^-1 lam (grad P / rho0 + g z_hat P / (G0 rho0))
    S(P) = P - lam F0 . u_p - lam rho0 G0 div u_p                 (left-hand side)
    b    = P_e - lam F0 . u_a - lam rho0 G0 div u_a               (right-hand side)
    u = u_a - u_p(P),  theta' = theta'_e - lam u . grad theta0,  rho' = (P - H0 theta') / G0

On the box, grad rho0, grad theta0 and F0 point along z, so A acts on w alone (the 1D
column operator's A) and u_a = u_e, v_a = v_e.  Gradients and divergences are the cG
derivatives: element-local LGL derivatives, then direct stiffness summation (Algorithm 2,
Sec. "Direct stiffness summation"), with "grad P first, then div of u_p" as for the 1D
form.  Walls: each velocity component is zero on the walls normal to it (u_a and u_p
both), the condition the 1D form imposes on w at the top and bottom.

The linear system S(P) = b is solved by BiCGstab with left preconditioning by a polynomial
s(S) (Algorithm "BiCGstabPBNO" and its PBNO procedure).  The paper's PBNO coefficients come
from a non-linear least-squares fit (Carr et al. 2016), not reproduced in the paper.
Reading: the coefficients c_i make y q(y) the Chebyshev minimax approximation of 1 on the
scaled spectrum interval [1 - delta, 1 + delta], delta = (l_max - l_min)/(l_max + l_min).
The residual polynomial is then 1 - y q(y) = T_{P+1}((1 - y)/delta) / T_{P+1}(1/delta).
The spectrum bounds are estimated once at start-up (l_min = 1: S is the identity plus
lam^2 times a discrete -rho0 G0 div(grad / rho0) operator; l_max by power iteration).
"""
import numpy as np

from .ark2 import ark_step, scheme_tableau
from .reference import GRAV
from .rhs import rhs


class Schur3D:
    """The 3D Schur-form operators of one box mesh and reference state."""

    def __init__(self, mesh, col):
        self.mesh, self.col = mesh, col
        self.l2g = mesh.l2g()
        self.mass = mesh.global_mass(self.l2g)
        self.iz = np.arange(mesh.nnode) % mesh.M
        self.walls = self._walls()
        D = mesh.D
        self.s = (2.0 / mesh.dx, 2.0 / mesh.dy, 2.0 / mesh.dz)
        self.D = D

    def _walls(self):
        from .rhs import wall_masks
        return wall_masks(self.mesh)

    # -- cG derivatives of a nodal field: element-local LGL derivative, then DSS ---------
    def _d(self, f, axis):
        f_loc = f[self.l2g]                           # (E, k, j, i)
        D, s = self.D, self.s[axis]
        if axis == 0:
            d = np.einsum("in,ekjn->ekji", D, f_loc)
        elif axis == 1:
            d = np.einsum("jn,ekni->ekji", D, f_loc)
        else:
            d = np.einsum("kn,enji->ekji", D, f_loc)
        return self.mesh.dss(d * s, self.l2g, self.mass)

    def _coef(self, lam):
        c = self.col
        iz = self.iz
        A = 1.0 + lam * lam * GRAV * c.dtheta0[iz] / c.theta0[iz]
        return c.rho0[iz], c.G0[iz], c.H0[iz], c.F0z[iz], c.dtheta0[iz], A

    def u_p(self, P, lam):
        rho0, G0, _, _, _, A = self._coef(lam)
        mx, my, mz = self.walls
        up = lam * self._d(P, 0) / rho0
        vp = lam * self._d(P, 1) / rho0
        wp = lam * (self._d(P, 2) / rho0 + GRAV * P / (G0 * rho0)) / A
        up[mx] = 0.0
        vp[my] = 0.0
        wp[mz] = 0.0
        return up, vp, wp

    def _div_terms(self, u, v, w, lam):
        rho0, G0, _, F0z, _, _ = self._coef(lam)
        div = self._d(u, 0) + self._d(v, 1) + self._d(w, 2)
        return lam * F0z * w + lam * rho0 * G0 * div

    def apply(self, P, lam):
        """S(P), the left-hand side (Eq. helm2nc)."""
        up, vp, wp = self.u_p(P, lam)
        return P - self._div_terms(up, vp, wp, lam)

    def rhs(self, q_e, lam):
        """(b, (u_a, v_a, w_a)) from q~_e of shape (5, nnode) (Eq. helm2nc, right side)."""
        rho0, G0, H0, _, _, A = self._coef(lam)
        r_e, u_e, v_e, w_e, t_e = q_e
        mx, my, mz = self.walls
        ua, va = u_e.copy(), v_e.copy()
        wa = (w_e + lam * GRAV * H0 * t_e / (G0 * rho0)) / A
        ua[mx] = 0.0
        va[my] = 0.0
        wa[mz] = 0.0
        Pe = G0 * r_e + H0 * t_e
        return Pe - self._div_terms(ua, va, wa, lam), (ua, va, wa)

    def extract(self, P, ua, t_e, lam):
        _, G0, H0, _, dth0, _ = self._coef(lam)
        up, vp, wp = self.u_p(P, lam)
        u, v, w = ua[0] - up, ua[1] - vp, ua[2] - wp
        th = t_e - lam * w * dth0
        rho = (P - H0 * th) / G0
        return np.stack([rho, u, v, w, th])


def chebyshev_pbno(order, l_min, l_max):
    """(c, lam_bar) of the PBNO recursion for the Chebyshev minimax polynomial: with
    y = lam_bar x, lam_bar = 2 / (l_min + l_max), the preconditioner is
    s(x) = lam_bar sum_i c_i y^(P - i), and 1 - y sum_i c_i y^(P - i) is the scaled
    Chebyshev polynomial T_{P+1}((1 - y)/delta) / T_{P+1}(1/delta)."""
    P = int(order)
    lam_bar = 2.0 / (l_min + l_max)
    delta = (l_max - l_min) / (l_max + l_min)
    C = np.polynomial.chebyshev.Chebyshev.basis(P + 1)
    T1 = C(1.0 / delta)
    # residual r(y) = T_{P+1}((1 - y)/delta) / T_{P+1}(1/delta) as a power series in y
    t = np.polynomial.Polynomial([1.0 / delta, -1.0 / delta])
    r = C.convert(kind=np.polynomial.Polynomial)(t) / T1
    q = (np.polynomial.Polynomial([1.0]) - r) // np.polynomial.Polynomial([0.0, 1.0])
    qc = np.zeros(P + 1)
    qc[:len(q.coef)] = q.coef
    return qc[::-1].copy(), lam_bar          # c_i multiplies y^(P - i)


def pbno_apply(apply, r, c, lam_bar):
    """The PBNO procedure: r <- lam_bar r; r* = c_0 r; r* = lam_bar S(r*) + c_i r."""
    r = lam_bar * r
    rs = c[0] * r
    for i in range(1, len(c)):
        rs = lam_bar * apply(rs) + c[i] * r
    return rs


def power_lmax(apply, n, iters=60, seed=0):
    """Largest-modulus eigenvalue estimate of S by power iteration (Rayleigh quotient)."""
    x = np.random.default_rng(seed).standard_normal(n)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply(x)
        lam = float(x @ y)
        x = y / np.linalg.norm(y)
    return lam


def bicgstab_pbno(apply, b, c, lam_bar, tol=1e-12, maxit=500):
    """BiCGstab left-preconditioned by PBNO (Algorithm "BiCGstabPBNO"); x0 = 0.  Returns
    (x, iterations).  Converged when the preconditioned residual's 2-norm has dropped by
    tol."""
    return bicgstab(apply, b, lambda v: pbno_apply(apply, v, c, lam_bar), tol, maxit)


def bicgstab(apply, b, M, tol=1e-12, maxit=500):
    """The iteration of Algorithm "BiCGstabPBNO" with any left preconditioner M."""
    x = np.zeros_like(b)
    rn = M(b)
    r0n = np.linalg.norm(rn)
    if r0n == 0.0:
        return x, 0
    p = rn.copy()
    ro = rn.copy()
    for it in range(1, maxit + 1):
        Ap = M(apply(p))
        ar = (rn @ ro) / (Ap @ ro)
        s = rn - ar * Ap
        As = M(apply(s))
        wr = (As @ s) / (As @ As)
        x = x + ar * p + wr * s
        re = s - wr * As
        if np.linalg.norm(re) / r0n <= tol:
            return x, it
        br = (re @ ro) / (rn @ ro) * ar / wr
        p = re + br * (p - wr * Ap)
        rn = re
    return x, maxit


class HEVI3D:
    """3D-IMEX integrator with the Schur form and BiCGstab + polynomial preconditioner
    (oracle).  order: polynomial degree P; tol: relative preconditioned-residual drop;
    scheme: one of ``ark2.SCHEMES``; precond: "pbno" (the paper's
    polynomial preconditioner, Chebyshev reading) or "column" (the 1D column Schur LU as a
    vertical-line preconditioner, a choice beyond the paper)."""

    def __init__(self, mesh, col, dt, order=2, tol=1e-12, scheme="ark2", precond="pbno"):
        self.mesh, self.col, self.dt = mesh, col, dt
        self.tab = scheme_tableau(scheme)
        at = self.tab[1]
        self.lam = at[1, 1] * dt
        self.op = Schur3D(mesh, col)
        self.l_min = 1.0
        self.l_max = 1.05 * power_lmax(lambda x: self.op.apply(x, self.lam), mesh.nnode)
        self.c, self.lam_bar = chebyshev_pbno(order, self.l_min, self.l_max)
        self.tol = tol
        self.iters = []
        self.precond = precond
        if precond == "column":
            # the 1D-IMEX column Schur matrix of the same lam, factored by Algorithm 9: the
            # vertical (stiffest) part of S solved exactly, column by column
            from .column import lu_nopivot_banded, lu_solve_banded
            LU = lu_nopivot_banded(col.jacobian_by_probing(self.lam), col.half_band)
            hb, sh = col.half_band, (mesh.ncol, mesh.M)
            self.M = lambda v: lu_solve_banded(LU, hb, v.reshape(sh)).ravel()
        elif precond == "pbno":
            self.M = lambda v: pbno_apply(lambda x: self.op.apply(x, self.lam), v, self.c,
                                          self.lam_bar)
        else:
            raise ValueError("precond must be 'pbno' or 'column'")

    def R(self, q):
        return rhs(self.mesh, self.col, q, self.op.l2g, self.op.mass)

    def solve(self, q_e, lam):
        assert abs(lam - self.lam) <= 1e-15 * abs(self.lam)
        b, ua = self.op.rhs(q_e, lam)
        P, it = bicgstab(lambda x: self.op.apply(x, lam), b, self.M, self.tol)
        self.iters.append(it)
        return self.op.extract(P, ua, q_e[4], lam)

    def step(self, q, nsteps=1):
        for _ in range(nsteps):
            q = ark_step(q, self.dt, self.R, self.solve, self.tab)
        return q
