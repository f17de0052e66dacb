"""The vertical (column) part of the HEVI 1D-IMEX method.

Test infrastructure (oracle).  All column arrays carry the vertical level as their LAST
axis (shape (..., M)); reference profiles broadcast along it.

The paper's pieces, restricted to the vertical direction z (box mesh; its radial
direction r is z here, Sec. "IMEX time integration", Eq. sieqn1d):

* D^DSS_z: the continuous-Galerkin vertical derivative on one column - the element-local
  LGL derivative (Algorithm 1, GradDiv-1D) followed by direct stiffness summation
  (Sec. "Direct stiffness summation").
* L_V: the vertical component of the Set2NC linear operator (Sec. "Equation Set2NC",
  operator L, with P' = G0 rho' + H0 theta' from Eq. 2ncp).  Box walls: no flux at the
  bottom and top, so the w-component is zero at the two end nodes.
* the Schur complement (Eqs. utteqn and helm2nc), evaluated the way the paper evaluates
  second-order terms: first grad P, then div f(P, grad P) (Sec. "Volume kernels"):
      w_p(P) = A^-1 lam (D_z P / rho0 + g P / (G0 rho0)),   zero at the end nodes,
      S(P)   = P - lam F0z w_p - lam rho0 G0 D_z w_p,
      b      = P_e - lam F0z w_a - lam rho0 G0 D_z w_a,
      w_a    = A^-1 (w_e + lam g theta'_e / theta0),        zero at the end nodes,
  with A = 1 + lam^2 (g / theta0) d(theta0)/dz and F0z = G0 d(rho0)/dz + H0 d(theta0)/dz.
* the extraction of (rho', w, theta') from P (Sec. "Implementation on manycore
  processors", item c; Eq. utteqn):  w = w_a - w_p(P),
  theta' = theta'_e - lam w d(theta0)/dz,  rho' = (P - H0 theta') / G0; u, v unchanged.
* the Jacobian of S by probing with unit vectors (Algorithm 7, BuildJacobian) and its
  banded LU without pivoting (Algorithm 9, LUdecompose), then forward/back substitution.
* the standard (non-Schur) column form the paper contrasts with the Schur form in memory
  and speed (Sec. "Performance of IMEX on manycore processors", comparison of the forms
  with a direct solver): the 3M x 3M system I - lam L_V on (rho', w, theta') itself,
  unknowns ordered level by level so that the matrix is banded (half-bandwidth 3N + 1),
  factored by the same banded LU without pivoting.

Readings where the paper defers to work not at hand: the "modified Jacobian for DSS"
(Sec. "Direct stiffness summation") is taken to be the composition above (gradient, DSS,
pointwise terms, divergence, DSS), whose half-bandwidth is 2N; the reference gradients
"computed once at startup" (Sec. "Volume kernels") are D_z applied to the nodal rho0 and
theta0.
"""
import numpy as np

from .reference import GRAV, reference_profile


def dz_matrix(mesh):
    """M x M matrix of the DSS'd vertical derivative on one column.

    Element ez gives its node m = ez*N + k the local row (2/dz) D[k, :] acting on the
    nodes ez*N .. ez*N + N, weighted by the LGL weight w_k; each row is then divided by
    the sum of its weights.  (The horizontal factors w_i w_j dx dy / 4 of the 3D local
    mass are the same for every vertical contribution at a node and cancel.)
    """
    N, nez, M = mesh.N, mesh.nez, mesh.M
    D, w = mesh.D, mesh.w
    num = np.zeros((M, M))
    den = np.zeros(M)
    for ez in range(nez):
        for k in range(N + 1):
            m = ez * N + k
            for n in range(N + 1):
                num[m, ez * N + n] += w[k] * D[k, n] * (2.0 / mesh.dz)
            den[m] += w[k]
    return num / den[:, None]


def _dz(Dz, f):
    """Apply D_z along the last axis."""
    return f @ Dz.T


def _zero_ends(f):
    f = np.array(f, dtype=np.float64, copy=True)
    f[..., 0] = 0.0
    f[..., -1] = 0.0
    return f


class Column:
    """Reference profile and vertical operators of one column of a box mesh."""

    def __init__(self, mesh, theta_s=300.0, n_bv=0.0):
        self.mesh = mesh
        self.M = mesh.M
        self.half_band = 2 * mesh.N
        self.Dz = dz_matrix(mesh)
        self.z = mesh.axis_coords(mesh.nez, mesh.dz)
        ref = reference_profile(self.z, theta_s, n_bv)
        self.theta0, self.rho0, self.P0 = ref["theta0"], ref["rho0"], ref["P0"]
        self.G0, self.H0 = ref["G0"], ref["H0"]
        # D_z annihilates constants (its rows sum to zero), so the surface value is taken
        # out first: exact in real arithmetic, and an isentropic theta0 gets a gradient of
        # exactly zero instead of rounding noise.
        self.drho0 = self.Dz @ (self.rho0 - self.rho0[0])
        self.dtheta0 = self.Dz @ (self.theta0 - self.theta0[0])
        self.F0z = self.G0 * self.drho0 + self.H0 * self.dtheta0

    # ---- Set2NC vertical linear operator -------------------------------------
    def A(self, lam):
        """A = 1 + lam^2 (g/theta0) d(theta0)/dz (Eq. utteqn, vertical component)."""
        return 1.0 + lam * lam * GRAV * self.dtheta0 / self.theta0

    def L_V(self, rho, w, theta):
        """Vertical linear operator: returns (L_rho, L_w, L_theta); L_u = L_v = 0."""
        P = self.G0 * rho + self.H0 * theta
        Lrho = -(w * self.drho0 + self.rho0 * _dz(self.Dz, w))
        Lw = _zero_ends(-(_dz(self.Dz, P) / self.rho0 + GRAV * rho / self.rho0))
        Ltheta = -(w * self.dtheta0)
        return Lrho, Lw, Ltheta

    # ---- Schur complement (Eqs. utteqn, helm2nc) ------------------------------
    def w_p(self, P, lam):
        return _zero_ends(lam * (_dz(self.Dz, P) / self.rho0 + GRAV * P / (self.G0 * self.rho0))
                          / self.A(lam))

    def w_a(self, w_e, theta_e, lam):
        return _zero_ends((w_e + lam * GRAV * theta_e / self.theta0) / self.A(lam))

    def schur_apply(self, P, lam):
        """Left-hand side S(P) (Algorithm 5, LHS-Schur, for Set2NC in 1D)."""
        wp = self.w_p(P, lam)
        return P - lam * self.F0z * wp - lam * self.rho0 * self.G0 * _dz(self.Dz, wp)

    def schur_rhs(self, rho_e, w_e, theta_e, lam):
        """Right-hand side b (Algorithm 4, RHS-Schur, for Set2NC in 1D).  Returns (b, w_a)."""
        Pe = self.G0 * rho_e + self.H0 * theta_e
        wa = self.w_a(w_e, theta_e, lam)
        return Pe - lam * self.F0z * wa - lam * self.rho0 * self.G0 * _dz(self.Dz, wa), wa

    def extract(self, P, wa, theta_e, lam):
        """(rho', w, theta') from the solved pressure P."""
        w = wa - self.w_p(P, lam)
        theta = theta_e - lam * w * self.dtheta0
        rho = (P - self.H0 * theta) / self.G0
        return rho, w, theta

    # ---- Jacobian ---------------------------------------------------------------
    def jacobian_by_probing(self, lam):
        """Algorithm 7 (BuildJacobian), Schur form (one dof per node): column m of S is
        the left-hand side applied to the unit vector at node m."""
        M = self.M
        S = np.zeros((M, M))
        for m in range(M):
            e = np.zeros(M)
            e[m] = 1.0
            S[:, m] = self.schur_apply(e, lam)
        return S

    def jacobian_direct(self, lam):
        """The same matrix written as a product of matrices."""
        M = self.M
        Dz, I = self.Dz, np.eye(M)
        Z = np.diag(np.r_[0.0, np.ones(M - 2), 0.0])
        Wp = Z @ np.diag(lam / self.A(lam)) @ (np.diag(1.0 / self.rho0) @ Dz
                                                + np.diag(GRAV / (self.G0 * self.rho0)))
        return I - lam * np.diag(self.F0z) @ Wp - lam * np.diag(self.rho0 * self.G0) @ Dz @ Wp

    def standard_matrix(self, lam):
        """(I - lam L_V) on the unknowns [rho'(M), w(M), theta'(M)] (the non-Schur form,
        Eq. imex2nc, vertical part).  The w rows of the two end nodes are replaced by the
        wall condition w = 0."""
        M = self.M
        Dz, I = self.Dz, np.eye(M)
        K = np.zeros((3 * M, 3 * M))
        r, w, t = slice(0, M), slice(M, 2 * M), slice(2 * M, 3 * M)
        K[r, r] = I
        K[r, w] = lam * (np.diag(self.drho0) + np.diag(self.rho0) @ Dz)
        K[w, r] = lam * (np.diag(1.0 / self.rho0) @ Dz @ np.diag(self.G0) + np.diag(GRAV / self.rho0))
        K[w, w] = I
        K[w, t] = lam * (np.diag(1.0 / self.rho0) @ Dz @ np.diag(self.H0))
        K[t, w] = lam * np.diag(self.dtheta0)
        K[t, t] = I
        for m in (0, M - 1):
            K[M + m, :] = 0.0
            K[M + m, M + m] = 1.0
        return K


def lu_nopivot_banded(A, half_band):
    """Algorithm 9 (LUdecompose): Doolittle LU without pivoting, restricted to the band.

    For each pivot k, the rows i in (k, min(k + half_band + 1, M)) below it are scaled by
    1/A[k,k] and the trailing band block is updated.  Returns one matrix holding the unit
    lower factor L (below the diagonal) and U (on and above it).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    M = A.shape[0]
    for k in range(M):
        E = min(k + half_band + 1, M)
        if A[k, k] == 0.0 or not np.isfinite(A[k, k]):
            raise ZeroDivisionError("zero or non-finite pivot at %d" % k)
        A[k + 1:E, k] /= A[k, k]
        A[k + 1:E, k + 1:E] -= np.outer(A[k + 1:E, k], A[k, k + 1:E])
    return A


def lu_solve_banded(LU, half_band, b):
    """Forward substitution with the unit lower factor, then back substitution with U.
    ``b`` has the level as its last axis; any leading axes are independent columns."""
    b = np.array(b, dtype=np.float64, copy=True)
    M = LU.shape[0]
    y = np.empty_like(b)
    for i in range(M):
        lo = max(0, i - half_band)
        y[..., i] = b[..., i] - y[..., lo:i] @ LU[i, lo:i]
    x = np.empty_like(b)
    for i in range(M - 1, -1, -1):
        hi = min(M, i + half_band + 1)
        x[..., i] = (y[..., i] - x[..., i + 1:hi] @ LU[i, i + 1:hi]) / LU[i, i]
    return x


def implicit_solve(col, LU, q_e, lam):
    """Solve q = q_e + lam L_V(q) for every column with the Schur form.

    ``q_e`` has shape (5, ncol, M) in the order (rho', u, v, w, theta'); ``LU`` is the
    banded factorisation of S(lam).  u and v are unchanged (L_V has no horizontal part).
    """
    rho_e, u_e, v_e, w_e, th_e = q_e
    b, wa = col.schur_rhs(rho_e, w_e, th_e, lam)
    P = lu_solve_banded(LU, col.half_band, b)
    rho, w, th = col.extract(P, wa, th_e, lam)
    return np.stack([rho, u_e, v_e, w, th])


def standard_interleaved(col, lam):
    """``Column.standard_matrix`` with the unknowns ordered level by level, (rho', w,
    theta') at each level: unknown 3*m + v is variable v at level m."""
    K = col.standard_matrix(lam)
    M = col.M
    perm = np.array([v * M + m for m in range(M) for v in range(3)])
    return K[np.ix_(perm, perm)]


def standard_half_band(mesh):
    """Half-bandwidth of the interleaved standard matrix: rho' and theta' couple to w over
    the N levels on either side (the D_z stencil), 3 unknowns per level: 3N + 1."""
    return 3 * mesh.N + 1


def implicit_solve_standard(col, LUs, q_e, lam):
    """Solve q = q_e + lam L_V(q) for every column with the standard form: the banded LU
    ``LUs`` of ``standard_interleaved(col, lam)`` and forward/back substitution.  The w
    equations of the two end nodes are the wall condition w = 0 (as in the Schur form, where
    w_a and w_p vanish there).  Shapes as ``implicit_solve``."""
    rho_e, u_e, v_e, w_e, th_e = q_e
    M = col.M
    rhs = np.stack([rho_e, w_e, th_e], axis=-1)          # (..., M, 3)
    rhs[..., 0, 1] = 0.0
    rhs[..., M - 1, 1] = 0.0
    x = lu_solve_banded(LUs, 3 * col.mesh.N + 1, rhs.reshape(rhs.shape[:-2] + (3 * M,)))
    x = x.reshape(x.shape[:-1] + (M, 3))
    return np.stack([x[..., 0], u_e, v_e, x[..., 1], x[..., 2]])

