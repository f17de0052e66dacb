"""Tangent-linear (TLM) and adjoint models of the HEVI 1D-IMEX step.

Test infrastructure (oracle).  The paper integrates forward in time only; the
differentiation form differentiates its method with the chain rule, one step of the
forward computation at a time:

* ``rhs_tlm``: R'(q) dq for the right-hand side of ``oracle.rhs`` (Sec. "Equation
  Set2NC", Algorithm 2 and the DSS of Sec. "Direct stiffness summation"), by the product
  rule applied to every term.  The equation of state P = p00 (rho R theta / p00)^gamma
  gives dP' = gamma P (drho'/rho + dtheta'/theta).
* ``rhs_adjoint``: R'(q)^T lam, the same linear steps transposed in reverse order: wall
  mask, DSS (a mass-weighted sum into the global nodes) transposed to a weighted spread,
  the pointwise products, the element derivative (D becomes D^T), the gather transposed
  to a scatter-add, and the equation of state.
* ``lu_solve_transposed_banded``: S^T x = b with the stored factors S = L U of
  Algorithm 9: U^T y = b (forward), then L^T x = y (backward).
* ``ColumnMap``: the implicit column solve q~ = solve(q~_e) (Sec. "Linear multi-stage
  methods" with the Schur form of Eqs. utteqn and helm2nc) is linear and the same on
  every column of a box mesh (the reference state depends on z only), so its matrix is
  built by applying the oracle's solve to unit vectors (the probing idea of Algorithm 7,
  on the whole column solve) and its adjoint is the transposed matrix.
* ``step_tlm`` / ``step_adjoint``: one ARK2 step (Table 1, stage form of Sec. "Linear
  multi-stage methods") differentiated stage by stage, and run backwards.
* ``misfit`` / ``gradient``: J(q0) = 1/2 sum_g (theta'_T[g] - target[g])^2 after n steps
  and dJ/dq0 by the adjoint of the whole run (every state stored).
"""
import numpy as np

from .ark2 import tableau
from .column import implicit_solve
from .reference import GAMMA, GRAV, pressure_perturbation
from .rhs import apply_wall_bc, rhs


def dpressure(rho_p, th_p, drho_p, dth_p, rho0, theta0, P0):
    """dP' = gamma P (drho'/rho + dtheta'/theta): derivative of the equation of state."""
    P = P0 + pressure_perturbation(rho_p, th_p, rho0, theta0, P0)
    return GAMMA * P * (drho_p / (rho0 + rho_p) + dth_p / (theta0 + th_p))


class _Elem:
    """Element-local derivative operators of a box mesh (the ones ``oracle.rhs`` uses)."""

    def __init__(self, mesh):
        self.D = mesh.D
        self.sx, self.sy, self.sz = 2.0 / mesh.dx, 2.0 / mesh.dy, 2.0 / mesh.dz

    def ddx(self, a):
        return np.einsum("in,ekjn->ekji", self.D, a) * self.sx

    def ddy(self, a):
        return np.einsum("jn,ekni->ekji", self.D, a) * self.sy

    def ddz(self, a):
        return np.einsum("kn,enji->ekji", self.D, a) * self.sz

    # transposes: (ddx^T b)[..., n] = sum_i D[i, n] b[..., i]
    def ddxT(self, b):
        return np.einsum("in,ekji->ekjn", self.D, b) * self.sx

    def ddyT(self, b):
        return np.einsum("jn,ekji->ekni", self.D, b) * self.sy

    def ddzT(self, b):
        return np.einsum("kn,ekji->enji", self.D, b) * self.sz


def rhs_tlm(mesh, col, q, dq, l2g=None, mass=None):
    """R'(q) dq for states of shape (5, nnode)."""
    l2g = mesh.l2g() if l2g is None else l2g
    mass = mesh.global_mass(l2g) if mass is None else mass
    op = _Elem(mesh)
    iz = l2g % mesh.M
    rho_p, u, v, w, th_p = q[:, l2g]
    drp, du, dv, dw, dth = dq[:, l2g]
    rho0, theta0, P0 = col.rho0[iz], col.theta0[iz], col.P0[iz]
    drho0, dtheta0 = col.drho0[iz], col.dtheta0[iz]
    rho = rho0 + rho_p
    Pp = pressure_perturbation(rho_p, th_p, rho0, theta0, P0)
    dPp = dpressure(rho_p, th_p, drp, dth, rho0, theta0, P0)

    def dadv(a, da):   # d(u.grad a)
        return (du * op.ddx(a) + u * op.ddx(da) + dv * op.ddy(a) + v * op.ddy(da)
                + dw * op.ddz(a) + w * op.ddz(da))

    div_u = op.ddx(u) + op.ddy(v) + op.ddz(w)
    ddiv = op.ddx(du) + op.ddy(dv) + op.ddz(dw)
    t_rho = -(dadv(rho_p, drp) + dw * drho0 + drp * div_u + rho * ddiv)
    t_u = -(dadv(u, du) + op.ddx(dPp) / rho - op.ddx(Pp) * drp / rho ** 2)
    t_v = -(dadv(v, dv) + op.ddy(dPp) / rho - op.ddy(Pp) * drp / rho ** 2)
    t_w = -(dadv(w, dw) + op.ddz(dPp) / rho - op.ddz(Pp) * drp / rho ** 2
            + GRAV * drp / rho - GRAV * rho_p * drp / rho ** 2)
    t_th = -(dadv(th_p, dth) + dw * dtheta0)
    out = np.stack([mesh.dss(t, l2g, mass) for t in (t_rho, t_u, t_v, t_w, t_th)])
    apply_wall_bc(mesh, out)
    return out


def rhs_adjoint(mesh, col, q, lam, l2g=None, mass=None):
    """R'(q)^T lam for states of shape (5, nnode)."""
    l2g = mesh.l2g() if l2g is None else l2g
    mass = mesh.global_mass(l2g) if mass is None else mass
    op = _Elem(mesh)
    iz = l2g % mesh.M
    rho_p, u, v, w, th_p = q[:, l2g]
    rho0, theta0, P0 = col.rho0[iz], col.theta0[iz], col.P0[iz]
    drho0, dtheta0 = col.drho0[iz], col.dtheta0[iz]
    rho = rho0 + rho_p
    Pp = pressure_perturbation(rho_p, th_p, rho0, theta0, P0)

    # wall mask (a projection: its own transpose), then DSS^T: the local copy (e, l) of
    # global node g receives W_l J lam_g / M_g
    lam = apply_wall_bc(mesh, np.array(lam, dtype=np.float64, copy=True))
    Wl = np.broadcast_to(mesh.local_weights(), l2g.shape)
    a_r, a_u, a_v, a_w, a_t = lam[:, l2g] * (Wl / mass[l2g])

    # the tendencies, written as  t = -(sum_axes coef * d_axis(field)) - pointwise:
    # t_rho = -(u r_x + v r_y + w r_z + w drho0 + rho (u_x + v_y + w_z))
    # t_u   = -(u u_x + v u_y + w u_z + P'_x / rho)       (t_v alike with y)
    # t_w   = -(u w_x + v w_y + w w_z + P'_z / rho + g rho' / rho)
    # t_th  = -(u th_x + v th_y + w th_z + w dtheta0)
    # Adjoint of each derivative input d_axis(field): the sum of its coefficients times
    # the tendency adjoints.
    fx = [-u * a_r, -(rho * a_r + u * a_u), -u * a_v, -u * a_w, -u * a_t, -a_u / rho]
    fy = [-v * a_r, -v * a_u, -(rho * a_r + v * a_v), -v * a_w, -v * a_t, -a_v / rho]
    fz = [-w * a_r, -w * a_u, -w * a_v, -(rho * a_r + w * a_w), -w * a_t, -a_w / rho]
    loc = [op.ddxT(fx[k]) + op.ddyT(fy[k]) + op.ddzT(fz[k]) for k in range(6)]

    # pointwise inputs: rho' (through rho), u, v, w
    fld = (rho_p, u, v, w, th_p)
    gx = [op.ddx(f) for f in fld] + [op.ddx(Pp)]
    gy = [op.ddy(f) for f in fld] + [op.ddy(Pp)]
    gz = [op.ddz(f) for f in fld] + [op.ddz(Pp)]
    div_u = gx[1] + gy[2] + gz[3]
    loc[0] = loc[0] + (-div_u * a_r + gx[5] / rho ** 2 * a_u + gy[5] / rho ** 2 * a_v
                       + (gz[5] + GRAV * rho_p) / rho ** 2 * a_w - GRAV / rho * a_w)
    loc[1] = loc[1] - (gx[0] * a_r + gx[1] * a_u + gx[2] * a_v + gx[3] * a_w + gx[4] * a_t)
    loc[2] = loc[2] - (gy[0] * a_r + gy[1] * a_u + gy[2] * a_v + gy[3] * a_w + gy[4] * a_t)
    loc[3] = loc[3] - ((gz[0] + drho0) * a_r + gz[1] * a_u + gz[2] * a_v + gz[3] * a_w
                       + (gz[4] + dtheta0) * a_t)

    # equation of state transposed: P' depends on rho' and theta'
    P = P0 + Pp
    loc[0] = loc[0] + GAMMA * P / rho * loc[5]
    loc[4] = loc[4] + GAMMA * P / (theta0 + th_p) * loc[5]

    # gather transposed: sum the local copies into the global nodes
    out = np.zeros((5, mesh.nnode))
    for k in range(5):
        np.add.at(out[k], l2g.ravel(), loc[k].ravel())
    return out


def lu_solve_transposed_banded(LU, half_band, b):
    """Solve S^T x = b where LU holds S = L U (unit lower L below the diagonal, U on and
    above it, as returned by ``column.lu_nopivot_banded``).  ``b`` has the level as its
    last axis.  S^T = U^T L^T: forward substitution with U^T, then back substitution
    with the unit upper L^T."""
    b = np.array(b, dtype=np.float64, copy=True)
    M = LU.shape[0]
    y = np.empty_like(b)
    for i in range(M):
        lo = max(0, i - half_band)
        y[..., i] = (b[..., i] - y[..., lo:i] @ LU[lo:i, i]) / LU[i, i]
    x = np.empty_like(b)
    for i in range(M - 1, -1, -1):
        hi = min(M, i + half_band + 1)
        x[..., i] = y[..., i] - x[..., i + 1:hi] @ LU[i + 1:hi, i]
    return x


class ColumnMap:
    """Matrix of the implicit column solve of an ``ark2.HEVI`` integrator.

    ``K[(f', m'), (f, m)]``: output field f' at level m' per unit input of field f at
    level m (fields in the order rho', u, v, w, theta').
    """

    def __init__(self, hevi):
        M = hevi.mesh.M
        self.M = M
        E = np.eye(5 * M).reshape(5 * M, 5, M).transpose(1, 0, 2)   # (5, probes, M)
        X = implicit_solve(hevi.col, hevi.LU, E, hevi.lam)          # (5, probes, M)
        self.K = X.transpose(0, 2, 1).reshape(5 * M, 5 * M)

    def _cols(self, x):
        return np.asarray(x).reshape(5, -1, self.M).transpose(1, 0, 2).reshape(-1, 5 * self.M)

    def _uncols(self, y, shape):
        return y.reshape(-1, 5, self.M).transpose(1, 0, 2).reshape(shape)

    def apply(self, x):
        return self._uncols(self._cols(x) @ self.K.T, np.shape(x))

    def apply_T(self, lam):
        return self._uncols(self._cols(lam) @ self.K, np.shape(lam))


def _stage_coefs(i):
    a, at, _, _ = tableau()
    return a, at, [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]


def step_tlm(hevi, q, dq):
    """One ARK2 step and its tangent: returns (q^{n+1}, dq^{n+1})."""
    mesh, col, dt = hevi.mesh, hevi.col, hevi.dt
    _, _, b, _ = tableau()
    Q, dQ = [q], [dq]
    Rs = [hevi.R(q)]
    dRs = [rhs_tlm(mesh, col, q, dq, hevi.l2g, hevi.mass)]
    for i in (1, 2):
        a, at, c = _stage_coefs(i)
        lam = at[i, i] * dt
        qt = q + dt * sum(a[i, j] * Rs[j] for j in range(i)) + sum(c[j] * Q[j] for j in range(i))
        dqt = dq + dt * sum(a[i, j] * dRs[j] for j in range(i)) + sum(c[j] * dQ[j] for j in range(i))
        Qi = hevi.solve(qt, lam) - sum(c[j] * Q[j] for j in range(i))
        dQi = hevi.solve(dqt, lam) - sum(c[j] * dQ[j] for j in range(i))
        Q.append(Qi)
        dQ.append(dQi)
        Rs.append(hevi.R(Qi))
        dRs.append(rhs_tlm(mesh, col, Qi, dQi, hevi.l2g, hevi.mass))
    return (q + dt * sum(b[i] * Rs[i] for i in range(3)),
            dq + dt * sum(b[i] * dRs[i] for i in range(3)))


def step_stages(hevi, q):
    """The stage states q(1) = q^n, q(2), q(3) of one ARK2 step."""
    dt = hevi.dt
    Q, Rs = [q], [hevi.R(q)]
    for i in (1, 2):
        a, at, c = _stage_coefs(i)
        lam = at[i, i] * dt
        qt = q + dt * sum(a[i, j] * Rs[j] for j in range(i)) + sum(c[j] * Q[j] for j in range(i))
        Qi = hevi.solve(qt, lam) - sum(c[j] * Q[j] for j in range(i))
        Q.append(Qi)
        Rs.append(hevi.R(Qi))
    return Q


def stage_adjoint(hevi, i, lam, cmap=None):
    """Adjoint of stage i in {1, 2} (rows 2 and 3 of Table 1; q(i+1) in the paper's
    numbering) as a linear map of its inputs q^n, R_j = R(q(j)) and q(j), j < i:

        q~_e = q^n + dt sum_j a_ij R_j + sum_j c_ij q(j),  q~ = solve(q~_e),
        q(i) = q~ - sum_j c_ij q(j),  with q(0) = q^n.

    Returns (qn*, [R_j*], [q(j)*]) for j < i; the q(0)* term is already in qn*."""
    dt = hevi.dt
    cmap = ColumnMap(hevi) if cmap is None else cmap
    a, _, c = _stage_coefs(i)
    qta = cmap.apply_T(lam)
    Ra = [dt * a[i, j] * qta for j in range(i)]
    Qa = [c[j] * (qta - lam) for j in range(i)]
    return qta + Qa[0], Ra, [None] + Qa[1:]


def step_adjoint(hevi, q, lam, cmap=None):
    """Adjoint of one ARK2 step at q^n: given lam = dJ/dq^{n+1}, returns dJ/dq^n."""
    mesh, col, dt = hevi.mesh, hevi.col, hevi.dt
    cmap = ColumnMap(hevi) if cmap is None else cmap
    _, _, b, _ = tableau()
    Q = step_stages(hevi, q)
    qa = np.array(lam, dtype=np.float64, copy=True)          # q^{n+1} = q^n + ...
    Ra = [dt * b[i] * lam for i in range(3)]
    Qa = [np.zeros_like(qa) for _ in range(3)]
    for i in (2, 1):
        Qa[i] = Qa[i] + rhs_adjoint(mesh, col, Q[i], Ra[i], hevi.l2g, hevi.mass)
        qn_a, Rj_a, Qj_a = stage_adjoint(hevi, i, Qa[i], cmap)
        qa = qa + qn_a
        for j in range(i):
            Ra[j] = Ra[j] + Rj_a[j]
            if j > 0:
                Qa[j] = Qa[j] + Qj_a[j]
    return qa + rhs_adjoint(mesh, col, Q[0], Ra[0], hevi.l2g, hevi.mass)


def misfit(qT, target):
    """J = 1/2 sum_g (theta'_T[g] - target[g])^2."""
    d = qT[4] - target
    return 0.5 * float(d @ d)


def gradient(hevi, q0, target, nsteps):
    """(J, dJ/dq0) for J = misfit(hevi.step(q0, nsteps), target)."""
    states = [q0]
    for _ in range(nsteps):
        states.append(hevi.step(states[-1]))
    lam = np.zeros_like(q0)
    lam[4] = states[-1][4] - target
    cmap = ColumnMap(hevi)
    for s in range(nsteps - 1, -1, -1):
        lam = step_adjoint(hevi, states[s], lam, cmap)
    return misfit(states[-1], target), lam
