"""Second-order ARK (IMEX) time step in the SDIRK predictor-corrector form.

Test infrastructure (oracle).

Tableau: Table 1 (double Butcher tableau of the second-order ARK scheme of Giraldo et
al. 2013).  The extracted table is garbled: its b row reads (-1/(2 sqrt2), -1/(2 sqrt2),
1 - 1/(2 sqrt2)), which sums to -0.41 and is not even first order, and the implicit row 3
carries the same stray minus signs.  Reading: the paper assumes b = b~ (Sec. "Linear
multi-stage methods") and the scheme is stiffly accurate, so b = b~ = the last implicit
row = (1/(2 sqrt2), 1/(2 sqrt2), 1 - 1/sqrt2).  The pins in tests/test_oracle_ark.py
show this reading satisfies the order conditions and the printed signs do not.

Stage algorithm (Sec. "Linear multi-stage methods"), with R = N + L and L linear:

    q(1) = q^n                                               (a~_11 = 0)
    for i = 2..s:
        q(i)_e  = q^n + dt sum_{j<i} a_ij R(q(j))
        c_ij    = (a~_ij - a_ij) / a~_ii
        q~_e    = q(i)_e + sum_{j<i} c_ij q(j)
        solve     q~ = q~_e + lam L(q~),      lam = a~_ii dt
        q(i)    = q~ - sum_{j<i} c_ij q(j)
    q^{n+1} = q^n + dt sum_i b_i R(q(i))                     (b = b~)

For the 1D-IMEX (HEVI) method L is the vertical operator L_V (Eq. sieqn1d).
"""
import math

import numpy as np

from .column import (implicit_solve, implicit_solve_standard, lu_nopivot_banded,
                     standard_half_band, standard_interleaved)
from .rhs import rhs

SQ2 = math.sqrt(2.0)


def tableau():
    """(a, at, b, c) of the ARK2 scheme; a explicit, at implicit (3x3 each)."""
    a = np.zeros((3, 3))
    a[1, 0] = 2.0 - SQ2
    a[2, 1] = (3.0 + 2.0 * SQ2) / 6.0
    a[2, 0] = 1.0 - a[2, 1]
    at = np.zeros((3, 3))
    at[1, 0] = at[1, 1] = 1.0 - 1.0 / SQ2
    at[2, 0] = at[2, 1] = 1.0 / (2.0 * SQ2)
    at[2, 2] = 1.0 - 1.0 / SQ2
    b = at[2].copy()
    c = a.sum(axis=1)
    return a, at, b, c


def printed_b():
    """The b row exactly as extracted from Table 1 (used only to show it is wrong)."""
    return np.array([-1.0 / (2.0 * SQ2), -1.0 / (2.0 * SQ2), 1.0 - 1.0 / (2.0 * SQ2)])


def ark_step(q, dt, R, solve, tab=None):
    """One ARK step for dq/dt = R(q) = N(q) + L(q) (ARK2 unless tab = (a, at, b, c) of
    another scheme with a~_11 = 0, one implicit diagonal and b = b~, such as ARK3 - ARK5).

    R(q) is the full right-hand side; solve(rhs, lam) returns x with x = rhs + lam L(x).
    """
    a, at, b, _ = tableau() if tab is None else tab
    s = len(b)
    Q = [q]
    Rs = [R(q)]
    for i in range(1, s):
        lam = at[i, i] * dt
        cij = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        q_e = q + dt * sum(a[i, j] * Rs[j] for j in range(i))
        qtt_e = q_e + sum(cij[j] * Q[j] for j in range(i))
        qtt = solve(qtt_e, lam)
        Qi = qtt - sum(cij[j] * Q[j] for j in range(i))
        Q.append(Qi)
        Rs.append(R(Qi))
    return q + dt * sum(b[i] * Rs[i] for i in range(s))


SCHEMES = ("ark2", "ark3", "ark4", "ark5")


def scheme_tableau(scheme):
    """(a, at, b, c) of "ark2" (Table 1), "ark3", "ark4" or "ark5" (``oracle.ark3``,
    ``oracle.ark4``, ``oracle.ark5``)."""
    if scheme not in SCHEMES:
        raise ValueError("scheme must be one of %s" % (SCHEMES,))
    if scheme == "ark2":
        return tableau()
    import importlib
    return importlib.import_module("." + scheme, __package__).tableau()


class HEVI:
    """The 1D-IMEX (HEVI) integrator on a box mesh (oracle).  form: "schur" (the paper's
    method) or "standard" (the non-Schur column system, same step otherwise); scheme:
    one of SCHEMES (``scheme_tableau``)."""

    def __init__(self, mesh, col, dt, form="schur", scheme="ark2"):
        if form not in ("schur", "standard"):
            raise ValueError("form must be 'schur' or 'standard'")
        self.tab = scheme_tableau(scheme)
        self.mesh, self.col, self.dt, self.form, self.scheme = mesh, col, dt, form, scheme
        at = self.tab[1]
        self.lam = at[1, 1] * dt                     # one implicit diagonal for every stage
        if form == "schur":
            self.LU = lu_nopivot_banded(col.jacobian_by_probing(self.lam), col.half_band)
        else:
            self.LU = lu_nopivot_banded(standard_interleaved(col, self.lam),
                                        standard_half_band(mesh))
        self.l2g = mesh.l2g()
        self.mass = mesh.global_mass(self.l2g)

    def R(self, q):
        return rhs(self.mesh, self.col, q, self.l2g, self.mass)

    def solve(self, q_e, lam):
        assert abs(lam - self.lam) <= 1e-15 * abs(self.lam)
        shape = q_e.shape
        qc = q_e.reshape(5, self.mesh.ncol, self.mesh.M)
        if self.form == "schur":
            return implicit_solve(self.col, self.LU, qc, lam).reshape(shape)
        return implicit_solve_standard(self.col, self.LU, qc, lam).reshape(shape)

    def step(self, q, nsteps=1):
        for _ in range(nsteps):
            q = ark_step(q, self.dt, self.R, self.solve, self.tab)
        return q
