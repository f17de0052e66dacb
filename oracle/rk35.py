"""Explicit five-stage, third-order strong-stability-preserving Runge-Kutta comparator.

Test infrastructure (oracle).

The paper compares IMEX against the SSP third-order five-stage RK35 of Spiteri & Ruuth
(Sec. "Performance of IMEX on manycore processors") but prints no coefficients, and that
publication is not at hand.  Reading: a five-stage third-order SSP scheme in the
two-register Shu-Osher form

    u_1 = u_0 + beta_1 dt F(u_0)
    u_i = alpha_i u_0 + (1 - alpha_i) u_{i-1} + beta_i dt F(u_{i-1}),   i = 2..5
    u^{n+1} = u_5

with alpha_2 = alpha_3 = alpha_5 = 0, beta_1 = beta_5 = 0.46 (SSP coefficient
1/0.46 = 2.17) and (beta_2, beta_3, beta_4, alpha_4) the real root of the four
third-order conditions with beta_2 > beta_3.  The values below were computed to 25
digits; tests/test_oracle_ark.py re-solves the conditions and checks the order.

PARITY UNPINNED in the sense of the paper: which five-stage scheme the paper ran cannot
be checked; this comparator is pinned only against its own order conditions.
"""
import numpy as np

from .rhs import rhs

BETA = np.array([0.46,
                 0.2805744403033042654640453,
                 0.22110850739434604175949,
                 0.1326553823821179192508848,
                 0.46])
ALPHA = np.array([0.0, 0.0, 0.0, 0.5764252463942515726402586, 0.0])


def butcher():
    """Butcher (A, b, c) of the scheme above (stage j is u_{j-1})."""
    s = 5
    rows = []
    prev = np.zeros(s)
    for i in range(s):
        cur = (1.0 - ALPHA[i]) * prev
        cur[i] += BETA[i]
        rows.append(cur)
        prev = cur
    A = np.zeros((s, s))
    for i in range(1, s):
        A[i] = rows[i - 1]
    b = rows[-1]
    return A, b, A.sum(axis=1)


def rk35_step(u0, dt, F):
    u = u0
    for i in range(5):
        u = ALPHA[i] * u0 + (1.0 - ALPHA[i]) * u + BETA[i] * dt * F(u)
    return u


class Explicit:
    """RK35 on a box mesh (oracle)."""

    def __init__(self, mesh, col):
        self.mesh, self.col = mesh, col
        self.l2g = mesh.l2g()
        self.mass = mesh.global_mass(self.l2g)

    def R(self, q):
        return rhs(self.mesh, self.col, q, self.l2g, self.mass)

    def step(self, q, dt, nsteps=1):
        for _ in range(nsteps):
            q = rk35_step(q, dt, self.R)
        return q
