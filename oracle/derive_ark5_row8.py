"""Derives the explicit entries a_86, a_87 of ARK5(4)8L[2]SA from its order conditions.

Test infrastructure (oracle).  With every other entry of the pair at its published value,
a_86 and a_87 are the least-squares solution of the 143 bicoloured-tree conditions of
orders 1 to 5 (``ark_order``), found by Gauss-Newton in 60-digit arithmetic and rounded
to rationals with denominators below 2e13.  Run as ``python -m oracle.derive_ark5_row8``:
it prints the two rationals stored in ``ark5`` and the largest residual per order.
"""
from fractions import Fraction

import mpmath as mp

from . import ark5
from .ark_order import gamma, residuals, trees


def _mpf(x):
    x = Fraction(x)
    return mp.mpf(x.numerator) / x.denominator


def solve(x0=(-7.2, 1.5), iters=60):
    """Gauss-Newton from x0; returns ((a86, a87) as mpf, largest residual)."""
    mp.mp.dps = 60
    at = [[_mpf(v) for v in row] for row in ark5.A_IMPLICIT]
    b = at[-1]
    rows = [[_mpf(v) for v in row] for row in ark5.A_EXPLICIT_ROWS_1_7]
    ts = [t for n in range(1, 6) for t in trees(n)]
    s = 8

    def phi(t, A):
        v = [mp.mpf(1)] * s
        for colour, u in t:
            pu = phi(u, A)
            M = A[colour]
            v = [v[i] * mp.fsum(M[i][j] * pu[j] for j in range(s)) for i in range(s)]
        return v

    def resid(x):
        a = rows + [[_mpf(v) for v in ark5.explicit_row8(0, 0)]]
        a[7][5], a[7][6] = x
        return [mp.fsum(b[i] * p for i, p in enumerate(phi(t, (a, at)))) - mp.mpf(1) / gamma(t)
                for t in ts]

    x = [mp.mpf(v) for v in x0]
    h = mp.mpf(10) ** -30
    for _ in range(iters):
        r = resid(x)
        J = mp.matrix(len(r), 2)
        for k in range(2):
            xp = list(x)
            xp[k] += h
            rp = resid(xp)
            for i in range(len(r)):
                J[i, k] = (rp[i] - r[i]) / h
        dx = mp.lu_solve(J.T * J, -(J.T * mp.matrix(r)))
        x = [x[0] + dx[0], x[1] + dx[1]]
        if max(abs(dx[0]), abs(dx[1])) < mp.mpf(10) ** -40:
            break
    return x, max(abs(v) for v in resid(x))


def rationals(x):
    return tuple(Fraction(mp.nstr(v, 55)).limit_denominator(2 * 10 ** 13) for v in x)


if __name__ == "__main__":
    x, r = solve()
    a86, a87 = rationals(x)
    print("a_86 =", a86, " a_87 =", a87, " (least-squares residual %.2e)" % float(r))
    a = ark5.A_EXPLICIT_ROWS_1_7 + (ark5.explicit_row8(a86, a87),)
    res = residuals(a, ark5.A_IMPLICIT, ark5.A_IMPLICIT[-1], 5)
    print({k: "%.1e" % float(v) for k, v in res.items()})
