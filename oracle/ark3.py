"""Third-order additive Runge-Kutta tableau for the HEVI step (ARK3).

Test infrastructure (oracle).  The paper reports ARK3, ARK4 and ARK5 runs next to ARK2
(Sec. "Performance of IMEX on manycore processors", acoustic wave problem) but prints no
tableau for them.  Reading: ARK3 is the ARK3(2)4L[2]SA scheme of Kennedy and Carpenter
(2003), the third-order member of the family the paper's ARK2 comes from.  It is an
explicit / ESDIRK pair with four stages, one implicit diagonal gamma (a~_11 = 0, a~_ii =
gamma otherwise), equal abscissae c = c~, and b = b~ = the last implicit row (stiffly
accurate).  It therefore fits the stage form of ``ark2.ark_step`` and one stored column
factorisation at lam = gamma dt.  The coefficients are the published rationals.  The pins
in tests/test_oracle_ark.py check the third-order conditions of both tableaux and of
their coupling in exact rational arithmetic, and third-order convergence on a stiff
linear split system.

PARITY UNPINNED in the sense of the paper: the paper does not print the tableau it ran, so
which scheme it used cannot be checked.  The pins fix this tableau only as an ARK pair of
its order (exact order conditions) and by its convergence rate.
"""
from fractions import Fraction as F

import numpy as np

GAMMA = F(1767732205903, 4055673282236)

A_IMPLICIT = (
    (0, 0, 0, 0),
    (GAMMA, GAMMA, 0, 0),
    (F(2746238789719, 10658868560708), F(-640167445237, 6845629431997), GAMMA, 0),
    (F(1471266399579, 7840856788654), F(-4482444167858, 7529755066697),
     F(11266239266428, 11593286722821), GAMMA),
)

A_EXPLICIT = (
    (0, 0, 0, 0),
    (F(1767732205903, 2027836641118), 0, 0, 0),
    (F(5535828885825, 10492691773637), F(788022342437, 10882634858940), 0, 0),
    (F(6485989280629, 16251701735622), F(-4246266847089, 9704473918619),
     F(10755448449292, 10357097424841), 0),
)


def rational_tableau():
    """(a, at, b, c) as tuples of Fractions (exact)."""
    a = A_EXPLICIT
    at = A_IMPLICIT
    b = at[3]
    c = tuple(sum(F(x) for x in row) for row in a)
    return a, at, b, c


def tableau():
    """(a, at, b, c) as float arrays, the layout of ``ark2.tableau``."""
    a, at, b, c = rational_tableau()
    f = lambda rows: np.array([[float(x) for x in r] for r in rows])
    return f(a), f(at), np.array([float(x) for x in b]), np.array([float(x) for x in c])
