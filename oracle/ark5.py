"""Fifth-order additive Runge-Kutta tableau for the HEVI step (ARK5).

Test infrastructure (oracle).  The paper runs ARK5 next to ARK2 (Sec. "Performance of IMEX
on manycore processors", acoustic wave problem) without printing its tableau.  Reading:
ARK5 is the ARK5(4)8L[2]SA scheme of Kennedy and Carpenter (2003): an explicit / ESDIRK
pair of eight stages with a~_11 = 0, one implicit diagonal gamma = 41/200, equal abscissae
c = c~ and b = b~ = the last implicit row, so it has the stage form of ``ark2.ark_step``
and one column factorisation at lam = gamma dt.

The coefficients are the published rationals, except the explicit entries a_86 and a_87.
Those two are the solution of the 143 bicoloured-tree conditions of orders 1 to 5 with
every other entry held at its published value (``derive_ark5_row8``): an overdetermined
system that they satisfy to 2e-26, the accuracy of the published rationals, so they are
the published scheme's entries to that accuracy, rounded to rationals with denominators
below 2e13.  tests/test_oracle_ark.py checks every condition up to order 5 in exact
arithmetic and the rate of convergence.

PARITY UNPINNED in the sense of the paper: the paper does not print the tableau it ran, so
which scheme it used cannot be checked.  The pins fix this tableau only as an ARK pair of
its order (exact order conditions) and by its convergence rate.
"""
from fractions import Fraction as F

import numpy as np

GAMMA = F(41, 200)

A_IMPLICIT = (
    (0, 0, 0, 0, 0, 0, 0, 0),
    (GAMMA, GAMMA, 0, 0, 0, 0, 0, 0),
    (F(41, 400), F(-567603406766, 11931857230679), GAMMA, 0, 0, 0, 0, 0),
    (F(683785636431, 9252920307686), 0, F(-110385047103, 1367015193373), GAMMA, 0, 0, 0, 0),
    (F(3016520224154, 10081342136671), 0, F(30586259806659, 12414158314087),
     F(-22760509404356, 11113319521817), GAMMA, 0, 0, 0),
    (F(218866479029, 1489978393911), 0, F(638256894668, 5436446318841),
     F(-1179710474555, 5321154724896), F(-60928119172, 8023461067671), GAMMA, 0, 0),
    (F(1020004230633, 5715676835656), 0, F(25762820946817, 25263940353407),
     F(-2161375909145, 9755907335909), F(-211217309593, 5846859502534),
     F(-4269925059573, 7827059040749), GAMMA, 0),
    (F(-872700587467, 9133579230613), 0, 0, F(22348218063261, 9555858737531),
     F(-1143369518992, 8141816002931), F(-39379526789629, 19018526304540),
     F(32727382324388, 42900044865799), GAMMA),
)

# explicit a_86, a_87 (see the module docstring)
A86 = F(-56156175540813, 7787401243552)
A87 = F(21501425855156, 14444669418411)

A_EXPLICIT_ROWS_1_7 = (
    (0, 0, 0, 0, 0, 0, 0, 0),
    (F(41, 100), 0, 0, 0, 0, 0, 0, 0),
    (F(367902744464, 2072280473677), F(677623207551, 8224143866563), 0, 0, 0, 0, 0, 0),
    (F(1268023523408, 10340822734521), 0, F(1029933939417, 13636558850479), 0, 0, 0, 0, 0),
    (F(14463281900351, 6315353703477), 0, F(66114435211212, 5879490589093),
     F(-54053170152839, 4284798021562), 0, 0, 0, 0),
    (F(14090043504691, 34967701212078), 0, F(15191511035443, 11219624916014),
     F(-18461159152457, 12425892160975), F(-281667163811, 9011619295870), 0, 0, 0),
    (F(19230459214898, 13134317526959), 0, F(21275331358303, 2942455364971),
     F(-38145345988419, 4862620318723), F(-1, 8), F(-1, 8), 0, 0),
)


def explicit_row8(a86, a87):
    """Explicit row 8 with the published a_81 .. a_85 and the given a_86, a_87."""
    return (F(-19977161125411, 11928030595625), 0, F(-40795976796054, 6384907823539),
            F(177454434618887, 12078138498510), F(782672205425, 8267701900261), a86, a87, 0)


def rational_tableau():
    """(a, at, b, c) as tuples of Fractions (exact)."""
    a = A_EXPLICIT_ROWS_1_7 + (explicit_row8(A86, A87),)
    at = A_IMPLICIT
    return a, at, at[-1], tuple(sum(F(x) for x in row) for row in a)


def tableau():
    """(a, at, b, c) as float arrays, the layout of ``ark2.tableau``."""
    a, at, b, c = rational_tableau()
    f = lambda rows: np.array([[float(x) for x in r] for r in rows])
    return f(a), f(at), np.array([float(x) for x in b]), np.array([float(x) for x in c])
