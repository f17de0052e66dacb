"""Order conditions of additive Runge-Kutta pairs, in exact rational arithmetic.

Test infrastructure (oracle).  An ARK pair (a, a~) with b = b~ integrates
dq/dt = N(q) + L(q) to order p when, for every rooted tree t of at most p vertices whose
non-root vertices each carry one of the two colours (0: explicit a, 1: implicit a~), the
elementary weight equals 1 / gamma(t) (Kennedy and Carpenter 2003, Sec. 2; the
bicoloured-tree form of the Butcher theory).  The elementary weight is
Phi(t) = sum_i b_i Phi_i(t), with Phi_i(t) the product over the root's children (colour
k, subtree u) of sum_j A^k_ij Phi_j(u); gamma(t) is the tree's order times the gammas of
its subtrees.  The numbers of such trees of order 1..6 are 1, 2, 7, 26, 107, 458.
"""
from fractions import Fraction


def trees(n):
    """The bicoloured rooted trees of order n (non-root vertices coloured 0 or 1), each a
    sorted tuple of (colour, subtree) children."""
    return _trees(n, {})


def _trees(n, memo):
    if n in memo:
        return memo[n]
    if n == 1:
        out = {()}
    else:
        out = set()

        def children(rem, lo):
            # multisets of (colour, subtree) with total order rem, in non-decreasing order
            if rem == 0:
                yield ()
                return
            for k in range(1, rem + 1):
                for sub in sorted(_trees(k, memo)):
                    for colour in (0, 1):
                        ch = (colour, sub)
                        if lo is not None and ch < lo:
                            continue
                        for rest in children(rem - k, ch):
                            yield (ch,) + rest

        for ch in children(n - 1, None):
            out.add(tuple(sorted(ch)))
    memo[n] = out
    return out


def order_of(t):
    return 1 + sum(order_of(u) for _, u in t)


def gamma(t):
    g = order_of(t)
    for _, u in t:
        g *= gamma(u)
    return g


def _phi(t, A, s):
    v = [Fraction(1)] * s
    for colour, u in t:
        pu = _phi(u, A, s)
        M = A[colour]
        v = [v[i] * sum(Fraction(M[i][j]) * pu[j] for j in range(s)) for i in range(s)]
    return v


def residuals(a, at, b, p):
    """{order: max over the trees of that order of |Phi(t) - 1/gamma(t)|} (Fractions), for
    the pair (a explicit, at implicit) with weights b, orders 1..p."""
    s = len(b)
    out = {}
    for n in range(1, p + 1):
        worst = Fraction(0)
        for t in trees(n):
            ph = _phi(t, (a, at), s)
            val = sum(Fraction(b[i]) * ph[i] for i in range(s))
            worst = max(worst, abs(val - Fraction(1, gamma(t))))
        out[n] = worst
    return out
