"""Legendre-Gauss-Lobatto (LGL) nodes, weights and derivative matrix.

Test infrastructure (oracle).  The paper evaluates every derivative with ``sD``, the
gradient of the nodal basis functions at the LGL points, held in shared memory
(Sec. "Volume kernels", Algorithms 1 and 2).  Its definition is the textbook one:

* nodes: -1, +1 and the N-1 roots of P_N'(x);
* weights: w_i = 2 / (N (N+1) P_N(x_i)^2);
* derivative matrix D_ij = l_j'(x_i):
  D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j,
  D_00 = -N(N+1)/4, D_NN = +N(N+1)/4, and D_ii = 0 otherwise.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre_PN(N, x):
    """P_N(x) by numpy's Legendre series evaluation (library primitive)."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    return npleg.legval(x, c)


def lgl_nodes(N):
    """LGL nodes on [-1, 1], ascending: the endpoints plus the roots of P_N'."""
    if N < 1:
        raise ValueError("N must be >= 1")
    c = np.zeros(N + 1)
    c[N] = 1.0
    dc = npleg.legder(c)
    interior = np.sort(npleg.legroots(dc).real) if N > 1 else np.zeros(0)
    # two Newton polishing steps on P_N' (library roots are accurate to ~1e-15 already)
    ddc = npleg.legder(dc)
    for _ in range(2):
        if interior.size:
            interior = interior - npleg.legval(interior, dc) / npleg.legval(interior, ddc)
    return np.concatenate([[-1.0], interior, [1.0]])


def lgl_weights(N, x):
    """Quadrature weights w_i = 2 / (N(N+1) P_N(x_i)^2)."""
    return 2.0 / (N * (N + 1) * legendre_PN(N, x) ** 2)


def lgl_derivative_matrix(N, x):
    """D[i, j] = derivative of the j-th Lagrange basis function at node i."""
    PN = legendre_PN(N, x)
    Nq = N + 1
    D = np.zeros((Nq, Nq))
    for i in range(Nq):
        for j in range(Nq):
            if i != j:
                D[i, j] = PN[i] / (PN[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def lgl(N):
    """Return (nodes, weights, D) for polynomial order N."""
    x = lgl_nodes(N)
    return x, lgl_weights(N, x), lgl_derivative_matrix(N, x)
