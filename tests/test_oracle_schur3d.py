"""Pins of the 3D-IMEX Schur-form oracle (not GPU).

* The Schur elimination is exact at the discrete level: the 3D Schur solve equals a dense
  solve of the standard system (I - lam L) q = q_e, with L built by probing the (separately
  pinned) tangent-linear RHS at rest, R'(0) = L.
* A horizontally uniform pressure with no horizontal velocity reduces the 3D operator to the
  1D column operator.
* BiCGstab with the polynomial preconditioner converges to the dense solution.
* The Chebyshev preconditioner polynomial has the closed-form residual and its maximum.
* The PBNO recursion applied to a diagonal operator is the polynomial at its entries.
* 3D-IMEX converges to explicit RK at small Courant numbers and stays bounded at
  C_V = C_H = 15, where the horizontally explicit 1D-IMEX does not.
"""
import numpy as np
import pytest

from helpers import Case
from oracle import schur3d as s3
from oracle.tangent import rhs_tlm


def _lam(case, C):
    return (1.0 - 1.0 / np.sqrt(2.0)) * case.dt_for(C)


def _dense(apply, n):
    A = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = apply(e)
    return A


@pytest.mark.parametrize("C", [1, 15, 150])
def test_schur_solve_equals_dense_standard_solve(C):
    case = Case(2, 1, 2, 2, 3e3, 2e3, 4e3, n_bv=0.012)
    m = case.mesh
    lam = _lam(case, C)
    n = 5 * m.nnode
    zero = np.zeros((5, m.nnode))
    J = _dense(lambda x: rhs_tlm(m, case.col, zero, x.reshape(5, -1)).ravel(), n)
    K = np.eye(n) - lam * J
    rng = np.random.default_rng(C)
    q_e = rng.standard_normal((5, m.nnode))
    q_e[0] *= 1e-3
    op = s3.Schur3D(m, case.col)
    mx, my, mz = op.walls
    q_e[1, mx] = 0.0
    q_e[2, my] = 0.0
    q_e[3, mz] = 0.0
    ref = np.linalg.solve(K, q_e.ravel()).reshape(5, -1)
    b, ua = op.rhs(q_e, lam)
    S = _dense(lambda x: op.apply(x, lam), m.nnode)
    P = np.linalg.solve(S, b)
    got = op.extract(P, ua, q_e[4], lam)
    for f in range(5):
        assert np.abs(got[f] - ref[f]).max() <= 1e-10 * C * np.abs(ref[f]).max()


def test_horizontally_uniform_pressure_gives_the_column_operator():
    case = Case(2, 2, 3, 3, 6e3, 6e3, 9e3, n_bv=0.01)
    m, col = case.mesh, case.col
    lam = _lam(case, 15)
    Pcol = np.random.default_rng(3).standard_normal(m.M)
    P = np.tile(Pcol, m.ncol)
    got = s3.Schur3D(m, col).apply(P, lam).reshape(m.ncol, m.M)
    ref = col.schur_apply(Pcol, lam)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_bicgstab_pbno_converges_to_the_dense_solution():
    case = Case(3, 2, 2, 3, 6e3, 4e3, 6e3, n_bv=0.01)
    m = case.mesh
    lam = _lam(case, 15)
    op = s3.Schur3D(m, case.col)
    apply = lambda x: op.apply(x, lam)
    lmax = 1.05 * s3.power_lmax(apply, m.nnode)
    c, lb = s3.chebyshev_pbno(2, 1.0, lmax)
    b = np.random.default_rng(1).standard_normal(m.nnode)
    x, it = s3.bicgstab_pbno(apply, b, c, lb, tol=1e-13)
    ref = np.linalg.solve(_dense(apply, m.nnode), b)
    assert it < 200
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("P", [1, 2, 4, 7])
@pytest.mark.parametrize("lmax", [3.0, 80.0])
def test_chebyshev_pbno_residual_polynomial(P, lmax):
    c, lb = s3.chebyshev_pbno(P, 1.0, lmax)
    assert lb == pytest.approx(2.0 / (1.0 + lmax), rel=1e-15)
    delta = (lmax - 1.0) / (lmax + 1.0)
    y = np.linspace(1.0 - delta, 1.0 + delta, 2001)
    q = sum(c[i] * y ** (P - i) for i in range(P + 1))
    res = 1.0 - y * q
    TP = np.cos((P + 1) * np.arccos(np.clip((1.0 - y) / delta, -1, 1)))
    T1 = np.cosh((P + 1) * np.arccosh(1.0 / delta))
    np.testing.assert_allclose(res, TP / T1, atol=1e-12)
    assert np.abs(res).max() == pytest.approx(1.0 / T1, rel=1e-9)


def test_pbno_recursion_on_a_diagonal_operator():
    d = np.linspace(1.0, 40.0, 17)
    c, lb = s3.chebyshev_pbno(3, 1.0, 40.0)
    r = np.random.default_rng(2).standard_normal(d.size)
    got = s3.pbno_apply(lambda v: d * v, r, c, lb)
    y = lb * d
    ref = lb * sum(c[i] * y ** (3 - i) for i in range(4)) * r
    np.testing.assert_allclose(got, ref, rtol=1e-13)


def test_hevi3d_converges_to_rk35_at_small_courant():
    from oracle import rk35
    case = Case(2, 2, 2, 3, 4e3, 4e3, 4e3)
    m, col = case.mesh, case.col
    q0 = case.state(21, kind="balanced")
    dt1 = case.dt_for(1.0)
    T = 8 * dt1
    ref = rk35.Explicit(m, col).step(q0, T / 64, 64)
    diffs = []
    for n in (16, 32):
        q = s3.HEVI3D(m, col, T / n, tol=1e-13).step(q0, n)
        diffs.append(np.linalg.norm(q[3] - ref[3]) / np.linalg.norm(ref[3]))
    assert diffs[1] < diffs[0] / 3.0 and diffs[1] < 1e-2, diffs


def test_hevi3d_bounded_where_1d_imex_is_not():
    """C_V = C_H = 15 on a cube of elements: the horizontally explicit 1D-IMEX blows up,
    3D-IMEX (acoustics implicit in every direction) stays bounded.  The warm perturbation
    (0.5 K) accelerates upward at g theta'/theta0, about 0.6 m/s per 36 s step, so after six
    steps w is a few m/s while theta' stays at its initial size."""
    from oracle import ark2
    case = Case(3, 3, 3, 3, 9e3, 9e3, 9e3)
    m, col = case.mesh, case.col
    q0 = case.state(22, kind="balanced")
    dt = case.dt_for(15.0)
    q3 = s3.HEVI3D(m, col, dt, tol=1e-12).step(q0, 6)
    with np.errstate(all="ignore"):
        q1 = ark2.HEVI(m, col, dt).step(q0, 6)
    assert np.isfinite(q3).all() and np.abs(q3[3]).max() < 5.0 and np.abs(q3[4]).max() < 1.0
    assert not (np.isfinite(q1).all() and np.abs(q1[3]).max() < 5.0)


def test_column_preconditioner_gives_the_same_solution():
    """The 1D column Schur LU as a left preconditioner (the vertical part of S solved
    exactly) converges to the same 3D steps as the polynomial preconditioner.  (Which needs
    less work depends on C_H / C_V: here, a cube of elements at C_H = C_V = 15, the column
    preconditioner needs more iterations, each of two operator applications and two column
    solves, against 2 (1 + P) operator applications.)"""
    case = Case(3, 3, 3, 3, 9e3, 9e3, 9e3, n_bv=0.01)
    m, col = case.mesh, case.col
    dt = case.dt_for(15.0)
    q0 = case.state(23, kind="balanced")
    a = s3.HEVI3D(m, col, dt, tol=1e-13)
    b = s3.HEVI3D(m, col, dt, tol=1e-13, precond="column")
    qa, qb = a.step(q0, 2), b.step(q0, 2)
    for f in range(5):
        assert np.abs(qa[f] - qb[f]).max() <= 1e-9 * np.abs(qa[f]).max()
    assert max(b.iters) < 500 and max(a.iters) < 500
