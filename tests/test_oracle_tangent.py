"""Pins of the oracle's tangent-linear and adjoint models (not GPU).

The TLM is pinned to centred finite differences of the (separately pinned) forward
oracle, with a Richardson ratio that only an exact derivative reaches; at rest it is
pinned to the column operator L_V.  The adjoints are pinned by dot-product identities
against the TLM and, on a tiny mesh, by the explicit transposed Jacobian.  The
transposed column solve is pinned to a dense library solve of S^T.
"""
import numpy as np
import pytest

from helpers import Case
from oracle import tangent as tg
from oracle.ark2 import HEVI
from oracle.column import lu_nopivot_banded
from oracle.reference import pressure_perturbation
from oracle.rhs import rhs


def _case(nex=3, nez=3, N=4, L=(30e3, 30e3, 10e3), n_bv=0.0):
    return Case(nex, nex, nez, N, *L, n_bv=n_bv)


def _pair(c, s1=1, s2=2):
    return c.state(s1, vel=5.0), c.state(s2, vel=5.0)


def _fd_errors(f, tlm, q, dq, hs):
    """Relative error of centred differences of f against tlm for each step in hs."""
    errs = []
    for h in hs:
        fd = (f(q + h * dq) - f(q - h * dq)) / (2.0 * h)
        errs.append(np.linalg.norm(fd - tlm) / np.linalg.norm(tlm))
    return np.array(errs)


def test_dpressure_is_the_derivative_of_the_eos():
    c = _case()
    col = c.col
    rng = np.random.default_rng(3)
    rp = 1e-2 * rng.standard_normal(c.mesh.M) * col.rho0
    tp = 2.0 * rng.standard_normal(c.mesh.M)
    dr = 1e-2 * rng.standard_normal(c.mesh.M) * col.rho0
    dtt = 2.0 * rng.standard_normal(c.mesh.M)
    d = tg.dpressure(rp, tp, dr, dtt, col.rho0, col.theta0, col.P0)

    def P(s):
        return pressure_perturbation(rp + s * dr, tp + s * dtt, col.rho0, col.theta0, col.P0)

    h = 1e-4
    fd = (P(h) - P(-h)) / (2 * h)
    np.testing.assert_allclose(fd, d, rtol=1e-7)


def test_rhs_tlm_matches_centred_differences_to_second_order():
    c = _case()
    q, dq = _pair(c)
    t = tg.rhs_tlm(c.mesh, c.col, q, dq)
    e = _fd_errors(lambda x: rhs(c.mesh, c.col, x), t, q, dq, [0.2, 0.1])
    assert e[1] < 1e-4
    assert 3.5 < e[0] / e[1] < 4.5          # O(h^2): the TLM is the exact derivative


def test_rhs_tlm_at_rest_is_the_column_operator():
    """Linearised about rest, a horizontally uniform perturbation with u = v = 0 feels
    only the vertical linear operator L_V (Sec. "Equation Set2NC", operator L)."""
    c = _case(n_bv=0.01)
    m, col = c.mesh, c.col
    rng = np.random.default_rng(5)
    rho = 1e-3 * col.rho0 * rng.standard_normal(m.M)
    w = rng.standard_normal(m.M)
    w[[0, -1]] = 0.0
    th = rng.standard_normal(m.M)
    dq = np.zeros((5, m.ncol, m.M))
    dq[0], dq[3], dq[4] = rho, w, th
    t = tg.rhs_tlm(m, col, np.zeros((5, m.nnode)), dq.reshape(5, -1)).reshape(5, m.ncol, m.M)
    Lr, Lw, Lt = col.L_V(rho, w, th)
    for f, L in ((0, Lr), (3, Lw), (4, Lt)):
        np.testing.assert_allclose(t[f], np.broadcast_to(L, (m.ncol, m.M)), rtol=1e-10,
                                   atol=1e-12 * np.abs(L).max())
    assert np.abs(t[1:3]).max() <= 1e-12 * np.abs(t).max()


def test_rhs_adjoint_dot_product():
    c = _case()
    q, dq = _pair(c)
    lam = c.state(9, vel=3.0)
    lhs = float(np.sum(lam * tg.rhs_tlm(c.mesh, c.col, q, dq)))
    rhs_ = float(np.sum(tg.rhs_adjoint(c.mesh, c.col, q, lam) * dq))
    assert abs(lhs - rhs_) <= 1e-13 * abs(lhs)


def test_rhs_adjoint_is_the_transposed_jacobian_on_a_tiny_mesh():
    c = Case(1, 2, 1, 2, 5e3, 8e3, 4e3)
    m = c.mesh
    q = c.state(4, vel=5.0)
    n = 5 * m.nnode
    J = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        J[:, k] = tg.rhs_tlm(m, c.col, q, e.reshape(5, -1)).ravel()
    JT = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        JT[:, k] = tg.rhs_adjoint(m, c.col, q, e.reshape(5, -1)).ravel()
    np.testing.assert_allclose(JT, J.T, rtol=1e-12, atol=1e-14 * np.abs(J).max())


@pytest.mark.parametrize("N,nez", [(2, 3), (4, 3), (5, 2)])
def test_transposed_lu_solve_matches_a_dense_solve(N, nez):
    c = Case(1, 1, nez, N, 10e3, 10e3, 10e3, n_bv=0.012)
    lam = 0.29 * c.dt_for(15.0)
    S = c.col.jacobian_by_probing(lam)
    LU = lu_nopivot_banded(S, c.col.half_band)
    b = np.random.default_rng(N).standard_normal((7, c.mesh.M))
    x = tg.lu_solve_transposed_banded(LU, c.col.half_band, b)
    ref = np.linalg.solve(S.T, b.T).T
    np.testing.assert_allclose(x, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def _hevi(c, C=15.0):
    return HEVI(c.mesh, c.col, c.dt_for(C))


def test_column_map_reproduces_the_solve_and_its_transpose():
    c = _case(n_bv=0.01)
    h = _hevi(c)
    cm = tg.ColumnMap(h)
    x = c.state(2, vel=4.0)
    np.testing.assert_allclose(cm.apply(x), h.solve(x, h.lam), rtol=1e-12,
                               atol=1e-13 * np.abs(x).max())
    y = c.state(3, vel=2.0)
    a = float(np.sum(y * h.solve(x, h.lam)))
    b = float(np.sum(cm.apply_T(y) * x))
    assert abs(a - b) <= 1e-13 * abs(a)


def test_step_tlm_matches_centred_differences_to_second_order():
    c = _case(n_bv=0.01)
    h = _hevi(c)
    q, dq = _pair(c, 5, 6)
    _, t = tg.step_tlm(h, q, dq)
    e = _fd_errors(lambda x: h.step(x), t, q, dq, [0.2, 0.1])
    assert e[1] < 1e-4
    assert 3.5 < e[0] / e[1] < 4.5


def test_step_adjoint_dot_product():
    c = _case(n_bv=0.01)
    h = _hevi(c)
    q, dq = _pair(c, 7, 8)
    lam = c.state(11, vel=2.0)
    _, t = tg.step_tlm(h, q, dq)
    a = float(np.sum(lam * t))
    b = float(np.sum(tg.step_adjoint(h, q, lam) * dq))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_gradient_matches_centred_differences_of_the_misfit():
    c = Case(2, 2, 2, 3, 300e3, 300e3, 8e3, n_bv=0.01)   # horizontal Courant number 0.4
    h = _hevi(c)
    q0 = c.state(1, vel=3.0)
    target = c.state(2)[4]
    J, g = tg.gradient(h, q0, target, 3)
    assert J == pytest.approx(tg.misfit(h.step(q0, 3), target), rel=1e-14)
    for s in (3, 4):
        d = c.state(s, vel=2.0)
        eps = 1e-3
        fd = (tg.misfit(h.step(q0 + eps * d, 3), target)
              - tg.misfit(h.step(q0 - eps * d, 3), target)) / (2 * eps)
        assert fd == pytest.approx(float(np.sum(g * d)), rel=1e-6)
