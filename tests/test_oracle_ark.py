"""Pins of the ARK2 tableau and stage algorithm, the RK35 comparator, and the HEVI step."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from golden_io import read, values
from oracle import ark2, rk35
from oracle.column import Column
from oracle.mesh import BoxMesh
from oracle.reference import GAMMA, R_GAS
import synthetic


def _golden(key):
    for row in read("paper_constants.txt"):
        if row[0] == key:
            return values(row[1:])
    raise KeyError(key)


def test_ark2_tableau_reading():
    a, at, b, c = ark2.tableau()
    np.testing.assert_allclose(c, _golden("ark2_c"), atol=1e-15)
    assert abs(a[2, 1] - _golden("ark2_a32")[0]) < 1e-15
    np.testing.assert_allclose(at.sum(1), c, atol=1e-15)       # c~ = c
    assert abs(b.sum() - 1) < 1e-15                               # order 1
    assert abs(b @ c - 0.5) < 1e-15                               # order 2
    assert abs(b @ (a @ c) - 1 / 6) < 1e-15
    assert np.all(np.diag(at)[1:] == at[1, 1]) and at[0, 0] == 0  # SDIRK, explicit first stage
    assert abs((at[1, 0] - a[1, 0]) / at[1, 1] + 1.0) < 1e-15     # c21 = -1
    pb = ark2.printed_b()                                         # the garbled printed row
    assert abs(pb.sum() - 1) > 1.0                                # not even consistent


def _split_system(n=6, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    Nmat = 0.3 * (A - A.T) + 0.05 * rng.standard_normal((n, n))   # non-stiff part
    B = rng.standard_normal((n, n))
    Lmat = -(B @ B.T) * 0.5 + 2.0 * (B - B.T)                      # stiff linear part
    return Nmat, Lmat


def _ark_direct(y, dt, Nmat, Lmat):
    """ARK2 straight from the double tableau: Y_i = y + dt sum a_ij N Y_j + dt sum a~_ij L Y_j."""
    a, at, b, _ = ark2.tableau()
    n = len(y)
    Y = []
    for i in range(3):
        rhs = y + dt * sum(a[i, j] * Nmat @ Y[j] + at[i, j] * Lmat @ Y[j] for j in range(i))
        Y.append(np.linalg.solve(np.eye(n) - dt * at[i, i] * Lmat, rhs))
    return y + dt * sum(b[i] * (Nmat + Lmat) @ Y[i] for i in range(3))


def test_predictor_corrector_form_equals_double_tableau():
    Nmat, Lmat = _split_system()
    y = np.random.default_rng(1).standard_normal(6)
    R = lambda q: (Nmat + Lmat) @ q
    solve = lambda r, lam: np.linalg.solve(np.eye(6) - lam * Lmat, r)
    for dt in (0.01, 0.3, 3.0):
        np.testing.assert_allclose(ark2.ark_step(y, dt, R, solve), _ark_direct(y, dt, Nmat, Lmat),
                                   rtol=1e-12, atol=1e-12)


def test_ark2_second_order():
    Nmat, Lmat = _split_system(seed=2)
    y0 = np.random.default_rng(3).standard_normal(6)
    R = lambda q: (Nmat + Lmat) @ q
    solve = lambda r, lam: np.linalg.solve(np.eye(6) - lam * Lmat, r)
    T = 1.0
    errs = []
    for n in (20, 40, 80):
        y = y0
        for _ in range(n):
            y = ark2.ark_step(y, T / n, R, solve)
        errs.append(np.linalg.norm(y - expm(T * (Nmat + Lmat)) @ y0))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), rates


def test_rk35_order_conditions_and_root():
    A, b, c = rk35.butcher()
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert abs(b @ (c * c) - 1 / 3) < 1e-15
    assert abs(b @ (A @ c) - 1 / 6) < 1e-15
    ratios = (1 - rk35.ALPHA) / rk35.BETA
    assert abs(ratios.min() - 1 / 0.46) < 1e-12       # SSP coefficient 2.17
    assert np.all(rk35.ALPHA >= 0) and np.all(rk35.BETA > 0)
    # re-solve the four conditions in extended precision from a nearby start
    import mpmath as mp
    mp.mp.dps = 40

    def conds(b2, b3, b4, a4):
        beta = [mp.mpf("0.46"), b2, b3, b4, mp.mpf("0.46")]
        alpha = [0, 0, 0, a4, 0]
        prev = [mp.mpf(0)] * 5
        out = []
        for i in range(5):
            cur = [(1 - alpha[i]) * p for p in prev]
            cur[i] += beta[i]
            out.append(cur)
            prev = cur
        Am = [[mp.mpf(0)] * 5] + out[:4]
        bb = out[-1]
        cc = [sum(r) for r in Am]
        Ac = [sum(Am[i][j] * cc[j] for j in range(5)) for i in range(5)]
        return [sum(bb) - 1, sum(bb[i] * cc[i] for i in range(5)) - mp.mpf(1) / 2,
                sum(bb[i] * cc[i] ** 2 for i in range(5)) - mp.mpf(1) / 3,
                sum(bb[i] * Ac[i] for i in range(5)) - mp.mpf(1) / 6]

    root = mp.findroot(conds, (0.28, 0.22, 0.13, 0.58))
    np.testing.assert_allclose([float(r) for r in root],
                               [rk35.BETA[1], rk35.BETA[2], rk35.BETA[3], rk35.ALPHA[3]], rtol=1e-15)


def test_rk35_third_order():
    Nmat, Lmat = _split_system(seed=4)
    Mmat = 0.2 * (Nmat + 0.1 * Lmat)
    y0 = np.random.default_rng(5).standard_normal(6)
    errs = []
    for n in (10, 20, 40):
        y = y0
        for _ in range(n):
            y = rk35.rk35_step(y, 1.0 / n, lambda q: Mmat @ q)
        errs.append(np.linalg.norm(y - expm(Mmat) @ y0))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates


def _box(nex=4, nez=4, L=10e3, Lz=10e3):
    m = BoxMesh(nex, nex, nez, 4, L, L, Lz)
    col = Column(m)
    dzmin = (m.xi[1] - m.xi[0]) * m.dz / 2
    return m, col, dzmin / np.sqrt(GAMMA * R_GAS * 300.0)


def test_hevi_converges_to_rk35_at_small_courant():
    """1D-IMEX at small C approaches explicit RK (the difference shrinks ~dt^2)."""
    m, col, dt1 = _box(nex=3, nez=3)
    xg, yg, zg = m.coords()
    q0 = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Ly, m.Lz, col.rho0, col.theta0, 11)
    T = 8 * dt1
    E = rk35.Explicit(m, col)
    ref = E.step(q0, T / 32, 32)
    diffs = []
    for n in (8, 16):
        H = ark2.HEVI(m, col, T / n)
        q = H.step(q0, n)
        diffs.append(np.linalg.norm(q[3] - ref[3]) / np.linalg.norm(ref[3]))
    assert diffs[1] < diffs[0] / 3.0 and diffs[1] < 1e-2, diffs


@pytest.mark.parametrize("C,L", [(150, 3000e3)])
def test_hevi_bounded_at_large_vertical_courant(C, L):
    """Horizontally wide box (C_H = 0.5): ten steps at C_V = 150 stay bounded."""
    m, col, dt1 = _box(L=L)
    xg, yg, zg = m.coords()
    q0 = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Ly, m.Lz, col.rho0, col.theta0, 12)
    H = ark2.HEVI(m, col, C * dt1)
    q = H.step(q0, 10)
    assert np.isfinite(q).all()
    assert np.abs(q[3]).max() < 1.0 and np.abs(q[4]).max() < 1.0


@pytest.mark.parametrize("C", [15, 150])
def test_standard_form_step_equals_schur_step(C):
    """The standard (non-Schur) column system gives the same HEVI steps."""
    m, col, dt1 = _box(nex=2, nez=3, L=2000e3)
    xg, yg, zg = m.coords()
    q0 = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Lx, m.Lz, col.rho0, col.theta0, 13)
    a = ark2.HEVI(m, col, C * dt1).step(q0, 3)
    b = ark2.HEVI(m, col, C * dt1, form="standard").step(q0, 3)
    for f in range(5):
        assert np.abs(a[f] - b[f]).max() <= 1e-10 * max(np.abs(a[f]).max(), 1e-300)


# ---- ARK3 (ARK3(2)4L[2]SA; the paper prints no ARK3 tableau) ------------------------------
def test_ark3_order_conditions_exact():
    """Third order for the explicit and implicit tableaux and their coupling, c = c~,
    stiffly accurate (b = last implicit row), one implicit diagonal: checked in exact
    rational arithmetic (the published rationals approximate irrational coefficients to
    about 1e-26)."""
    from fractions import Fraction as F
    from oracle import ark3
    a, at, b, c = ark3.rational_tableau()
    s = 4
    tol = F(1, 10 ** 20)
    ct = [sum(F(x) for x in row) for row in at]
    assert all(abs(c[i] - ct[i]) < tol for i in range(s))
    assert tuple(b) == tuple(at[3])
    assert at[0][0] == 0 and all(at[i][i] == ark3.GAMMA for i in range(1, s))
    conds = [
        (sum(b), 1),
        (sum(b[i] * c[i] for i in range(s)), F(1, 2)),
        (sum(b[i] * c[i] ** 2 for i in range(s)), F(1, 3)),
    ]
    for A1 in (a, at):
        for A2 in (a, at):
            conds.append((sum(b[i] * A1[i][j] * c[j] for i in range(s) for j in range(s)), F(1, 6)))
            conds.append((sum(b[i] * A1[i][j] * sum(F(x) for x in A2[j]) for i in range(s)
                              for j in range(s)), F(1, 6)))
    for got, want in conds:
        assert abs(F(got) - want) < tol


def _ark_direct_tab(y, dt, Nmat, Lmat, tab):
    a, at, b, _ = tab
    n, s = len(y), len(b)
    Y = []
    for i in range(s):
        rhs = y + dt * sum(a[i, j] * Nmat @ Y[j] + at[i, j] * Lmat @ Y[j] for j in range(i))
        Y.append(np.linalg.solve(np.eye(n) - dt * at[i, i] * Lmat, rhs))
    return y + dt * sum(b[i] * (Nmat + Lmat) @ Y[i] for i in range(s))


def test_ark3_predictor_corrector_form_equals_double_tableau():
    from oracle import ark3
    Nmat, Lmat = _split_system(seed=4)
    y = np.random.default_rng(5).standard_normal(6)
    R = lambda q: (Nmat + Lmat) @ q
    solve = lambda r, lam: np.linalg.solve(np.eye(6) - lam * Lmat, r)
    tab = ark3.tableau()
    for dt in (0.01, 0.3, 3.0):
        np.testing.assert_allclose(ark2.ark_step(y, dt, R, solve, tab),
                                   _ark_direct_tab(y, dt, Nmat, Lmat, tab), rtol=1e-12, atol=1e-12)


def test_ark3_third_order():
    from oracle import ark3
    Nmat, Lmat = _split_system(seed=6)
    y0 = np.random.default_rng(7).standard_normal(6)
    R = lambda q: (Nmat + Lmat) @ q
    solve = lambda r, lam: np.linalg.solve(np.eye(6) - lam * Lmat, r)
    T = 1.0
    exact = expm((Nmat + Lmat) * T) @ y0
    tab = ark3.tableau()
    errs = []
    for n in (40, 80, 160):
        y = y0.copy()
        for _ in range(n):
            y = ark2.ark_step(y, T / n, R, solve, tab)
        errs.append(np.linalg.norm(y - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates


def test_hevi_ark3_converges_faster_than_ark2():
    """On the Set2NC box with resolved vertical acoustics (C = 1, 0.5): against a fine
    ARK3 run, ARK3's error at C = 0.5 is at least 3x below ARK2's, and it drops at a rate
    above 2.5 (ARK2: below 2.3)."""
    m, col, dt1 = _box(nex=2, nez=3, L=400e3)
    xg, yg, zg = m.coords()
    q0 = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Lx, m.Lz, col.rho0, col.theta0, 15)
    T = 16 * dt1
    ref = ark2.HEVI(m, col, T / 128, scheme="ark3").step(q0, 128)
    err = {}
    for s in ("ark2", "ark3"):
        for n in (16, 32):
            q = ark2.HEVI(m, col, T / n, scheme=s).step(q0, n)
            err[(s, n)] = np.linalg.norm(q[3] - ref[3]) / np.linalg.norm(ref[3])
    assert err[("ark3", 32)] < err[("ark2", 32)] / 3.0, err
    assert np.log2(err[("ark3", 16)] / err[("ark3", 32)]) > 2.5, err
    assert np.log2(err[("ark2", 16)] / err[("ark2", 32)]) < 2.3, err


# ---- ARK4, ARK5 and the order-condition machinery --------------------------------------

def test_bicoloured_tree_counts():
    """The numbers of rooted trees with two-coloured non-root vertices (oriented rooted
    trees, OEIS A000151): 1, 2, 7, 26, 107, 458."""
    from oracle.ark_order import trees
    assert [len(trees(n)) for n in range(1, 7)] == [1, 2, 7, 26, 107, 458]


def test_order_conditions_on_textbook_pairs():
    """The classical fourth-order Runge-Kutta method used as both halves of a pair is of
    order exactly 4; the explicit / implicit Euler pair of order exactly 1; a 1e-6 change of
    one ARK4 entry breaks order 2 or more."""
    from fractions import Fraction as F
    from oracle import ark4
    from oracle.ark_order import residuals
    h = F(1, 2)
    rk4 = ((0, 0, 0, 0), (h, 0, 0, 0), (0, h, 0, 0), (0, 0, 1, 0))
    res = residuals(rk4, rk4, (F(1, 6), F(1, 3), F(1, 3), F(1, 6)), 5)
    assert all(res[n] == 0 for n in range(1, 5)) and res[5] > F(1, 1000)
    res = residuals(((0, 0), (1, 0)), ((0, 0), (0, 1)), (0, 1), 2)
    assert res[1] == 0 and res[2] >= F(1, 2)
    a, at, b, _ = ark4.rational_tableau()
    bad = [list(r) for r in a]
    bad[4][2] += F(1, 10 ** 6)
    res = residuals(bad, at, b, 4)
    assert res[1] == 0 and max(res[n] for n in (2, 3, 4)) > F(1, 10 ** 8)


@pytest.mark.parametrize("name,p", [("ark3", 3), ("ark4", 4), ("ark5", 5)])
def test_ark_tableau_order_conditions_exact(name, p):
    """Every bicoloured-tree condition up to order p holds to the accuracy of the published
    rationals (<= 1e-25), order p + 1 fails, c = c~, b = the last implicit row, and one
    implicit diagonal over an explicit first stage."""
    import importlib
    from fractions import Fraction as F
    from oracle.ark_order import residuals
    m = importlib.import_module("oracle." + name)
    a, at, b, c = m.rational_tableau()
    s = len(b)
    tol = F(1, 10 ** 25)
    res = residuals(a, at, b, p + 1)
    assert all(res[n] < tol for n in range(1, p + 1)), res
    assert res[p + 1] > F(1, 10 ** 4)
    ct = [sum(F(x) for x in row) for row in at]
    assert all(abs(F(c[i]) - ct[i]) < tol for i in range(s))
    assert tuple(b) == tuple(at[-1])
    assert at[0][0] == 0 and all(at[i][i] == m.GAMMA for i in range(1, s))
    assert all(a[i][j] == 0 for i in range(s) for j in range(i, s))
    assert all(at[i][j] == 0 for i in range(s) for j in range(i + 1, s))


def test_ark5_row8_is_the_order_condition_solution():
    """The two derived ARK5 entries are the least-squares solution of the fifth-order
    conditions: Gauss-Newton started there does not move them."""
    pytest.importorskip("mpmath")
    from oracle import ark5, derive_ark5_row8
    x, r = derive_ark5_row8.solve((float(ark5.A86), float(ark5.A87)), iters=4)
    assert derive_ark5_row8.rationals(x) == (ark5.A86, ark5.A87)
    assert float(r) < 1e-25


@pytest.mark.parametrize("name", ["ark4", "ark5"])
def test_ark45_predictor_corrector_form_equals_double_tableau(name):
    Nmat, Lmat = _split_system(seed=8)
    y = np.random.default_rng(9).standard_normal(6)
    R = lambda q: (Nmat + Lmat) @ q
    solve = lambda r, lam: np.linalg.solve(np.eye(6) - lam * Lmat, r)
    tab = ark2.scheme_tableau(name)
    for dt in (0.01, 0.3, 3.0):
        np.testing.assert_allclose(ark2.ark_step(y, dt, R, solve, tab),
                                   _ark_direct_tab(y, dt, Nmat, Lmat, tab), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name,rate", [("ark2", 1.9), ("ark3", 2.7), ("ark4", 3.8), ("ark5", 4.7)])
def test_ark_rate_on_a_nonlinear_split_system(name, rate):
    """y' = N(y) + L y with N nonlinear (sin of a random mixing plus a quadratic) and L a
    moderately stiff linear part, against an adaptive eighth-order Dormand-Prince solution:
    the error drops at the scheme's order (nonlinear N exercises the coupling conditions
    that a linear test cannot)."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(11)
    n = 4
    Lm = -np.diag([1.0, 3.0, 8.0, 20.0]) + 0.3 * rng.standard_normal((n, n))
    K = rng.standard_normal((n, n))
    R = lambda y: np.sin(K @ y) + 0.5 * y[::-1] ** 2 + Lm @ y
    solve = lambda r, lam: np.linalg.solve(np.eye(n) - lam * Lm, r)
    y0 = 0.5 * rng.standard_normal(n)
    ref = solve_ivp(lambda t, y: R(y), (0.0, 1.0), y0, method="DOP853", rtol=3e-14,
                    atol=1e-15).y[:, -1]
    tab = ark2.scheme_tableau(name)
    errs = []
    for k in (32, 64):
        y = y0.copy()
        for _ in range(k):
            y = ark2.ark_step(y, 1.0 / k, R, solve, tab)
        errs.append(np.linalg.norm(y - ref))
    assert np.log2(errs[0] / errs[1]) > rate, errs


def test_hevi_ark4_ark5_rates_on_the_box():
    """HEVI with ARK4 and ARK5 on the Set2NC box with resolved vertical acoustics: against a
    fine run of the same scheme the error drops at rates above 3.4 and 4.4, and ARK5 is
    at least 3x more accurate than ARK4 at the same step."""
    m, col, dt1 = _box(nex=2, nez=3, L=400e3)
    xg, yg, zg = m.coords()
    q0 = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Lx, m.Lz, col.rho0, col.theta0, 15)
    T = 16 * dt1
    err = {}
    for s in ("ark4", "ark5"):
        ref = ark2.HEVI(m, col, T / 64, scheme=s).step(q0, 64)
        for n in (8, 16):
            q = ark2.HEVI(m, col, T / n, scheme=s).step(q0, n)
            err[(s, n)] = np.linalg.norm(q[3] - ref[3]) / np.linalg.norm(ref[3])
    assert np.log2(err[("ark4", 8)] / err[("ark4", 16)]) > 3.4, err
    assert np.log2(err[("ark5", 8)] / err[("ark5", 16)]) > 4.4, err
    assert err[("ark5", 16)] < err[("ark4", 16)] / 3.0, err
