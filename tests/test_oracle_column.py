"""Pins of the oracle's vertical operator, Schur complement, probing, banded LU and solve."""
import numpy as np
import pytest

from oracle.column import Column, implicit_solve, lu_nopivot_banded, lu_solve_banded
from oracle.mesh import BoxMesh
from oracle.reference import GAMMA, R_GAS


def _col(nez=4, N=4, Lz=10e3, n_bv=0.0):
    m = BoxMesh(2, 2, nez, N, 4e3, 4e3, Lz)
    return m, Column(m, 300.0, n_bv)


def _lam(col, m, C):
    dzmin = (m.xi[1] - m.xi[0]) * m.dz / 2
    return (1 - 1 / np.sqrt(2)) * C * dzmin / np.sqrt(GAMMA * R_GAS * 300.0)


@pytest.mark.parametrize("N", [2, 4, 7])
def test_dz_exact_on_global_polynomials(N):
    m, col = _col(nez=3, N=N, Lz=3.0)
    z = col.z
    for p in range(N + 1):
        dp = p * z ** (p - 1) if p else np.zeros_like(z)
        np.testing.assert_allclose(col.Dz @ z ** p, dp, atol=1e-10 * N ** 3)


@pytest.mark.parametrize("n_bv", [0.0, 0.02])
@pytest.mark.parametrize("C", [1, 15, 150])
def test_probing_equals_direct_and_band(C, n_bv):
    m, col = _col(n_bv=n_bv)
    lam = _lam(col, m, C)
    S = col.jacobian_by_probing(lam)
    np.testing.assert_allclose(S, col.jacobian_direct(lam), rtol=0, atol=1e-13 * np.abs(S).max())
    hb = col.half_band
    assert np.all(np.triu(S, hb + 1) == 0) and np.all(np.tril(S, -hb - 1) == 0)
    assert np.abs(np.diag(S, hb)).max() > 0 and np.abs(np.diag(S, -hb)).max() > 0


@pytest.mark.parametrize("nez,N", [(4, 4), (2, 4), (12, 4), (3, 7)])
@pytest.mark.parametrize("C", [1, 15, 150])
def test_lu_solve_matches_dense_solve(nez, N, C):
    m, col = _col(nez=nez, N=N)
    lam = _lam(col, m, C)
    S = col.jacobian_by_probing(lam)
    LU = lu_nopivot_banded(S, col.half_band)
    L = np.tril(LU, -1) + np.eye(m.M)
    U = np.triu(LU)
    np.testing.assert_allclose(L @ U, S, atol=1e-12 * np.abs(S).max())
    b = np.random.default_rng(nez * N + C).standard_normal((3, m.M))
    x = lu_solve_banded(LU, col.half_band, b)
    xd = np.linalg.solve(S, b.T).T
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-11 * np.linalg.cond(S) * np.abs(xd).max())


@pytest.mark.parametrize("n_bv", [0.0, 0.02])
@pytest.mark.parametrize("C", [1, 15, 150])
def test_schur_form_equals_standard_form(C, n_bv):
    """The Schur elimination is exact at the discrete level: solving the 3M x 3M
    standard system for (rho', w, theta') gives the Schur solution after extraction."""
    m, col = _col(n_bv=n_bv)
    lam = _lam(col, m, C)
    rng = np.random.default_rng(C)
    re = 1e-3 * rng.standard_normal(m.M) * col.rho0
    we = rng.standard_normal(m.M)
    te = rng.standard_normal(m.M)
    we[0] = we[-1] = 0.0
    sol = np.linalg.solve(col.standard_matrix(lam), np.concatenate([re, we, te]))
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    b, wa = col.schur_rhs(re, we, te, lam)
    P = lu_solve_banded(LU, col.half_band, b)
    r, w, t = col.extract(P, wa, te, lam)
    M = m.M
    for got, ref in ((r, sol[:M]), (w, sol[M:2 * M]), (t, sol[2 * M:])):
        assert np.abs(got - ref).max() <= 1e-12 * C * (np.abs(ref).max() + 1e-300)


@pytest.mark.parametrize("n_bv", [0.0, 0.02])
def test_implicit_solve_residual(n_bv):
    """q = q_e + lam L_V(q) holds for the solved columns (u, v pass through)."""
    m, col = _col(n_bv=n_bv)
    lam = _lam(col, m, 15)
    rng = np.random.default_rng(1)
    q_e = rng.standard_normal((5, 3, m.M))
    q_e[0] *= 1e-3
    q_e[3][:, [0, -1]] = 0.0
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    q = implicit_solve(col, LU, q_e, lam)
    Lr, Lw, Lt = col.L_V(q[0], q[3], q[4])
    for f, L in ((0, Lr), (3, Lw), (4, Lt)):
        np.testing.assert_allclose(q[f] - lam * L, q_e[f], atol=1e-11 * np.abs(q_e[f]).max())
    np.testing.assert_array_equal(q[1], q_e[1])
    np.testing.assert_array_equal(q[2], q_e[2])


def test_small_lambda_gives_identity():
    m, col = _col()
    S = col.jacobian_by_probing(1e-9)
    assert np.abs(S - np.eye(m.M)).max() < 1e-6


def test_lowest_acoustic_mode_of_short_column():
    """Short closed column (H = 100 m): the lowest eigenfrequency of L_V is the pipe mode
    pi / T, T = int_0^H dz / c(z), c = sqrt(gamma P0 / rho0) the local sound speed
    (gravity corrections are ~1e-6 here)."""
    m = BoxMesh(1, 1, 2, 4, 1.0, 1.0, 100.0)
    col = Column(m)
    M = m.M
    K = np.zeros((3 * M, 3 * M))
    for j in range(3 * M):
        e = np.zeros(3 * M)
        e[j] = 1.0
        Lr, Lw, Lt = col.L_V(e[:M], e[M:2 * M], e[2 * M:])
        K[:, j] = np.concatenate([Lr, Lw, Lt])
    ev = np.linalg.eigvals(K)
    osc = np.abs(ev.imag[np.abs(ev.imag) > 1e-3])
    from oracle.reference import reference_profile, sound_speed
    zz = np.linspace(0.0, 100.0, 20001)
    r = reference_profile(zz, 300.0)
    inv_c = 1.0 / sound_speed(r["P0"], r["rho0"])
    T = np.sum(0.5 * (inv_c[1:] + inv_c[:-1]) * np.diff(zz))
    assert abs(osc.min() - np.pi / T) < 2e-5 * np.pi / T
    assert np.abs(ev.real).max() < 1e-6 * np.abs(ev).max()   # non-dissipative


# ---- standard (non-Schur) column form ---------------------------------------------------
@pytest.mark.parametrize("N,nez", [(2, 5), (4, 3), (7, 2)])
def test_interleaved_standard_matrix_is_banded(N, nez):
    from oracle.column import standard_half_band, standard_interleaved
    m = BoxMesh(1, 1, nez, N, 1e3, 1e3, 10e3)
    col = Column(m, 300.0, 0.01)
    K = standard_interleaved(col, 3.0)
    i, j = np.nonzero(K)
    assert np.abs(i - j).max() == standard_half_band(m) == 3 * N + 1


@pytest.mark.parametrize("n_bv", [0.0, 0.02])
@pytest.mark.parametrize("C", [1, 15, 150])
def test_standard_form_solve_equals_schur_solve(C, n_bv):
    """Banded no-pivot LU of the standard system and the Schur path give the same
    columns; w is zero at the walls in both (non-zero w_e there is overridden)."""
    from oracle.column import (implicit_solve_standard, standard_half_band,
                               standard_interleaved)
    m, col = _col(n_bv=n_bv)
    lam = _lam(col, m, C)
    rng = np.random.default_rng(10 + C)
    q_e = rng.standard_normal((5, 4, m.M))
    q_e[0] *= 1e-3 * col.rho0
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    LUs = lu_nopivot_banded(standard_interleaved(col, lam), standard_half_band(m))
    a = implicit_solve(col, LU, q_e, lam)
    b = implicit_solve_standard(col, LUs, q_e, lam)
    assert np.abs(b[3][:, [0, -1]]).max() == 0.0
    for f in range(5):
        assert np.abs(a[f] - b[f]).max() <= 1e-12 * C * np.abs(a[f]).max()


@pytest.mark.parametrize("N,nez", [(2, 5), (3, 4), (4, 1), (4, 6), (7, 3)])
@pytest.mark.parametrize("n_bv", [0.0, 0.02])
@pytest.mark.parametrize("C", [1, 150])
def test_lu_fill_stays_in_the_envelope(N, nez, n_bv, C):
    """The column kernels skip the factor entries outside the envelope of S(lam): column j
    of L reaches 2N - r levels below the diagonal and column j of U N + r above it, with
    r = j mod N (2N at an element interface, r = 0).  S has the pattern of D_z^2 and a
    no-pivot LU keeps its fill inside that envelope, so those entries of the oracle's own
    factors are exact zeros, and the outermost entries inside it are not all zero (the
    envelope is tight)."""
    m, col = _col(nez=nez, N=N, n_bv=n_bv)
    lam = _lam(col, m, C)
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    M = m.M
    env_l = lambda r: 2 * N if r == 0 else 2 * N - r
    env_u = lambda r: 2 * N if r == 0 else N + r
    edge_l, edge_u = [], []
    for j in range(M):
        r = j % N
        below = LU[j + 1 + env_l(r):, j]
        above = LU[:max(0, j - env_u(r)), j]
        assert np.all(below == 0.0) and np.all(above == 0.0), j
        if j + env_l(r) < M:
            edge_l.append(LU[j + env_l(r), j])
        if j - env_u(r) >= 0:
            edge_u.append(LU[j - env_u(r), j])
    if edge_l:
        assert np.any(np.array(edge_l) != 0.0)
        assert np.any(np.array(edge_u) != 0.0)


@pytest.mark.parametrize("N,nez", [(4, 12), (3, 5), (7, 2), (2, 1)])
def test_envelope_counts_used_by_the_benchmark(N, nez):
    """bench.envelope_entries (the algorithmic factor entries of the column-solve roofline)
    counts the entries of the oracle's factors that lie inside the envelope: L's below the
    diagonal, U's on and above it."""
    import bench
    m, col = _col(nez=nez, N=N)
    LU = lu_nopivot_banded(col.jacobian_by_probing(_lam(col, m, 15)), col.half_band)
    M = m.M
    nl = sum(min(2 * N if j % N == 0 else 2 * N - j % N, M - 1 - j) for j in range(M))
    nu = sum(min(2 * N if j % N == 0 else N + j % N, j) + 1 for j in range(M))
    assert bench.envelope_entries(N, nez) == (nl, nu)
    inside_l = sum(np.count_nonzero(LU[j + 1:, j]) for j in range(M))
    inside_u = sum(np.count_nonzero(LU[:j + 1, j]) for j in range(M))
    assert inside_l <= nl and inside_u <= nu          # no nonzero outside (see above)
    assert inside_l >= 0.9 * nl and inside_u >= 0.9 * nu
