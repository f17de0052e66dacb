"""The standard (non-Schur) column form on the GPU against the FP64 oracle.

Same tolerances as the Schur form: single stages and factors <= 1e-11 relative (factors
entrywise against the band's largest entry), steps after a run <= 1e-9 per field.
The two forms solve the same column system, so a run with the standard form also matches
the Schur form's run (<= 1e-10).
"""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-11
RUN_TOL = 1e-9


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_1702_04316_gb300 as p
    p.lib()
    return p


def ctx(pkg, case, dt, form="standard"):
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, column_form=form)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,nez", [(2, 4), (4, 3), (7, 2)])
def test_factors_match_oracle(pkg, torch, N, nez):
    from oracle.column import lu_nopivot_banded, standard_half_band, standard_interleaved
    case = Case(2, 3, nez, N, 5e3, 7e3, 8e3, n_bv=0.012)
    dt = case.dt_for(15.0)
    g = ctx(pkg, case, dt)
    hb = standard_half_band(case.mesh)
    assert g.query(pkg.Q_HALF_BAND) == hb
    assert g.query(pkg.Q_COLUMN_FORM) == 1
    lam = (1.0 - 1.0 / np.sqrt(2.0)) * dt
    LU = lu_nopivot_banded(standard_interleaved(case.col, lam), hb)
    n = 3 * case.mesh.M
    ref = np.zeros((n, 2 * hb + 1))
    for i in range(n):
        for j in range(max(0, i - hb), min(n, i + hb + 1)):
            ref[i, j - i + hb] = LU[i, j]
    got = g.column_factors(5)
    assert got.shape == (n, 2 * hb + 1)
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


def test_factor_memory_against_schur(pkg, torch):
    case = Case(3, 3, 12, 4, 6e3, 6e3, 15e3)
    dt = case.dt_for(15.0)
    a = ctx(pkg, case, dt, "schur").query(pkg.Q_FACTOR_BYTES)
    b = ctx(pkg, case, dt, "standard").query(pkg.Q_FACTOR_BYTES)
    N = 4
    assert b * (4 * N + 1) == a * 3 * (6 * N + 3)      # 3M (6N+3) vs M (4N+1) per column


@pytest.mark.parametrize("C", [15, 150])
def test_stages_match_oracle(pkg, torch, C):
    from oracle import ark2
    from oracle.rhs import rhs
    case = Case(3, 5, 2, 3, 7e3, 9e3, 4e3, n_bv=0.02)
    dt = case.dt_for(C)
    g = ctx(pkg, case, dt)
    h = ark2.HEVI(case.mesh, case.col, dt, form="standard")
    m, col = case.mesh, case.col
    a, at, b, _ = ark2.tableau()
    q0 = case.state(7)

    def stage_ref(i, Q, Rs):
        cij = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        qtt_e = q0 + dt * sum(a[i, j] * Rs[j] for j in range(i)) + sum(cij[j] * Q[j] for j in range(i))
        return h.solve(qtt_e, h.lam) - sum(cij[j] * Q[j] for j in range(i))

    R1 = rhs(m, col, q0)
    q2 = stage_ref(1, [q0], [R1])
    R2 = rhs(m, col, q2)
    q3 = stage_ref(2, [q0, q2], [R1, R2])
    g2 = g.imex_stage(2, dev(torch, q0), dev(torch, R1)).cpu().numpy()
    assert np.all(rel_l2(g2, q2) <= TOL), rel_l2(g2, q2)
    g3 = g.imex_stage(3, dev(torch, q0), dev(torch, R1), dev(torch, R2), dev(torch, q2)).cpu().numpy()
    assert np.all(rel_l2(g3, q3) <= TOL), rel_l2(g3, q3)


@pytest.mark.parametrize("C,L,nsteps", [(15, 400e3, 6), (150, 4000e3, 4)])
def test_run_matches_oracle_and_schur_form(pkg, torch, C, L, nsteps):
    from oracle import ark2
    case = Case(4, 3, 3, 4, L, 0.75 * L, 10e3, n_bv=0.01)
    dt = case.dt_for(C)
    q0 = case.state(41, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt, form="standard").step(q0, nsteps)
    assert np.isfinite(ref).all()
    out = ctx(pkg, case, dt).step_imex1d(dev(torch, q0), None, nsteps).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)
    schur = ctx(pkg, case, dt, "schur").step_imex1d(dev(torch, q0), None, nsteps).cpu().numpy()
    assert np.all(rel_l2(out, schur) <= 1e-10), rel_l2(out, schur)


def test_standard_form_rejections(pkg, torch):
    case = Case(2, 2, 2, 4, 4e3, 4e3, 4e3)
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    with pytest.raises(pkg.NumaError):
        pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, 1.0, precision="mixed", column_form="standard")
    g = ctx(pkg, case, case.dt_for(15.0))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.solve_columns(torch.zeros(case.mesh.ncol * case.mesh.M, dtype=torch.float64, device="cuda"))
    q = dev(torch, case.state(1))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.rhs_adjoint(q, q)
