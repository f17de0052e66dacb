"""3D-IMEX (Schur form, BiCGstab + polynomial preconditioner) on the GPU against the oracle.

Tolerances: the Schur operator is a short FP64 stencil sum like the RHS (<= 1e-11 relative
L2).  Solves are iterative, stopping when the preconditioned residual has dropped by
1e-13 here.  So solutions, stages and runs are compared at 1e-9, the run bar; the GPU and
the oracle build their preconditioners from their own spectrum estimates.
"""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-11
RUN_TOL = 1e-9
KTOL = 1e-13


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_1702_04316_gb300 as p
    p.lib()
    return p


def ctx(pkg, case, dt, **kw):
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    kw.setdefault("krylov_tol", KTOL)
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, imex="3d", **kw)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def lam_of(dt):
    return (1.0 - 1.0 / np.sqrt(2.0)) * dt


CASES = [(3, 2, 2, 4, 9e3, 6e3, 6e3), (2, 3, 3, 3, 6e3, 9e3, 9e3), (2, 2, 2, 6, 6e3, 6e3, 4e3)]


@pytest.mark.parametrize("dims", CASES)
def test_schur3d_operator_matches_oracle(pkg, torch, dims):
    from oracle.schur3d import Schur3D
    case = Case(*dims, n_bv=0.01)
    dt = case.dt_for(15.0)
    g = ctx(pkg, case, dt)
    P = np.random.default_rng(1).standard_normal(case.mesh.nnode)
    got = g.schur3d_apply(dev(torch, P)).cpu().numpy()
    ref = Schur3D(case.mesh, case.col).apply(P, lam_of(dt))
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


def test_preconditioner_coefficients_match_oracle(pkg, torch):
    from oracle import schur3d as s3
    case = Case(*CASES[0], n_bv=0.01)
    dt = case.dt_for(15.0)
    for P in (1, 2, 4):
        g = ctx(pkg, case, dt, pbno_order=P)
        info = g.imex3d_info()
        c, lb = s3.chebyshev_pbno(P, 1.0, info["l_max"])
        assert info["lam_bar"] == pytest.approx(lb, rel=1e-14)
        np.testing.assert_allclose(info["coeffs"], c, rtol=1e-9, atol=1e-12 * np.abs(c).max())
    op = s3.Schur3D(case.mesh, case.col)
    lmax = s3.power_lmax(lambda x: op.apply(x, lam_of(dt)), case.mesh.nnode, iters=300)
    assert info["l_max"] == pytest.approx(1.05 * lmax, rel=0.05)


@pytest.mark.parametrize("P", [0, 2, 4])
def test_solve_matches_dense_oracle_solution(pkg, torch, P):
    from oracle.schur3d import Schur3D
    case = Case(*CASES[1], n_bv=0.01)
    dt = case.dt_for(15.0)
    g = ctx(pkg, case, dt, pbno_order=P if P else 1)
    op = Schur3D(case.mesh, case.col)
    n = case.mesh.nnode
    S = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        S[:, k] = op.apply(e, lam_of(dt))
    b = np.random.default_rng(2).standard_normal(n)
    x, it = g.solve_schur3d(dev(torch, b))
    ref = np.linalg.solve(S, b)
    assert 0 < it < 500
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("stage", [2, 3])
def test_stages_match_oracle(pkg, torch, stage):
    from oracle import ark2
    from oracle.rhs import rhs
    from oracle.schur3d import HEVI3D
    case = Case(*CASES[0], n_bv=0.02)
    dt = case.dt_for(15.0)
    g = ctx(pkg, case, dt)
    h = HEVI3D(case.mesh, case.col, dt, tol=KTOL)
    a, at, b, _ = ark2.tableau()
    q0 = case.state(7)
    m, col = case.mesh, case.col

    def stage_ref(i, Q, Rs):
        cij = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        qtt_e = q0 + dt * sum(a[i, j] * Rs[j] for j in range(i)) + sum(cij[j] * Q[j] for j in range(i))
        return h.solve(qtt_e, h.lam) - sum(cij[j] * Q[j] for j in range(i))

    R1 = rhs(m, col, q0)
    q2 = stage_ref(1, [q0], [R1])
    if stage == 2:
        got, it = g.imex3d_stage(2, dev(torch, q0), dev(torch, R1))
        assert np.all(rel_l2(got.cpu().numpy(), q2) <= RUN_TOL), rel_l2(got.cpu().numpy(), q2)
    else:
        R2 = rhs(m, col, q2)
        q3 = stage_ref(2, [q0, q2], [R1, R2])
        got, it = g.imex3d_stage(3, dev(torch, q0), dev(torch, R1), dev(torch, R2), dev(torch, q2))
        assert np.all(rel_l2(got.cpu().numpy(), q3) <= RUN_TOL), rel_l2(got.cpu().numpy(), q3)
    assert it > 0


@pytest.mark.parametrize("scheme", ["ark2", "ark3"])
def test_run_matches_oracle_at_large_horizontal_courant(pkg, torch, scheme):
    """C_V = C_H = 15 on a cube of elements (1D-IMEX is unstable here)."""
    from oracle.schur3d import HEVI3D
    case = Case(3, 3, 3, 3, 9e3, 9e3, 9e3)
    dt = case.dt_for(15.0)
    q0 = case.state(22, kind="balanced")
    ref = HEVI3D(case.mesh, case.col, dt, tol=KTOL, scheme=scheme).step(q0, 3)
    g = ctx(pkg, case, dt, scheme=scheme)
    out = g.step_imex3d(dev(torch, q0), g.empty_state(), 3).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)
    assert g.imex3d_info()["iters_last_step"] > 0
    assert g.status() == pkg.NUMA_OK


def test_imex3d_rejections(pkg, torch):
    case = Case(2, 2, 2, 4, 4e3, 4e3, 4e3)
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    with pytest.raises(pkg.NumaError):
        pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, 1.0, precision="mixed", imex="3d")
    with pytest.raises(pkg.NumaError):
        pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, 1.0, column_form="standard", imex="3d")
    g = ctx(pkg, case, case.dt_for(15.0))
    q = dev(torch, case.state(1))
    assert g.query(pkg.Q_IMEX) == 1 and g.query(pkg.Q_FACTOR_BYTES) == 0
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.step_imex1d(q, g.empty_state(), 1)
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.solve_columns(torch.zeros(case.mesh.nnode, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.rhs_adjoint(q, q)
    one_d = pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, case.dt_for(15.0))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        one_d.step_imex3d(q, one_d.empty_state(), 1)


def test_column_preconditioner_matches_oracle(pkg, torch):
    from oracle.schur3d import HEVI3D
    case = Case(3, 3, 3, 3, 9e3, 9e3, 9e3, n_bv=0.01)
    dt = case.dt_for(15.0)
    q0 = case.state(23, kind="balanced")
    ref = HEVI3D(case.mesh, case.col, dt, tol=KTOL, precond="column").step(q0, 2)
    g = ctx(pkg, case, dt, precond="column")
    assert g.query(pkg.Q_FACTOR_BYTES) > 0
    out = g.step_imex3d(dev(torch, q0), g.empty_state(), 2).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)
    pb = ctx(pkg, case, dt).step_imex3d(dev(torch, q0), None, 2).cpu().numpy()
    assert np.all(rel_l2(out, pb) <= RUN_TOL), rel_l2(out, pb)
