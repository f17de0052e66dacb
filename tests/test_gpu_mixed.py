"""The mixed-precision form (FP32 right-hand side over the FP64 reference, FP32 column LU
with FP64 iterative refinement, FP64 state accumulation) against the FP64 oracle.

Its errors are stated, not bit tolerances: FP32 arithmetic in the right-hand side gives
~1e-7 relative errors; the refined solves reach FP64 accuracy."""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu


def ctx(case, dt=0.0, iters=1):
    import paper_1702_04316_gb300 as pkg
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, precision="mixed",
                    refine_iters=iters)


@pytest.mark.parametrize("dims,n_bv", [((4, 4, 4, 4, 10e3, 10e3, 10e3), 0.0),
                                        ((3, 4, 2, 7, 9e3, 8e3, 6e3), 0.01)])
def test_mixed_rhs_error(dims, n_bv):
    import torch
    from oracle.rhs import rhs
    case = Case(*dims[:3], dims[3], *dims[4:], n_bv)
    g = ctx(case)
    q0 = case.state(21)
    r = g.rhs_explicit(torch.from_numpy(q0).cuda()).cpu().numpy()
    e = rel_l2(r, rhs(case.mesh, case.col, q0))
    assert np.all(e < 2e-6), e


@pytest.mark.parametrize("C,iters,tol", [(15, 1, 1e-10), (15, 2, 1e-12), (150, 3, 1e-11)])
def test_mixed_solve_refined_to_fp64(C, iters, tol):
    import torch
    from oracle.column import lu_nopivot_banded, lu_solve_banded
    case = Case(3, 3, 4, 4, 9e3, 9e3, 10e3)
    dt = case.dt_for(C)
    g = ctx(case, dt, iters)
    col = case.col
    LU = lu_nopivot_banded(col.jacobian_by_probing((1 - 1 / np.sqrt(2)) * dt), col.half_band)
    m = case.mesh
    fac = g.column_factors(m.ncol // 2)
    band = np.zeros_like(fac)
    hb = col.half_band
    for i in range(m.M):
        for j in range(max(0, i - hb), min(m.M, i + hb + 1)):
            band[i, j - i + hb] = LU[i, j]
    assert np.abs(fac - band).max() < 1e-5 * np.abs(band).max()        # FP32 factors
    b = np.random.default_rng(C).standard_normal((m.ncol, m.M))
    x = g.solve_columns(torch.from_numpy(b.ravel()).cuda()).cpu().numpy().reshape(m.ncol, m.M)
    xr = lu_solve_banded(LU, hb, b)
    assert np.linalg.norm(x - xr) <= tol * np.linalg.norm(xr)


def test_mixed_stage_with_fp64_inputs():
    import torch
    from oracle import ark2
    from oracle.column import implicit_solve, lu_nopivot_banded
    from oracle.rhs import rhs
    case = Case(3, 5, 2, 3, 7e3, 9e3, 4e3, 0.02)
    dt = case.dt_for(15)
    g = ctx(case, dt, 2)
    m, col = case.mesh, case.col
    a, at, b, _ = ark2.tableau()
    lam = at[1, 1] * dt
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    q0 = case.state(7)
    R1 = rhs(m, col, q0)
    cij = (at[1, 0] - a[1, 0]) / at[1, 1]
    qtt_e = q0 + dt * a[1, 0] * R1 + cij * q0
    q2 = implicit_solve(col, LU, qtt_e.reshape(5, m.ncol, m.M), lam).reshape(5, -1) - cij * q0
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g2 = g.imex_stage(2, T(q0), T(R1)).cpu().numpy()
    assert np.all(rel_l2(g2, q2) < 1e-10), rel_l2(g2, q2)


@pytest.mark.parametrize("C,L", [(15, 300e3), (150, 3000e3)])
def test_mixed_run_error_is_stated(C, L):
    """Ten steps on the horizontally wide box: FP32 right-hand sides bound the error."""
    import torch
    from oracle import ark2
    case = Case(4, 4, 4, 4, L, L, 10e3)
    dt = case.dt_for(C)
    q0 = case.state(31, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, 10)
    g = ctx(case, dt, 2)
    out = g.step_imex1d(torch.from_numpy(q0).cuda(), g.empty_state(), 10).cpu().numpy()
    e = rel_l2(out, ref)
    print("mixed-form relative L2 after 10 steps, C=%d:" % C, e)
    assert np.all(e[[0, 3, 4]] < 1e-4), e


def test_mixed_rk35_run():
    import torch
    from oracle import rk35
    case = Case(4, 4, 4, 4, 10e3, 10e3, 10e3)
    dt = case.dt_for(1.0)
    q0 = case.state(5, kind="balanced")
    ref = rk35.Explicit(case.mesh, case.col).step(q0, dt, 10)
    g = ctx(case)
    out = g.step_explicit_rk(torch.from_numpy(q0).cuda(), dt, g.empty_state(), 10).cpu().numpy()
    e = rel_l2(out, ref)
    assert np.all(e[[0, 3, 4]] < 1e-4), e


# ---- FP32 right-hand side with the FP64 column factors (NUMA_PREC_RHS32) ------------------
def ctx32(case, dt=0.0):
    import paper_1702_04316_gb300 as pkg
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, precision="rhs32")


def test_rhs32_factors_are_fp64():
    import paper_1702_04316_gb300 as pkg
    case = Case(3, 3, 3, 4, 6e3, 6e3, 6e3)
    dt = case.dt_for(15.0)
    a = ctx32(case, dt)
    b = pkg.Numa(*case.args[:6], case.args[6], dt)
    assert a.query(pkg.Q_PRECISION) == 2
    assert a.query(pkg.Q_FACTOR_BYTES) == b.query(pkg.Q_FACTOR_BYTES)
    np.testing.assert_array_equal(a.column_factors(7), b.column_factors(7))


@pytest.mark.parametrize("C,L", [(15, 300e3), (150, 3000e3)])
def test_rhs32_run_error_is_stated(C, L):
    """Ten steps on the horizontally wide box: only the FP32 right-hand sides differ from
    the FP64 method; errors of the same size as the mixed form's."""
    import torch
    from oracle import ark2
    case = Case(4, 4, 4, 4, L, L, 10e3)
    dt = case.dt_for(C)
    q0 = case.state(31, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, 10)
    g = ctx32(case, dt)
    out = g.step_imex1d(torch.from_numpy(q0).cuda(), g.empty_state(), 10).cpu().numpy()
    e = rel_l2(out, ref)
    print("rhs32 relative L2 after 10 steps, C=%d:" % C, e)
    assert np.all(e[[0, 3, 4]] < 1e-4), e
