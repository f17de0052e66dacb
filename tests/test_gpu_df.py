"""The double-float right-hand side (precision "df") against the FP64 oracle, at the FP64
method's bars: relative L2 <= 1e-11 per RHS, <= 1e-9 after a run.  The derivative sums carry
about 48 significant bits (products by Dekker's method, sums by TwoSum), the rest is FP64."""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-11
RUN_TOL = 1e-9


def ctx(case, dt=0.0):
    import paper_1702_04316_gb300 as pkg
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, precision="df")


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    "tiny4": (4, 4, 4, 4, 10e3, 10e3, 10e3),
    "ragged": (3, 5, 2, 3, 7e3, 9e3, 4e3),
    "n2": (5, 2, 3, 2, 6e3, 3e3, 5e3),
    "n7": (2, 3, 2, 7, 8e3, 9e3, 6e3),
    "n8": (2, 2, 2, 8, 4e3, 4e3, 4e3),
    "single": (1, 1, 1, 4, 2e3, 2e3, 2e3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_df_rhs_matches_oracle(name):
    from oracle.rhs import rhs
    case = Case(*CASES[name], n_bv=0.01)
    q = case.state(3, vel=5.0)
    out = ctx(case).rhs_explicit(dev(q)).cpu().numpy()
    ref = rhs(case.mesh, case.col, q)
    e = rel_l2(out, ref)
    assert np.all(e <= RHS_TOL), e


@pytest.mark.parametrize("name", ["tiny4", "ragged", "n7"])
def test_df_rhs_of_a_balanced_state(name):
    """Bubble balance: P' = 0 in exact arithmetic, so the horizontal tendencies are the
    derivatives of rounding noise (no relative error is defined for them); they must be
    negligible against the buoyancy tendency, which matches the oracle to 1e-11."""
    from oracle.rhs import rhs
    case = Case(*CASES[name], n_bv=0.01)
    q = case.state(3, kind="balanced")
    out = ctx(case).rhs_explicit(dev(q)).cpu().numpy()
    ref = rhs(case.mesh, case.col, q)
    e = rel_l2(out, ref)
    assert e[3] <= RHS_TOL, e
    assert np.abs(out[1:3]).max() <= 1e-9 * np.abs(ref[3]).max()


@pytest.mark.parametrize("C,L", [(15, 400e3), (150, 4000e3)])
def test_df_run_matches_oracle(C, L):
    from oracle import ark2
    case = Case(4, 3, 3, 4, L, 0.75 * L, 10e3, n_bv=0.01)
    dt = case.dt_for(C)
    q0 = case.state(31, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, 6)
    g = ctx(case, dt)
    out = g.step_imex1d(dev(q0), g.empty_state(), 6).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)


def test_df_rk35_run_matches_oracle():
    from oracle import rk35
    case = Case(*CASES["tiny4"])
    dt = case.dt_for(1.0)
    q0 = case.state(5, kind="balanced")
    ref = rk35.Explicit(case.mesh, case.col).step(q0, dt, 10)
    g = ctx(case)
    out = g.step_explicit_rk(dev(q0), dt, g.empty_state(), 10).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)


def test_df_against_fp64_kernel():
    """The two kernels differ only in the derivative sums' arithmetic."""
    import paper_1702_04316_gb300 as pkg
    case = Case(6, 6, 4, 4, 12e3, 12e3, 8e3, n_bv=0.01)
    q = dev(case.state(7, vel=5.0))
    a = ctx(case).rhs_explicit(q)
    b = pkg.Numa(*case.args[:6], case.args[6], 0.0, 300.0, 0.01).rhs_explicit(q)
    e = rel_l2(a.cpu().numpy(), b.cpu().numpy())
    assert np.all(e <= 1e-12), e
    assert a.dtype == b.dtype
