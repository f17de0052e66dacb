"""ARK4 and ARK5 (the paper's fourth- and fifth-order runs: ARK4(3)6L[2]SA and ARK5(4)8L[2]SA)
and the general fused stage on the GPU against the FP64 oracle.

Tolerances as for ARK2: a single stage <= 1e-11 relative L2 per field, a run <= 1e-9.
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


def ctx(pkg, case, dt, **kw):
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv, **kw)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("scheme", ["ark2", "ark3", "ark4", "ark5"])
def test_every_stage_matches_oracle(pkg, torch, scheme):
    """Each stage i = 2..s of the scheme from the oracle's own earlier stages (so that each
    stage is checked on its own), through numa_imex_stage_s."""
    from oracle import ark2
    from oracle.rhs import rhs
    case = Case(3, 5, 2, 3, 70e3, 90e3, 4e3, n_bv=0.02)
    m, col = case.mesh, case.col
    dt = case.dt_for(15.0)
    g = ctx(pkg, case, dt, scheme=scheme)
    h = ark2.HEVI(m, col, dt, scheme=scheme)
    a, at, b, _ = h.tab
    q0 = case.state(7)
    Q, Rs = [q0], [rhs(m, col, q0)]
    for i in range(1, len(b)):
        cij = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        qtt_e = q0 + dt * sum(a[i, j] * Rs[j] for j in range(i)) + sum(cij[j] * Q[j] for j in range(i))
        qi = h.solve(qtt_e, h.lam) - sum(cij[j] * Q[j] for j in range(i))
        gi = g.imex_stage_s(i + 1, dev(torch, q0), [dev(torch, r) for r in Rs],
                            [dev(torch, x) for x in Q[1:]]).cpu().numpy()
        assert np.all(rel_l2(gi, qi) <= TOL), (i + 1, rel_l2(gi, qi))
        Q.append(qi)
        Rs.append(rhs(m, col, qi))


@pytest.mark.parametrize("scheme", ["ark2", "ark3"])
def test_general_stage_equals_the_fixed_stage_bitwise(pkg, torch, scheme):
    """Where every coefficient is nonzero the general stage does the fixed-arity stage's
    arithmetic in the same order: stages 2 and 3 agree bit for bit."""
    from oracle.rhs import rhs
    case = Case(3, 4, 2, 4, 60e3, 80e3, 5e3, n_bv=0.01)
    g = ctx(pkg, case, case.dt_for(15.0), scheme=scheme)
    q0 = case.state(9)
    R1 = rhs(case.mesh, case.col, q0)
    d0, dR1 = dev(torch, q0), dev(torch, R1)
    q2 = g.imex_stage(2, d0, dR1)
    assert torch.equal(g.imex_stage_s(2, d0, [dR1]), q2)
    dR2 = dev(torch, rhs(case.mesh, case.col, q2.cpu().numpy()))
    q3 = g.imex_stage(3, d0, dR1, dR2, q2)
    assert torch.equal(g.imex_stage_s(3, d0, [dR1, dR2], [q2]), q3)


@pytest.mark.parametrize("scheme,C,L,nsteps,N", [
    ("ark4", 15, 400e3, 4, 4), ("ark4", 150, 4000e3, 3, 4), ("ark4", 15, 300e3, 2, 3),
    ("ark5", 15, 400e3, 3, 4), ("ark5", 150, 4000e3, 2, 4), ("ark5", 15, 300e3, 2, 7)])
def test_run_matches_oracle(pkg, torch, scheme, C, L, nsteps, N):
    from oracle import ark2
    case = Case(4, 3, 3, N, L, 0.75 * L, 10e3, n_bv=0.01)
    dt = case.dt_for(C)
    q0 = case.state(52, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt, scheme=scheme).step(q0, nsteps)
    assert np.isfinite(ref).all()
    g = ctx(pkg, case, dt, scheme=scheme)
    assert g.query(pkg.Q_SCHEME) == pkg.SCHEMES[scheme]
    qg = dev(torch, q0)
    out = g.step_imex1d(qg, g.empty_state(), nsteps).cpu().numpy()
    assert np.all(rel_l2(out, ref) <= RUN_TOL), rel_l2(out, ref)
    g.step_imex1d(qg, None, nsteps)                       # in place: the same bits
    np.testing.assert_array_equal(qg.cpu().numpy(), out)


def test_higher_order_schemes_converge_faster(pkg, torch):
    """With the vertical acoustic modes resolved (C = 2 and 1), against an ARK5 run at a
    sixteenth of the step: the errors order ARK5 < ARK4 < ARK3 at C = 1, and ARK4 and
    ARK5 fall at rates above 3.4 and 4.2 when the step halves."""
    case = Case(2, 2, 3, 4, 400e3, 400e3, 10e3, n_bv=0.01)
    T = 16 * case.dt_for(1.0)
    q0 = dev(torch, case.state(61, kind="balanced"))

    def run(scheme, n):
        return ctx(pkg, case, T / n, scheme=scheme).step_imex1d(q0.clone(), None, n)

    ref = run("ark5", 128)
    err = {(s, n): float((run(s, n) - ref)[3].norm() / ref[3].norm())
           for s in ("ark3", "ark4", "ark5") for n in (8, 16)}
    assert err[("ark5", 16)] < err[("ark4", 16)] < err[("ark3", 16)], err
    assert np.log2(err[("ark4", 8)] / err[("ark4", 16)]) > 3.4, err
    assert np.log2(err[("ark5", 8)] / err[("ark5", 16)]) > 4.2, err


def test_ark45_rejections(pkg, torch):
    case = Case(2, 2, 2, 4, 4e3, 4e3, 4e3)
    for kw in ({"precision": "mixed"}, {"column_form": "standard"}, {"imex": "3d"}):
        with pytest.raises(pkg.NumaError):
            ctx(pkg, case, 1.0, scheme="ark4", **kw)
    g = ctx(pkg, case, case.dt_for(15.0), scheme="ark5")
    q = dev(torch, case.state(1))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.imex_stage_s(9, q, [q] * 8, [q] * 7)
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.rhs_adjoint(q, q)
