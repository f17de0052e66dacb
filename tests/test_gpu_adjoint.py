"""Differentiation form on the GPU (through the C ABI) against the FP64 oracle.

Tolerances: TLM and adjoint right-hand sides, transposed column solves and stage adjoints
relative L2 <= 1e-11 per field (the RHS bar: both sides are short FP64 sums of the same
terms); one step's TLM and adjoint <= 1e-10 per field; a multi-step gradient <= 1e-9 (the
run bar).  Properties at the differentiation workload (16 x 16 x 8 elements, N = 4, 20
steps at C = 15, checkpoints every 5 steps): dot-product identities to 1e-10, centred
finite differences of the misfit with step 1e-6, bitwise independence of the gradient from
the checkpoint interval, and forward-mode AD equal to the TLM kernels.
"""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-11
STEP_TOL = 1e-10
RUN_TOL = 1e-9
DOT_TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_1702_04316_gb300 as p
    p.lib()
    return p


CASES = {
    "tiny4": (4, 4, 4, 4, 10e3, 10e3, 10e3),
    "ragged": (3, 5, 2, 3, 7e3, 9e3, 4e3),
    "n2": (5, 2, 3, 2, 6e3, 3e3, 5e3),
    "n7": (2, 3, 2, 7, 8e3, 9e3, 6e3),
    "single": (1, 1, 1, 4, 2e3, 2e3, 2e3),
}


def make(name, n_bv=0.0):
    nex, ney, nez, N, Lx, Ly, Lz = CASES[name]
    return Case(nex, ney, nez, N, Lx, Ly, Lz, n_bv)


def diff_workload():
    """The differentiation workload: 16 x 16 x 8 elements of order 4 over 600 x 600 x 10
    km (horizontal Courant number 0.5 at vertical C = 15)."""
    return Case(16, 16, 8, 4, 600e3, 600e3, 10e3)


def gpu_ctx(pkg, case, dt=0.0):
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv)


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def dot(a, b):
    return float((a * b).sum())


@pytest.mark.parametrize("name", ["tiny4", "ragged", "n2", "n7", "single"])
def test_rhs_tlm_matches_oracle(torch, pkg, name):
    from oracle.tangent import rhs_tlm
    case = make(name, 0.01)
    q, dq = case.state(1, vel=5.0), case.state(2, vel=3.0)
    g = gpu_ctx(pkg, case)
    out = host(g.rhs_tlm(dev(torch, q), dev(torch, dq)))
    ref = rhs_tlm(case.mesh, case.col, q, dq)
    assert rel_l2(out, ref).max() <= TOL


@pytest.mark.parametrize("name", ["tiny4", "ragged", "n2", "n7", "single"])
def test_rhs_adjoint_matches_oracle(torch, pkg, name):
    from oracle.tangent import rhs_adjoint
    case = make(name, 0.01)
    q, lam = case.state(3, vel=5.0), case.state(4, vel=2.0)
    g = gpu_ctx(pkg, case)
    out = host(g.rhs_adjoint(dev(torch, q), dev(torch, lam)))
    ref = rhs_adjoint(case.mesh, case.col, q, lam)
    assert rel_l2(out, ref).max() <= TOL


def test_rhs_adjoint_is_bitwise_reproducible(torch, pkg):
    case = make("tiny4")
    g = gpu_ctx(pkg, case)
    q, lam = dev(torch, case.state(5, vel=5.0)), dev(torch, case.state(6))
    a = g.rhs_adjoint(q, lam)
    b = g.rhs_adjoint(q, lam)
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["tiny4", "ragged", "n2", "n7"])
def test_transposed_column_solve_matches_oracle(torch, pkg, name):
    from oracle.column import lu_nopivot_banded
    from oracle.tangent import lu_solve_transposed_banded
    case = make(name, 0.012)
    dt = case.dt_for(15.0)
    g = gpu_ctx(pkg, case, dt)
    lam = (1.0 - 1.0 / np.sqrt(2.0)) * dt
    LU = lu_nopivot_banded(case.col.jacobian_by_probing(lam), case.col.half_band)
    b = np.random.default_rng(7).standard_normal((case.mesh.ncol, case.mesh.M))
    out = host(g.solve_columns_transposed(dev(torch, b.ravel()))).reshape(b.shape)
    ref = lu_solve_transposed_banded(LU, case.col.half_band, b)
    assert np.linalg.norm(out - ref) <= TOL * np.linalg.norm(ref)
    # and S^T (S^-T b) = b through the forward solve's transpose identity
    y = dev(torch, np.random.default_rng(8).standard_normal(b.size))
    x = g.solve_columns(dev(torch, b.ravel()))
    xt = g.solve_columns_transposed(y)
    assert abs(dot(y, x) - dot(xt, dev(torch, b.ravel()))) <= 1e-12 * abs(dot(y, x))


@pytest.mark.parametrize("stage", [2, 3])
@pytest.mark.parametrize("name", ["tiny4", "ragged", "n7"])
def test_stage_adjoint_matches_oracle(torch, pkg, name, stage):
    from oracle.ark2 import HEVI
    from oracle.tangent import ColumnMap, stage_adjoint
    case = make(name, 0.01)
    dt = case.dt_for(15.0)
    g = gpu_ctx(pkg, case, dt)
    h = HEVI(case.mesh, case.col, dt)
    lam = case.state(9, vel=2.0)
    z = [torch.zeros(5, case.mesh.nnode, dtype=torch.float64, device="cuda") for _ in range(4)]
    g.imex_stage_adjoint(stage, dev(torch, lam), z[0], z[1], z[2] if stage == 3 else None,
                         z[3] if stage == 3 else None)
    cm = ColumnMap(h)
    qa, Ra, Qa = stage_adjoint(h, stage - 1, lam, cm)
    # q^n* = (1 + c_i1) q~_e* - c_i1 lam with c_21 = -1 (to rounding): the two terms cancel
    # for stage 2, so the error is measured against the size of q~_e* = solve^T(lam), the
    # scale of the rounding in either evaluation order.
    scale = np.maximum(np.linalg.norm(qa, axis=1), np.linalg.norm(cm.apply_T(lam), axis=1))
    assert (np.linalg.norm(host(z[0]) - qa, axis=1) <= TOL * scale).all()
    assert rel_l2(host(z[1]), Ra[0]).max() <= TOL
    if stage == 3:
        assert rel_l2(host(z[2]), Ra[1]).max() <= TOL
        assert rel_l2(host(z[3]), Qa[1]).max() <= TOL


@pytest.mark.parametrize("stage", [2, 3])
def test_stage_adjoint_dot_product(torch, pkg, stage):
    """The stage is linear in (q^n, R1, R2, q(2)): <lam, stage(x)> = <stage^T lam, x>."""
    case = make("ragged", 0.01)
    g = gpu_ctx(pkg, case, case.dt_for(15.0))
    x = [dev(torch, case.state(20 + k, vel=3.0)) for k in range(4)]
    lam = dev(torch, case.state(30, vel=2.0))
    out = g.imex_stage(stage, x[0], x[1], x[2] if stage == 3 else None,
                       x[3] if stage == 3 else None)
    z = [torch.zeros_like(lam) for _ in range(4)]
    g.imex_stage_adjoint(stage, lam, z[0], z[1], z[2], z[3])
    lhs = dot(lam, out)
    rhs = sum(dot(z[k], x[k]) for k in range(4 if stage == 3 else 2))
    assert abs(lhs - rhs) <= DOT_TOL * abs(lhs)


@pytest.mark.parametrize("name", ["tiny4", "ragged"])
def test_step_tlm_and_adjoint_match_oracle(torch, pkg, name):
    from oracle.ark2 import HEVI
    from oracle.tangent import step_adjoint, step_tlm
    case = make(name, 0.01)
    dt = case.dt_for(15.0)
    g = gpu_ctx(pkg, case, dt)
    h = HEVI(case.mesh, case.col, dt)
    q, dq, lam = case.state(1, vel=5.0), case.state(2, vel=3.0), case.state(3, vel=2.0)
    q1, dq1 = g.step_imex1d_tlm(dev(torch, q), dev(torch, dq))
    rq1, rdq1 = step_tlm(h, q, dq)
    assert rel_l2(host(q1), rq1).max() <= STEP_TOL
    assert rel_l2(host(dq1), rdq1).max() <= STEP_TOL
    la = host(g.step_imex1d_adjoint(dev(torch, q), dev(torch, lam)))
    assert rel_l2(la, step_adjoint(h, q, lam)).max() <= STEP_TOL


def test_gradient_matches_oracle_over_several_steps(torch, pkg):
    from oracle.ark2 import HEVI
    from oracle.tangent import gradient
    case = Case(3, 2, 2, 4, 240e3, 160e3, 8e3, n_bv=0.01)
    dt = case.dt_for(15.0)
    g = gpu_ctx(pkg, case, dt)
    h = HEVI(case.mesh, case.col, dt)
    q0 = case.state(1, vel=3.0)
    target = case.state(2)[4]
    J, grad = gradient(h, q0, target, 6)
    x = dev(torch, q0).requires_grad_(True)
    qT = g.trajectory(x, 6, every=4)
    Jg = 0.5 * ((qT[4] - dev(torch, target)) ** 2).sum()
    Jg.backward()
    assert float(Jg.detach()) == pytest.approx(J, rel=1e-12)
    assert rel_l2(host(x.grad), grad).max() <= RUN_TOL


# ---- the differentiation workload ----------------------------------------------------------
@pytest.fixture(scope="module")
def dw(torch, pkg):
    case = diff_workload()
    g = gpu_ctx(pkg, case, case.dt_for(15.0))
    q0 = dev(torch, case.state(11, vel=5.0))
    target = dev(torch, case.state(12)[4])
    return case, g, q0, target


def _misfit(torch, g, q, target, nsteps=20, every=5):
    qT = g.trajectory(q, nsteps, every)
    return 0.5 * ((qT[4] - target) ** 2).sum()


def test_diff_workload_rhs_tlm_and_adjoint_match_oracle(torch, pkg, dw):
    from oracle.tangent import rhs_adjoint, rhs_tlm
    case, g, q0, _ = dw
    q = host(q0)
    dq, lam = case.state(13, vel=3.0), case.state(14, vel=2.0)
    assert rel_l2(host(g.rhs_tlm(q0, dev(torch, dq))), rhs_tlm(case.mesh, case.col, q, dq)).max() <= TOL
    assert rel_l2(host(g.rhs_adjoint(q0, dev(torch, lam))),
                  rhs_adjoint(case.mesh, case.col, q, lam)).max() <= TOL


def test_diff_workload_dot_product_of_the_run(torch, pkg, dw):
    case, g, q0, _ = dw
    dq = dev(torch, case.state(15, vel=3.0))
    lam = dev(torch, case.state(16, vel=2.0))
    _, dqT = g.step_imex1d_tlm(q0, dq, 20)
    qT, ckpt = g.forward_checkpointed(q0, 20, 5)
    lam0 = g.adjoint_checkpointed(ckpt, 20, 5, lam)
    a, b = dot(lam, dqT), dot(lam0, dq)
    assert abs(a - b) <= DOT_TOL * abs(a)
    assert g.count_nonfinite(qT) == 0
    assert g.status() == pkg.NUMA_OK


def test_diff_workload_gradient_matches_centred_differences(torch, pkg, dw):
    case, g, q0, target = dw
    x = q0.clone().requires_grad_(True)
    J = _misfit(torch, g, x, target)
    J.backward()
    grad = x.grad
    eps = 1e-6
    with torch.no_grad():
        for seed in (17, 18):
            d = dev(torch, case.state(seed, vel=3.0))
            fd = (float(_misfit(torch, g, q0 + eps * d, target))
                  - float(_misfit(torch, g, q0 - eps * d, target))) / (2 * eps)
            ad = dot(grad, d)
            assert abs(fd - ad) <= 1e-6 * abs(ad)


def test_diff_workload_gradient_does_not_depend_on_the_checkpoint_interval(torch, pkg, dw):
    case, g, q0, target = dw
    grads = []
    for every in (1, 5, 7, 20):
        x = q0.clone().requires_grad_(True)
        _misfit(torch, g, x, target, 20, every).backward()
        grads.append(x.grad)
    for gr in grads[1:]:
        assert torch.equal(gr, grads[0])


def test_forward_mode_matches_the_tlm_kernels(torch, pkg, dw):
    import torch.autograd.forward_ad as fwAD
    case, g, q0, _ = dw
    dq = dev(torch, case.state(19, vel=3.0))
    with fwAD.dual_level():
        out = g.rhs_autograd(fwAD.make_dual(q0, dq))
        t_rhs = fwAD.unpack_dual(out).tangent
        qT = g.trajectory(fwAD.make_dual(q0, dq), 3, 1)
        t_run = fwAD.unpack_dual(qT).tangent
    assert torch.equal(t_rhs, g.rhs_tlm(q0, dq))
    assert torch.equal(t_run, g.step_imex1d_tlm(q0, dq, 3)[1])


def test_rhs_autograd_backward_is_the_adjoint(torch, pkg, dw):
    case, g, q0, _ = dw
    lam = dev(torch, case.state(21, vel=2.0))
    x = q0.clone().requires_grad_(True)
    (g.rhs_autograd(x) * lam).sum().backward()
    assert torch.equal(x.grad, g.rhs_adjoint(q0, lam))


def test_differentiation_needs_an_fp64_context(torch, pkg):
    case = make("tiny4")
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    g = pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, case.dt_for(15.0), precision="mixed")
    q = dev(torch, case.state(1))
    with pytest.raises(pkg.NumaError):
        g.rhs_adjoint(q, q)
