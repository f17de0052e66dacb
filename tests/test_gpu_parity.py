"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: integer connectivity bit-exact; explicit RHS relative L2 <= 1e-11 per field;
factors, solves and single stages <= 1e-11; states after full steps <= 1e-9 per field.
"""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-11
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


def gpu_ctx(pkg, case, dt=0.0):
    nex, ney, nez, Lx, Ly, Lz, N = case.args
    return pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt, 300.0, case.n_bv)


CASES = {
    "tiny4": (4, 4, 4, 4, 10e3, 10e3, 10e3),          # 4 x 4 x 4 elements, N = 4, 10 km box
    "ragged": (3, 5, 2, 3, 7e3, 9e3, 4e3),
    "n2": (5, 2, 3, 2, 6e3, 3e3, 5e3),
    "n7": (2, 3, 2, 7, 8e3, 9e3, 6e3),
    "n8": (2, 2, 2, 8, 4e3, 4e3, 4e3),
    "n1": (6, 5, 4, 1, 6e3, 5e3, 4e3),
    "single": (1, 1, 1, 4, 2e3, 2e3, 2e3),
}


def make(name, n_bv=0.0):
    nex, ney, nez, N, Lx, Ly, Lz = CASES[name]
    return Case(nex, ney, nez, N, Lx, Ly, Lz, n_bv)


@pytest.mark.parametrize("name", ["tiny4", "ragged", "n2", "n7", "single"])
def test_connectivity_bit_exact(pkg, name):
    case = make(name)
    g = gpu_ctx(pkg, case)
    l2g, g2l = g.connectivity()
    ref = case.mesh.l2g()
    np.testing.assert_array_equal(l2g.cpu().numpy().astype(np.int64), ref)
    # inverse map from the oracle's l2g
    flat = ref.ravel()
    order = np.argsort(flat, kind="stable")
    inv = -np.ones((case.mesh.nnode, 8), dtype=np.int64)
    counts = np.zeros(case.mesh.nnode, dtype=np.int64)
    for lid in order:
        gid = flat[lid]
        inv[gid, counts[gid]] = lid
        counts[gid] += 1
    # (a stable argsort leaves each node's local ids ascending, padded with -1)
    np.testing.assert_array_equal(g2l.cpu().numpy().astype(np.int64), inv)


@pytest.mark.parametrize("n_bv", [0.0, 0.015])
def test_reference_levels(pkg, n_bv):
    case = make("tiny4", n_bv)
    g = gpu_ctx(pkg, case)
    lev = g.reference_levels()
    c = case.col
    for key, ref in (("z", c.z), ("rho0", c.rho0), ("theta0", c.theta0), ("P0", c.P0),
                     ("G0", c.G0), ("H0", c.H0), ("drho0", c.drho0)):
        np.testing.assert_allclose(lev[key], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(lev["dtheta0"], c.dtheta0, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(pkg, torch, name):
    from oracle.rhs import rhs
    case = make(name, 0.01 if name == "ragged" else 0.0)
    g = gpu_ctx(pkg, case)
    q0 = case.state(100 + len(name))
    r = g.rhs_explicit(torch.from_numpy(q0).cuda()).cpu().numpy()
    e = rel_l2(r, rhs(case.mesh, case.col, q0))
    assert np.all(e <= RHS_TOL), e


def test_rhs_rest_state_is_exactly_zero(pkg, torch):
    case = make("tiny4")
    g = gpu_ctx(pkg, case)
    r = g.rhs_explicit(torch.zeros(5, case.mesh.nnode, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(r).item() == 0


@pytest.mark.parametrize("C", [1, 15, 150])
@pytest.mark.parametrize("name,n_bv", [("tiny4", 0.0), ("ragged", 0.02), ("n7", 0.0), ("n1", 0.0)])
def test_factors_and_solve(pkg, torch, name, n_bv, C):
    from oracle.column import lu_nopivot_banded, lu_solve_banded
    case = make(name, n_bv)
    dt = case.dt_for(C)
    g = gpu_ctx(pkg, case, dt)
    col = case.col
    lam = (1 - 1 / np.sqrt(2)) * dt
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    hb, M = col.half_band, case.mesh.M
    band = np.zeros((M, 2 * hb + 1))
    for i in range(M):
        for j in range(max(0, i - hb), min(M, i + hb + 1)):
            band[i, j - i + hb] = LU[i, j]
    ncol = case.mesh.ncol
    for c in sorted({0, ncol // 2, ncol - 1}):
        fac = g.column_factors(c)
        np.testing.assert_allclose(fac, band, rtol=0, atol=1e-12 * np.abs(band).max())
    b = np.random.default_rng(C).standard_normal((ncol, M))
    x = g.solve_columns(torch.from_numpy(b.ravel()).cuda()).cpu().numpy().reshape(ncol, M)
    xr = lu_solve_banded(LU, hb, b)
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.norm(xr)
    # in place
    bt = torch.from_numpy(b.ravel()).cuda()
    g.solve_columns(bt, bt)
    assert np.linalg.norm(bt.cpu().numpy().reshape(ncol, M) - xr) <= 1e-12 * np.linalg.norm(xr)
    assert g.status() == pkg.NUMA_OK


_SOLVE_SCRIPT = r"""
import hashlib, sys, torch
import paper_1702_04316_gb300 as pkg
nex, ney, nez, N = (int(v) for v in sys.argv[1:5])
g = pkg.Numa(nex, ney, nez, 2e3 * nex, 2e3 * ney, 1.25e3 * nez, N, 9.32)
nn = g.ncol * g.M
gen = torch.Generator(device="cuda").manual_seed(5)
b = torch.randn(nn, dtype=torch.float64, device="cuda", generator=gen)
x = g.solve_columns(b)
assert g.status() == pkg.NUMA_OK
print(hashlib.sha1(x.cpu().numpy().tobytes()).hexdigest())
"""


@pytest.mark.parametrize("mesh", [(4, 4, 4, 4), (3, 5, 2, 3), (2, 3, 2, 7), (21, 19, 6, 4)])
def test_bulk_copy_solve_equals_register_solve(mesh):
    """The stand-alone solve stages its factor stream with bulk (TMA) copies; with
    NUMA_SOLVE=regs it runs the register-pipelined kernel instead.  Both do the same
    arithmetic in the same order, so the solutions agree bit for bit (ragged last blocks of
    32 columns included: 3 x 5 x 2 at N = 3 has 16 x 10 columns)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for mode in ("", "regs"):
        env = dict(os.environ, NUMA_SOLVE=mode, PYTHONPATH=root)
        r = subprocess.run([sys.executable, "-c", _SOLVE_SCRIPT] + [str(v) for v in mesh],
                           env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out[mode] = r.stdout.strip()
    assert out[""] == out["regs"]


def test_bulk_copy_solve_unaligned_buffers(pkg, torch):
    """Buffers that are 8- but not 16-byte aligned take plain loads and stores for the
    right-hand side and the solution; the result bits do not change."""
    case = make("tiny4")
    g = gpu_ctx(pkg, case, case.dt_for(15))
    nn = case.mesh.ncol * case.mesh.M
    b = torch.randn(nn, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(3))
    x = g.solve_columns(b)
    bu = torch.empty(nn + 1, dtype=torch.float64, device="cuda")[1:]
    xu = torch.empty(nn + 1, dtype=torch.float64, device="cuda")[1:]
    bu.copy_(b)
    g.solve_columns(bu, xu)
    assert torch.equal(xu, x)
    g.solve_columns(bu, bu)                          # in place, unaligned
    assert torch.equal(bu, x)
    assert g.status() == pkg.NUMA_OK


def test_bulk_copy_solve_is_repeatable(pkg, torch):
    """Twenty solves of one right-hand side give the same bits (the shared-memory ring of
    factor rows is refilled while other warps stream: a refill that overtook a read would
    show here).  N = 7, 169 x 169 columns of 43 levels, half-band 14."""
    case = Case(24, 24, 6, 7, 48e3, 48e3, 7.5e3)
    g = gpu_ctx(pkg, case, case.dt_for(15))
    nn = case.mesh.ncol * case.mesh.M
    b = torch.randn(nn, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(4))
    x0 = g.solve_columns(b)
    x = torch.empty_like(b)
    for _ in range(20):
        g.solve_columns(b, x)
        assert torch.equal(x, x0)
    assert g.status() == pkg.NUMA_OK


@pytest.mark.parametrize("C", [15, 150])
def test_imex_stages(pkg, torch, C):
    """Rows 2 and 3 of Table 1 on their own, inputs from the oracle."""
    from oracle import ark2
    from oracle.column import implicit_solve, lu_nopivot_banded
    from oracle.rhs import rhs
    case = make("ragged", 0.02)
    dt = case.dt_for(C)
    g = gpu_ctx(pkg, case, dt)
    m, col = case.mesh, case.col
    a, at, b, _ = ark2.tableau()
    lam = at[1, 1] * dt
    LU = lu_nopivot_banded(col.jacobian_by_probing(lam), col.half_band)
    q0 = case.state(7)
    R1 = rhs(m, col, q0)

    def stage_ref(i, Q, Rs):
        cij = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        q_e = q0 + dt * sum(a[i, j] * Rs[j] for j in range(i))
        qtt_e = q_e + sum(cij[j] * Q[j] for j in range(i))
        qtt = implicit_solve(col, LU, qtt_e.reshape(5, m.ncol, m.M), lam).reshape(5, -1)
        return qtt - sum(cij[j] * Q[j] for j in range(i))

    q2 = stage_ref(1, [q0], [R1])
    R2 = rhs(m, col, q2)
    q3 = stage_ref(2, [q0, q2], [R1, R2])
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g2 = g.imex_stage(2, T(q0), T(R1)).cpu().numpy()
    assert np.all(rel_l2(g2, q2) <= RHS_TOL), rel_l2(g2, q2)
    g3 = g.imex_stage(3, T(q0), T(R1), T(R2), T(q2)).cpu().numpy()
    assert np.all(rel_l2(g3, q3) <= RHS_TOL), rel_l2(g3, q3)


@pytest.mark.parametrize("label,dims,C,nsteps,n_bv", [
    ("tiny4-C15-1step", (4, 4, 4, 4, 10e3, 10e3, 10e3), 15, 1, 0.0),
    ("tiny4-C1-10steps", (4, 4, 4, 4, 10e3, 10e3, 10e3), 1, 10, 0.0),
    ("wide-C15-10steps", (4, 4, 4, 4, 300e3, 300e3, 10e3), 15, 10, 0.0),
    ("wide-C150-10steps", (4, 4, 4, 4, 3000e3, 3000e3, 10e3), 150, 10, 0.0),
    ("wide-stratified-C15", (3, 4, 5, 4, 300e3, 400e3, 10e3), 15, 5, 0.012),
])
def test_imex_run_parity(pkg, torch, label, dims, C, nsteps, n_bv):
    from oracle import ark2
    nex, ney, nez, N, Lx, Ly, Lz = dims
    case = Case(nex, ney, nez, N, Lx, Ly, Lz, n_bv)
    dt = case.dt_for(C)
    q0 = case.state(31, kind="balanced")
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, nsteps)
    assert np.isfinite(ref).all()
    g = gpu_ctx(pkg, case, dt)
    qg = torch.from_numpy(q0).cuda()
    out = g.step_imex1d(qg, g.empty_state(), nsteps).cpu().numpy()
    e = rel_l2(out, ref)
    assert np.all(e <= RUN_TOL), (label, e)
    # in place gives the same bits
    g.step_imex1d(qg, None, nsteps)
    np.testing.assert_array_equal(qg.cpu().numpy(), out)


def test_rk35_run_parity(pkg, torch):
    from oracle import rk35
    case = make("tiny4")
    dt = case.dt_for(1.0)
    q0 = case.state(5, kind="balanced")
    ref = rk35.Explicit(case.mesh, case.col).step(q0, dt, 10)
    g = gpu_ctx(pkg, case)
    out = g.step_explicit_rk(torch.from_numpy(q0).cuda(), dt, g.empty_state(), 10).cpu().numpy()
    e = rel_l2(out, ref)
    assert np.all(e <= RUN_TOL), e


def test_zero_steps_and_errors(pkg, torch):
    case = make("n2")
    g = gpu_ctx(pkg, case)              # dt = 0: not factored
    q = torch.from_numpy(case.state(3)).cuda()
    with pytest.raises(pkg.NumaError, match="NOT_FACTORED"):
        g.step_imex1d(q, g.empty_state(), 1)
    with pytest.raises(pkg.NumaError, match="NOT_FACTORED"):
        g.solve_columns(torch.zeros(case.mesh.ncol * case.mesh.M, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.factor_columns(-1.0)
    g.factor_columns(case.dt_for(15))
    out = g.step_imex1d(q, g.empty_state(), 0)
    assert torch.equal(out, q)
    out = g.step_explicit_rk(q, 1.0, g.empty_state(), 0)
    assert torch.equal(out, q)
    with pytest.raises(pkg.NumaError, match="ERR_ARG"):
        g.rhs_explicit(q, q)
    bad = q.clone()
    bad[2, 17] = float("nan")
    bad[4, 3] = float("inf")
    assert g.count_nonfinite(bad) == 2
    assert g.count_nonfinite(q) == 0


def test_host_buffer_driver(pkg, torch):
    from oracle import ark2
    case = make("tiny4")
    dt = case.dt_for(15)
    q0 = case.state(9, kind="balanced")
    g = gpu_ctx(pkg, case, dt)
    qh = torch.from_numpy(q0.copy()).pin_memory()
    g.run_host(0, qh, 1)
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, 1)
    assert np.all(rel_l2(qh.numpy(), ref) <= RUN_TOL)


def test_stage_rejects_an_output_overlapping_an_input():
    """The fused stage parks intermediate values in its output, so numa_imex_stage and
    numa_imex_stage_s refuse an output that overlaps an input."""
    import torch
    import paper_1702_04316_gb300 as pkg
    g = pkg.Numa(3, 3, 2, 30e3, 30e3, 8e3, 3, 1.0)
    q = torch.zeros(5, g.nnode, dtype=torch.float64, device="cuda")
    R1 = torch.zeros_like(q)
    with pytest.raises(pkg.NumaError):
        g.imex_stage(2, q, R1, out=q)
    with pytest.raises(pkg.NumaError):
        g.imex_stage(2, q, R1, out=R1)
    g.close()
