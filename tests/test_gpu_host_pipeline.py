"""numa_run_host with host buffers: the FP64 ARK2 path overlaps the upload with the first
right-hand side and the download with the final update, slab by slab (runs of whole tile
rows of the right-hand side's thread order).  The result must be bit for bit the device
path's: the same kernels do the same arithmetic for every node, only the launch order
changes.
"""
import numpy as np
import pytest

from helpers import Case

pytestmark = pytest.mark.gpu


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


# one tile row (a single slab); ten tile rows in eight uneven slabs; six rows of N = 3
MESHES = [(4, 4, 4, 4, 40e3), (4, 40, 3, 4, 400e3), (3, 23, 2, 3, 300e3)]


@pytest.mark.parametrize("mesh", MESHES)
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_host_run_equals_the_device_run_bitwise(pkg, torch, mesh, nsteps):
    nex, ney, nez, N, L = mesh
    case = Case(nex, ney, nez, N, L, L * ney / nex, 10e3, n_bv=0.01)
    dt = case.dt_for(15.0)
    q0 = case.state(71, kind="balanced")
    g = ctx(pkg, case, dt)
    ref = g.step_imex1d(torch.from_numpy(q0).cuda(), None, nsteps).cpu()
    qin = torch.from_numpy(q0.copy()).pin_memory()
    qout = torch.empty_like(qin).pin_memory()
    g.run_host(0, qin, nsteps, 0.0, qout)
    assert torch.equal(qout, ref)
    assert torch.equal(qin, torch.from_numpy(q0))            # input untouched
    g.run_host(0, qin, nsteps)                               # in place on the host buffer
    assert torch.equal(qin, ref)
    g.run_host(0, qin, 0)                                    # zero steps: a plain copy back
    assert torch.equal(qin, ref)


@pytest.mark.parametrize("precision", ["mixed", "rhs32"])
def test_other_forms_keep_the_plain_host_run(pkg, torch, precision):
    case = Case(4, 8, 3, 4, 80e3, 160e3, 10e3, n_bv=0.01)
    dt = case.dt_for(15.0)
    q0 = case.state(72, kind="balanced")
    g = ctx(pkg, case, dt, precision=precision)
    ref = g.step_imex1d(torch.from_numpy(q0).cuda(), None, 2).cpu()
    qin = torch.from_numpy(q0.copy()).pin_memory()
    g.run_host(0, qin, 2)
    assert torch.equal(qin, ref)


def test_explicit_host_run_is_unchanged(pkg, torch):
    case = Case(4, 8, 3, 4, 80e3, 160e3, 10e3, n_bv=0.01)
    dt = case.dt_for(1.0)
    q0 = case.state(73, kind="balanced")
    g = ctx(pkg, case, case.dt_for(15.0))
    ref = g.step_explicit_rk(torch.from_numpy(q0).cuda(), dt, None, 3).cpu()
    qin = torch.from_numpy(q0.copy()).pin_memory()
    g.run_host(1, qin, 3, dt)
    assert torch.equal(qin, ref)
