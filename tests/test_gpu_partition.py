"""The partitioned HEVI step on one GPU: several partitions of one mesh held in one process
(paper_1702_04316_gb300.partition.step_partitions with local_exchange), which runs the
library's phased step (numa_step_phase), its halo gather / scatter kernels and the
partition plan exactly as a multi-GPU run does, with the messages copied on the device
instead of sent.  Every owned node must equal the single-context step bit for bit: the
same kernels do the same arithmetic per node and per column.  No kernel of one partition
waits for another's: the partitions run one after the other on one stream."""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu


def _partitioned(pkg, dims, dt, q0, px, py, nsteps, **kw):
    import torch
    from paper_1702_04316_gb300.partition import PartitionedHEVI, local_exchange, step_partitions
    nex, ney, nez, N, Lx, Ly, Lz = dims
    parts = [PartitionedHEVI(nex, ney, nez, Lx, Ly, Lz, N, dt, px, py, r, **kw)
             for r in range(px * py)]
    qg = torch.from_numpy(q0).cuda()
    q_in = [p.restrict(qg) for p in parts]
    q_out = [torch.empty_like(q) for q in q_in]
    step_partitions(parts, q_in, q_out, nsteps, lambda fl: local_exchange(parts, fl))
    out = torch.full((5, ney * N + 1, nex * N + 1, nez * N + 1), float("nan"),
                     dtype=torch.float64, device="cuda")
    for p, qo in zip(parts, q_out):
        _, (gy, gx) = p.owned_slices()
        out[:, gy, gx, :] = p.owned(qo)
        assert p.ctx.status() == pkg.NUMA_OK
        p.close()
    return out.reshape(5, -1)


@pytest.mark.parametrize("px,py", [(2, 1), (1, 3), (2, 2), (3, 2)])
def test_partitioned_steps_equal_the_single_context(px, py):
    import torch
    import paper_1702_04316_gb300 as pkg
    from oracle import ark2
    dims = (8, 6, 2, 3, 1600e3, 1200e3, 8e3)       # C_H = 0.3 at C_V = 15: bounded
    case = Case(*dims[:3], dims[3], *dims[4:])
    dt = case.dt_for(15.0)
    q0 = case.state(616)
    got = _partitioned(pkg, dims, dt, q0, px, py, 3)
    assert not torch.isnan(got).any()
    g = pkg.Numa(*dims[:3], *dims[4:], dims[3], dt)
    ref = g.step_imex1d(torch.from_numpy(q0).cuda(), g.empty_state(), 3)
    g.close()
    assert torch.equal(got, ref)
    e = rel_l2(got.cpu().numpy(), ark2.HEVI(case.mesh, case.col, dt).step(q0, 3))
    assert np.all(e <= 1e-9), e


@pytest.mark.parametrize("precision", ["mixed", "rhs32"])
def test_partitioned_precision_forms(precision):
    """The forms without a fused P' (the next right-hand side recomputes it): only the five
    state fields cross the cut."""
    import torch
    import paper_1702_04316_gb300 as pkg
    dims = (6, 4, 2, 4, 1200e3, 800e3, 8e3)
    case = Case(*dims[:3], dims[3], *dims[4:])
    dt = case.dt_for(15.0)
    q0 = case.state(617)
    got = _partitioned(pkg, dims, dt, q0, 2, 2, 2, precision=precision)
    g = pkg.Numa(*dims[:3], *dims[4:], dims[3], dt, precision=precision)
    ref = g.step_imex1d(torch.from_numpy(q0).cuda(), g.empty_state(), 2)
    g.close()
    assert torch.equal(got, ref)


def test_partitioned_step_at_full_size():
    """The 96 x 96 x 12 workload (N = 4) on a 2 x 2 partition, one step at C = 15: every
    owned node equals the single-context step bit for bit."""
    import torch
    import paper_1702_04316_gb300 as pkg
    dims = (96, 96, 12, 4, 200e3, 200e3, 15e3)
    case = Case(*dims[:3], dims[3], *dims[4:])
    dt = case.dt_for(15.0)
    q0 = case.state(2001, kind="balanced")
    got = _partitioned(pkg, dims, dt, q0, 2, 2, 1)
    g = pkg.Numa(*dims[:3], *dims[4:], dims[3], dt)
    ref = g.step_imex1d(torch.from_numpy(q0).cuda(), g.empty_state(), 1)
    g.close()
    assert torch.equal(got, ref)


def test_gather_scatter_columns():
    import torch
    import paper_1702_04316_gb300 as pkg
    g = pkg.Numa(3, 2, 2, 30e3, 20e3, 8e3, 3, 0.0)
    M, ncol = g.M, g.ncol
    q = torch.randn(5, g.nnode, dtype=torch.float64, device="cuda")
    pp = torch.randn(g.nnode, dtype=torch.float64, device="cuda")
    cols = torch.tensor([7, 0, ncol - 1, 12, 7], dtype=torch.int32, device="cuda")
    fields = [q[f] for f in range(5)] + [pp]
    buf = torch.empty(6 * cols.numel() * M, dtype=torch.float64, device="cuda")
    g.gather_columns(fields, cols, buf)
    ref = torch.stack([f.view(ncol, M)[cols.long()] for f in fields]).reshape(-1)
    assert torch.equal(buf, ref)
    tgt = [torch.zeros_like(f) for f in fields]
    uniq = torch.tensor([3, 9, 1], dtype=torch.int32, device="cuda")
    b2 = torch.randn(6 * 3 * M, dtype=torch.float64, device="cuda")
    g.scatter_columns(tgt, uniq, b2)
    for i, f in enumerate(tgt):
        assert torch.equal(f.view(ncol, M)[uniq.long()], b2.view(6, 3, M)[i])
        assert torch.count_nonzero(f).item() == torch.count_nonzero(b2.view(6, 3, M)[i]).item()
    assert g.status() == pkg.NUMA_OK
    # a column id outside the context is skipped and reported, not accessed
    bad = torch.tensor([1, ncol, -1], dtype=torch.int32, device="cuda")
    g.gather_columns(fields, bad, buf[:6 * 3 * M])
    assert g.status() == pkg.NUMA_ERR_ARG
    assert torch.equal(buf[:M], fields[0].view(ncol, M)[1])
    g.close()


def test_phased_step_rejects_what_it_cannot_run():
    import torch
    import paper_1702_04316_gb300 as pkg
    g = pkg.Numa(3, 3, 2, 30e3, 30e3, 8e3, 3, 1.0, scheme="ark3")
    q = torch.zeros(5, g.nnode, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.NumaError):
        g.step_phase(0, q)
    g.close()
    g = pkg.Numa(3, 3, 2, 30e3, 30e3, 8e3, 3, 1.0)
    q2, _, _, _ = g.step_buffers()
    with pytest.raises(pkg.NumaError):      # the input may not be a stage buffer
        g.step_phase(0, q2)
    with pytest.raises(pkg.NumaError):
        g.step_phase(3, q)
    g.close()
