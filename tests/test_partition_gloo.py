"""The partitioned step's host logic on CPU ranks (gloo): the library's partition plan
(numa_part_plan / numa_part_columns, host-only calls of libnuma), the package's halo exchange
(paper_1702_04316_gb300.partition: HaloExchange, step_partitions) and the phase order, with
each rank's window computed by the oracle (the same three phases as numa_step_phase:
R1 and stage 2; R2 and stage 3; the final update).

World sizes 2 (2 x 1) and 4 (2 x 2, which exercises the diagonal neighbours) on 127.0.0.1.
The owned nodes assembled from the ranks must equal the one-rank run (the same driver on a
1 x 1 grid, whose window is the whole mesh) to 1e-12 and the oracle's whole-mesh steps to
1e-9 (relative L2 per field)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (8, 6, 2, 3, 1600e3, 1200e3, 8e3)   # nex, ney, nez, N, Lx, Ly, Lz (C_H = 0.3 at C_V = 15)
NSTEPS = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OraclePartition:
    """One rank's window, computed by the oracle, with the package's halo exchange."""

    def __init__(self, px, py, rank, dist, dt):
        import torch
        from oracle import ark2
        from oracle.column import Column, lu_nopivot_banded
        from oracle.mesh import BoxMesh
        from paper_1702_04316_gb300 import part_plan
        from paper_1702_04316_gb300.partition import HaloExchange
        nex, ney, nez, N, Lx, Ly, Lz = DIMS
        self.torch, self.rank, self.dt, self.N = torch, rank, dt, N
        self.plan = part_plan(nex, ney, nez, Lx, Ly, Lz, N, px, py, rank)
        w = self.plan["window"]
        self.mesh = BoxMesh(w["nex"], w["ney"], nez, N, w["Lx"], w["Ly"], Lz)
        self.col = Column(self.mesh)
        self.a, self.at, self.b, _ = ark2.tableau()
        self.lam = self.at[1, 1] * dt
        self.LU = lu_nopivot_banded(self.col.jacobian_by_probing(self.lam), self.col.half_band)
        self.l2g = self.mesh.l2g()
        self.mass = self.mesh.global_mass(self.l2g)
        self.M = self.mesh.M
        self.halo = HaloExchange(self.plan, self.M, dist, "cpu")
        n = self.mesh.nnode
        self.q2 = torch.zeros(5, n, dtype=torch.float64)
        self.q3 = torch.zeros(5, n, dtype=torch.float64)
        self.R = [None, None, None]

    def _R(self, q):
        from oracle.rhs import rhs
        return rhs(self.mesh, self.col, q.numpy(), self.l2g, self.mass)

    def _stage(self, i, Q):
        from oracle.column import implicit_solve
        a, at, dt = self.a, self.at, self.dt
        c = [(at[i, j] - a[i, j]) / at[i, i] for j in range(i)]
        q_e = Q[0] + dt * sum(a[i, j] * self.R[j] for j in range(i))
        qtt_e = q_e + sum(c[j] * Q[j] for j in range(i))
        qtt = implicit_solve(self.col, self.LU, qtt_e.reshape(5, self.mesh.ncol, self.M),
                             self.lam).reshape(5, -1)
        return qtt - sum(c[j] * Q[j] for j in range(i))

    def phase(self, k, q_n, q_out):
        qn = q_n.numpy()
        if k == 0:
            self.R[0] = self._R(q_n)
            self.q2.copy_(self.torch.from_numpy(self._stage(1, [qn])))
        elif k == 1:
            self.R[1] = self._R(self.q2)
            self.q3.copy_(self.torch.from_numpy(self._stage(2, [qn, self.q2.numpy()])))
        else:
            self.R[2] = self._R(self.q3)
            out = qn + self.dt * sum(self.b[i] * self.R[i] for i in range(3))
            q_out.copy_(self.torch.from_numpy(out))

    def halo_fields(self, k, q_out):
        src = (self.q2, self.q3, q_out)[k]
        return [src[i] for i in range(5)]

    def gather(self, fields, cols, buf):
        idx = cols.long()
        buf.copy_(self.torch.stack([f.view(-1, self.M)[idx] for f in fields]).reshape(-1))

    def scatter(self, fields, cols, buf):
        b = buf.view(len(fields), cols.numel(), self.M)
        idx = cols.long()
        for i, f in enumerate(fields):
            f.view(-1, self.M)[idx] = b[i]

    def restrict(self, qg):
        nex, ney, nez, N = DIMS[:4]
        wx0, wx1, wy0, wy1 = self.plan["window_elems"]
        q = qg.reshape(5, ney * N + 1, nex * N + 1, -1)
        return np.ascontiguousarray(q[:, wy0 * N:wy1 * N + 1, wx0 * N:wx1 * N + 1, :]).reshape(5, -1)

    def owned_global(self, qw):
        """(global y slice, global x slice, owned values (5, ny, nx, M))."""
        N = self.N
        x0, x1, y0, y1 = self.plan["own_cols"]
        wx0, _, wy0, _ = self.plan["window_elems"]
        q = qw.reshape(5, self.mesh.nyg, self.mesh.nxg, self.M)
        return ((wy0 * N + y0, wy0 * N + y1), (wx0 * N + x0, wx0 * N + x1), q[:, y0:y1, x0:x1, :])


def _rank_main(rank, world, px, py, port, q0, dt, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_1702_04316_gb300.partition import step_partitions
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = OraclePartition(px, py, rank, dist, dt)
        qin = torch.from_numpy(p.restrict(q0))
        qout = torch.zeros_like(qin)
        exch = lambda fl: p.halo.exchange(p.gather, p.scatter, fl[0])
        step_partitions([p], [qin], [qout], NSTEPS, exch)
        out[rank] = p.owned_global(qout.numpy())
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(px, py, q0, dt):
    import torch.multiprocessing as mp
    world = px * py
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, px, py, _free_port(), q0, dt, out), nprocs=world,
                 join=True)
        parts = dict(out)
    nex, ney, nez, N = DIMS[:4]
    qg = np.full((5, ney * N + 1, nex * N + 1, nez * N + 1), np.nan)
    for (y0, y1), (x0, x1), v in parts.values():
        assert np.all(np.isnan(qg[:, y0:y1, x0:x1, :]))      # every node owned once
        qg[:, y0:y1, x0:x1, :] = v
    assert not np.isnan(qg).any()
    return qg.reshape(5, -1)


@pytest.fixture(scope="module")
def problem():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import Case
    nex, ney, nez, N, Lx, Ly, Lz = DIMS
    case = Case(nex, ney, nez, N, Lx, Ly, Lz)
    q0 = case.state(515)
    dt = case.dt_for(15.0)
    return case, q0, dt


@pytest.fixture(scope="module")
def one_rank(problem):
    case, q0, dt = problem
    return _run(1, 1, q0, dt)


def test_one_rank_run_is_the_oracle_step(problem, one_rank):
    from oracle import ark2
    from helpers import rel_l2
    case, q0, dt = problem
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, NSTEPS)
    assert np.all(rel_l2(one_rank, ref) <= 1e-13)


@pytest.mark.parametrize("px,py", [(2, 1), (2, 2)])
def test_partitioned_steps_equal_the_one_rank_steps(problem, one_rank, px, py):
    from oracle import ark2
    from helpers import rel_l2
    case, q0, dt = problem
    got = _run(px, py, q0, dt)
    assert np.all(rel_l2(got, one_rank) <= 1e-12), rel_l2(got, one_rank)
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, NSTEPS)
    assert np.all(rel_l2(got, ref) <= 1e-9)


def test_plan_lists_pair_up_and_cover_the_halo():
    """Every halo column of every window is received from exactly one rank, which lists the
    same global columns, in the same order, for sending."""
    from paper_1702_04316_gb300 import part_plan
    nex, ney, nez, N, Lx, Ly, Lz = 13, 9, 2, 4, 1.0, 1.0, 1.0
    px, py = 3, 2
    plans = [part_plan(nex, ney, nez, Lx, Ly, Lz, N, px, py, r) for r in range(px * py)]

    def gid(plan, local):
        wx0, wx1, wy0, _ = plan["window_elems"]
        nxw = (wx1 - wx0) * N + 1
        return (wy0 * N + local // nxw) * (nex * N + 1) + wx0 * N + local % nxw

    owner = np.full((ney * N + 1) * (nex * N + 1), -1)
    for r, p in enumerate(plans):
        x0, x1, y0, y1 = p["own_cols"]
        wx0, wx1, wy0, _ = p["window_elems"]
        for iy in range(y0, y1):
            for ix in range(x0, x1):
                g = (wy0 * N + iy) * (nex * N + 1) + wx0 * N + ix
                assert owner[g] == -1
                owner[g] = r
    assert np.all(owner >= 0)
    for r, p in enumerate(plans):
        wx0, wx1, wy0, wy1 = p["window_elems"]
        nxw, nyw = (wx1 - wx0) * N + 1, (wy1 - wy0) * N + 1
        halo = set()
        for nb in p["neighbours"]:
            g_recv = [gid(p, c) for c in nb["recv"]]
            assert all(owner[g] == nb["rank"] for g in g_recv)
            halo.update(g_recv)
            q = plans[nb["rank"]]
            back = [x for x in q["neighbours"] if x["rank"] == r][0]
            assert [gid(q, c) for c in back["send"]] == g_recv
        window = {gid(p, c) for c in range(nxw * nyw)}
        assert halo == {g for g in window if owner[g] != r}
