"""Several GPUs: the HEVI step on a horizontal partition of the box, with a halo exchange.

In HEVI the implicit column solves cross no partition boundary (Sec. "IMEX time
integration"); the explicit right-hand side reads one element across it, so a partition
needs one halo refresh per right-hand side (the direct stiffness summation across the cut;
Sec. "Scalability").  The library plans the partition (numa_part_plan, numa_part_columns:
rectangles, windows, exchange lists), runs the step in three phases (numa_step_phase) and
packs and unpacks the halo messages (numa_gather_columns, numa_scatter_columns).  This module
only sequences those calls and moves the packed messages with torch.distributed
point-to-point operations (NCCL between GPUs; any backend whose tensors the gather and
scatter callables accept).

A rank's state is its window's state (an ordinary state of the window's context).  Every
owned node of it evolves bit for bit as on the whole mesh.
"""
import numpy as np

from . import Numa, part_plan

# fields refreshed after each phase: q(2) (+ P'), q(3) (+ P'), the step's output
PHASES = (0, 1, 2)


class HaloExchange:
    """The halo messages of one rank: per neighbour, its send and receive column lists (on
    `device`) and message buffers of up to `nf_max` fields of M levels; `exchange` packs,
    swaps the messages with every neighbour in one batch of point-to-point operations, and
    unpacks."""

    def __init__(self, plan, M, dist, device, nf_max=6, dtype=None):
        import torch
        self.torch, self.dist, self.M = torch, dist, M
        dtype = torch.float64 if dtype is None else dtype
        self.peers, self.send_cols, self.recv_cols, self.send_buf, self.recv_buf = [], [], [], [], []
        for nb in plan["neighbours"]:
            self.peers.append(nb["rank"])
            self.send_cols.append(torch.from_numpy(nb["send"]).to(device))
            self.recv_cols.append(torch.from_numpy(nb["recv"]).to(device))
            self.send_buf.append(torch.empty(nf_max * len(nb["send"]) * M, dtype=dtype, device=device))
            self.recv_buf.append(torch.empty(nf_max * len(nb["recv"]) * M, dtype=dtype, device=device))

    def pack(self, gather, fields):
        nf = len(fields)
        for k in range(len(self.peers)):
            gather(fields, self.send_cols[k], self.send_buf[k][:nf * self.send_cols[k].numel() * self.M])

    def unpack(self, scatter, fields):
        nf = len(fields)
        for k in range(len(self.peers)):
            scatter(fields, self.recv_cols[k], self.recv_buf[k][:nf * self.recv_cols[k].numel() * self.M])

    def swap(self, nf):
        """Every neighbour's message in, ours out: one batch of isend / irecv pairs."""
        if not self.peers:
            return
        d = self.dist
        ops = []
        for k, peer in enumerate(self.peers):
            ops.append(d.P2POp(d.isend, self.send_buf[k][:nf * self.send_cols[k].numel() * self.M], peer))
            ops.append(d.P2POp(d.irecv, self.recv_buf[k][:nf * self.recv_cols[k].numel() * self.M], peer))
        for r in d.batch_isend_irecv(ops):
            r.wait()

    def exchange(self, gather, scatter, fields):
        self.pack(gather, fields)
        self.swap(len(fields))
        self.unpack(scatter, fields)


class PartitionedHEVI:
    """One rank's share of the HEVI ARK2 step on a px x py partition of the global box
    (nex x ney x nez elements of order N over Lx x Ly x Lz): a context of its window and its
    halo exchange.  dist: torch.distributed (or None for a partition driven in one process by
    `step_partitions`).  Further keyword arguments go to the window's context."""

    def __init__(self, nex, ney, nez, Lx, Ly, Lz, N, dt, px, py, rank, dist=None,
                 theta_s=300.0, n_bv=0.0, device="cuda", **ctx_kw):
        self.global_dims = (nex, ney, nez, Lx, Ly, Lz, N)
        self.rank, self.px, self.py = rank, px, py
        self.plan = part_plan(nex, ney, nez, Lx, Ly, Lz, N, px, py, rank, theta_s, n_bv)
        w = self.plan["window"]
        self.ctx = Numa(w["nex"], w["ney"], nez, w["Lx"], w["Ly"], Lz, N, dt, theta_s, n_bv, **ctx_kw)
        self.q2, self.q3, self.pp, self.pp_fused = self.ctx.step_buffers()
        self.halo = HaloExchange(self.plan, self.ctx.M, dist, device)
        self.nxw = w["nex"] * N + 1
        self.nyw = w["ney"] * N + 1
        if dist is not None:
            # every rank constructs its share: one collective here sets up the group's
            # communicators before the first batch of point-to-point operations
            dist.barrier()

    # -- the phases and what each must refresh ------------------------------------------
    def phase(self, k, q_n, q_out=None):
        self.ctx.step_phase(k, q_n, q_out if k == 2 else None)

    def halo_fields(self, k, q_out):
        """The fields whose halo must hold the owners' values after phase k."""
        src = (self.q2, self.q3, q_out)[k]
        f = [src[i] for i in range(5)]
        if k < 2 and self.pp_fused:
            f.append(self.pp)
        return f

    def refresh(self, fields):
        self.halo.exchange(self.ctx.gather_columns, self.ctx.scatter_columns, fields)

    def step(self, q_in, q_out, nsteps=1):
        """nsteps ARK2 steps of this rank's window state; q_in's halo must hold the owners'
        values (as after a previous step or `restrict`); so does q_out's on return."""
        step_partitions([self], [q_in], [q_out], nsteps, lambda fl: self.refresh(fl[0]))
        return q_out

    # -- window <-> global ---------------------------------------------------------------
    def window_slices(self):
        """(y, x) slices of the window's node columns in the global node lattice."""
        N = self.global_dims[6]
        wx0, wx1, wy0, wy1 = self.plan["window_elems"]
        return slice(wy0 * N, wy1 * N + 1), slice(wx0 * N, wx1 * N + 1)

    def owned_slices(self):
        """(y, x) slices of the owned node columns, in window-local and in global indices."""
        N = self.global_dims[6]
        x0, x1, y0, y1 = self.plan["own_cols"]
        wx0, _, wy0, _ = self.plan["window_elems"]
        return ((slice(y0, y1), slice(x0, x1)),
                (slice(wy0 * N + y0, wy0 * N + y1), slice(wx0 * N + x0, wx0 * N + x1)))

    def restrict(self, q_global):
        """The window's part of a global state ((5, nyg, nxg, M) or (5, nnode); a numpy
        array or a torch tensor), as a (5, nnode_window) contiguous copy."""
        nex, ney, nez, _, _, _, N = self.global_dims
        sy, sx = self.window_slices()
        q = q_global.reshape(5, ney * N + 1, nex * N + 1, nez * N + 1)[:, sy, sx, :]
        if isinstance(q, np.ndarray):
            return np.array(q, copy=True).reshape(5, -1)
        return q.clone(memory_format=self.ctx._torch.contiguous_format).reshape(5, -1)

    def owned(self, q_window):
        """The owned node columns of a window state, as (5, ny_own, nx_own, M)."""
        (ly, lx), _ = self.owned_slices()
        return q_window.reshape(5, self.nyw, self.nxw, -1)[:, ly, lx, :]

    def close(self):
        self.ctx.close()


def step_partitions(parts, q_ins, q_outs, nsteps, exchange):
    """nsteps ARK2 steps of every partition in `parts` (their window states q_ins -> q_outs):
    phase k of every partition, then exchange(list of each partition's halo_fields(k)).  With
    one partition per process, exchange swaps messages with the other processes; with
    several in one process, `local_exchange` serves."""
    cur = list(q_ins)
    for _ in range(nsteps):
        for k in PHASES:
            for p, qn, qo in zip(parts, cur, q_outs):
                p.phase(k, qn, qo)
            exchange([p.halo_fields(k, qo) for p, qo in zip(parts, q_outs)])
        cur = list(q_outs)


def local_exchange(parts, field_lists):
    """The halo exchange of partitions held in one process: each pack, the messages are
    copied between the partners' buffers, each unpacks."""
    by_rank = {p.rank: p for p in parts}
    for p, fl in zip(parts, field_lists):
        p.halo.pack(p.ctx.gather_columns, fl)
    for p, fl in zip(parts, field_lists):
        nf = len(fl)
        for k, peer in enumerate(p.halo.peers):
            q = by_rank[peer]
            j = q.halo.peers.index(p.rank)
            n = nf * p.halo.recv_cols[k].numel() * p.halo.M
            p.halo.recv_buf[k][:n].copy_(q.halo.send_buf[j][:n])
    for p, fl in zip(parts, field_lists):
        p.halo.unpack(p.ctx.scatter_columns, fl)


def process_grid(nranks):
    """px x py = nranks with px, py as close as possible (px <= py)."""
    px = max(d for d in range(1, int(nranks ** 0.5) + 1) if nranks % d == 0)
    return px, nranks // px
