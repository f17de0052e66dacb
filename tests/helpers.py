"""Shared test helpers: oracle cases, error norms and the windowed oracle."""
import numpy as np

import synthetic
from oracle.column import Column
from oracle.mesh import BoxMesh
from oracle.reference import GAMMA, R_GAS

C_S = float(np.sqrt(GAMMA * R_GAS * 300.0))


class Case:
    def __init__(self, nex, ney, nez, N, Lx, Ly, Lz, n_bv=0.0):
        self.mesh = BoxMesh(nex, ney, nez, N, Lx, Ly, Lz)
        self.col = Column(self.mesh, 300.0, n_bv)
        self.n_bv = n_bv
        self.args = (nex, ney, nez, Lx, Ly, Lz, N)

    def dt_for(self, C):
        m = self.mesh
        dzmin = (m.xi[1] - m.xi[0]) * m.dz / 2
        return C * dzmin / C_S

    def state(self, seed, kind="random", **kw):
        m, col = self.mesh, self.col
        xg, yg, zg = m.coords()
        f = synthetic.random_state if kind == "random" else synthetic.balanced_state
        return f(xg, yg, zg, m.Lx, m.Ly, m.Lz, col.rho0, col.theta0, seed, **kw)


def rel_l2(a, b):
    """Per-field relative L2 error of a against reference b (arrays (5, n))."""
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    out = []
    for f in range(5):
        nb = np.linalg.norm(b[f])
        out.append(np.linalg.norm(a[f] - b[f]) / nb if nb > 0 else np.linalg.norm(a[f]))
    return np.array(out)


def window(mesh, q, ex0, ey0, W):
    """Sub-box of W x W elements (all z) starting at element (ex0, ey0): its mesh and the
    restriction of the state q (5, nnode)."""
    N = mesh.N
    sub = BoxMesh(W, W, mesh.nez, N, W * mesh.dx, W * mesh.dy, mesh.Lz)
    qq = q.reshape(5, mesh.nyg, mesh.nxg, mesh.M)
    ix0, iy0 = ex0 * N, ey0 * N
    qs = qq[:, iy0:iy0 + W * N + 1, ix0:ix0 + W * N + 1, :]
    return sub, np.ascontiguousarray(qs).reshape(5, -1)


def window_nodes(mesh, ex0, ey0, W, margin):
    """Global ids (of the full mesh) of the window nodes at least `margin` elements away
    from the window's lateral edges, and their ids within the window."""
    N = mesh.N
    lo, hi = margin * N, (W - margin) * N
    loc = np.arange(lo, hi + 1)
    ixs = ex0 * N + loc
    iys = ey0 * N + loc
    nw = W * N + 1
    gi = ((iys[:, None, None] * mesh.nxg + ixs[None, :, None]) * mesh.M
          + np.arange(mesh.M)[None, None, :]).ravel()
    wi = ((loc[:, None, None] * nw + loc[None, :, None]) * mesh.M
          + np.arange(mesh.M)[None, None, :]).ravel()
    return gi, wi
