"""Box mesh of hexahedral spectral elements, element-to-global map and DSS.

Test infrastructure (oracle).

Numbering (Sec. "1D-IMEX kernels": the nodes of one column are numbered consecutively so
that the global vertical Jacobian is block diagonal):

* global node (ix, iy, iz), ix in [0, nxg), iy in [0, nyg), iz in [0, M),
  nxg = nex*N + 1, nyg = ney*N + 1, M = nez*N + 1;
* column id  col = iy*nxg + ix;  global id  g = col*M + iz;
* element id e = ex + nex*(ey + ney*ez);
* element-local node (i, j, k) -> ix = ex*N + i, iy = ey*N + j, iz = ez*N + k, stored in
  the local order [k][j][i] of the paper's ``sq[k][j][i]`` (Algorithms 1-2).

Direct stiffness summation (Sec. "Direct stiffness summation"): an element-local field
f_e is summed into the global nodes with the local mass weights w_i w_j w_k J_e and
divided by the global (lumped) mass:  DSS(f)_g = sum_{(e,l)->g} W_l J_e f_e[l] / M_g,
M_g = sum_{(e,l)->g} W_l J_e.
"""
import numpy as np

from .lgl import lgl


class BoxMesh:
    """Uniform box [0,Lx]x[0,Ly]x[0,Lz] with nex x ney x nez elements of order N."""

    def __init__(self, nex, ney, nez, N, Lx, Ly, Lz):
        if min(nex, ney, nez) < 1 or N < 1:
            raise ValueError("bad mesh")
        self.nex, self.ney, self.nez, self.N = nex, ney, nez, N
        self.Lx, self.Ly, self.Lz = float(Lx), float(Ly), float(Lz)
        self.Nq = N + 1
        self.nxg, self.nyg, self.M = nex * N + 1, ney * N + 1, nez * N + 1
        self.ncol = self.nxg * self.nyg
        self.nnode = self.ncol * self.M
        self.nelem = nex * ney * nez
        self.dx, self.dy, self.dz = self.Lx / nex, self.Ly / ney, self.Lz / nez
        self.xi, self.w, self.D = lgl(N)
        # Jacobian determinant of the affine element map (box: dx dy dz / 8)
        self.J = self.dx * self.dy * self.dz / 8.0

    # -- coordinates ---------------------------------------------------------
    def axis_coords(self, n_elem, h):
        """Global 1D node coordinates along one axis: x = e*h + (1 + xi_i) h / 2."""
        c = np.empty(n_elem * self.N + 1)
        for e in range(n_elem):
            for i in range(self.Nq):
                c[e * self.N + i] = e * h + (1.0 + self.xi[i]) * h / 2.0
        return c

    def coords(self):
        """(xg, yg, zg): 1D coordinate arrays of the global node lines."""
        return (self.axis_coords(self.nex, self.dx), self.axis_coords(self.ney, self.dy),
                self.axis_coords(self.nez, self.dz))

    def global_id(self, ix, iy, iz):
        return (iy * self.nxg + ix) * self.M + iz

    # -- element-to-global map -------------------------------------------------
    def l2g(self):
        """int64 array [nelem, Nq, Nq, Nq] (local order [k][j][i]) of global ids."""
        N, Nq = self.N, self.Nq
        out = np.empty((self.nelem, Nq, Nq, Nq), dtype=np.int64)
        for ez in range(self.nez):
            for ey in range(self.ney):
                for ex in range(self.nex):
                    e = ex + self.nex * (ey + self.ney * ez)
                    for k in range(Nq):
                        for j in range(Nq):
                            for i in range(Nq):
                                out[e, k, j, i] = self.global_id(ex * N + i, ey * N + j, ez * N + k)
        return out

    def local_weights(self):
        """W[k, j, i] J: local mass of each element-local node (same for every element)."""
        w = self.w
        return w[:, None, None] * w[None, :, None] * w[None, None, :] * self.J

    def multiplicity(self, l2g=None):
        """Number of element-local copies of every global node (1, 2, 4 or 8)."""
        l2g = self.l2g() if l2g is None else l2g
        return np.bincount(l2g.ravel(), minlength=self.nnode)

    def global_mass(self, l2g=None):
        """Lumped global mass M_g = DSS-sum of the local masses."""
        l2g = self.l2g() if l2g is None else l2g
        Wl = np.broadcast_to(self.local_weights(), l2g.shape)
        m = np.zeros(self.nnode)
        np.add.at(m, l2g.ravel(), Wl.ravel())
        return m

    def dss(self, f_local, l2g=None, mass=None):
        """DSS of an element-local field f_local[nelem, Nq, Nq, Nq] -> global [nnode]."""
        l2g = self.l2g() if l2g is None else l2g
        mass = self.global_mass(l2g) if mass is None else mass
        Wl = np.broadcast_to(self.local_weights(), l2g.shape)
        acc = np.zeros(self.nnode)
        np.add.at(acc, l2g.ravel(), (Wl * f_local).ravel())
        return acc / mass
