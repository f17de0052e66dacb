"""Explicit right-hand side R(q) of the Set2NC perturbation equations (cG).

Test infrastructure (oracle).  Sec. "Equation Set2NC", perturbation form:

    d rho'/dt  = -( u.grad rho' + u.grad rho0 + (rho0 + rho') div u )
    d u/dt     = -( u.grad u + grad P' / (rho0 + rho') + (rho' / (rho0 + rho')) g z_hat )
    d theta'/dt= -( u.grad theta' + u.grad theta0 )

with P' = P(rho0 + rho', theta0 + theta') - P0 from the equation of state (evaluated without
cancellation, see reference.pressure_perturbation).

Discretisation (Sec. "Spatial discretization", Algorithm 2 GradDiv-3D, Sec. "Direct
stiffness summation"): element by element, the five fields and P' are gathered to the
element's (N+1)^3 nodes, differentiated with the LGL matrix D along the three reference
directions and scaled by the (diagonal, box) metric 2/dx, 2/dy, 2/dz; the pointwise
tendency is formed at every element-local node, multiplied by the local mass w_i w_j w_k
J and summed into the global nodes, then divided by the global mass (DSS).  The
reference gradients are the precomputed nodal D_z rho0, D_z theta0 (they depend on z
only in the box).

Walls (no flux on all six faces; the paper states no-flux at the bottom and top): after
DSS the wall-normal velocity tendency is set to zero on each face (u on x-faces, v on
y-faces, w on z-faces).
"""
import numpy as np

from .reference import GRAV, pressure_perturbation


def rhs(mesh, col, q, l2g=None, mass=None):
    """R(q) for a state q of shape (5, nnode) in the order (rho', u, v, w, theta')."""
    l2g = mesh.l2g() if l2g is None else l2g
    mass = mesh.global_mass(l2g) if mass is None else mass
    D = mesh.D
    iz = l2g % mesh.M                                   # vertical level of every local node
    f = q[:, l2g]                                       # (5, E, k, j, i)
    rho_p, u, v, w, th_p = f
    rho0, theta0, P0 = col.rho0[iz], col.theta0[iz], col.P0[iz]
    drho0, dtheta0 = col.drho0[iz], col.dtheta0[iz]
    rho = rho0 + rho_p
    Pp = pressure_perturbation(rho_p, th_p, rho0, theta0, P0)

    sx, sy, sz = 2.0 / mesh.dx, 2.0 / mesh.dy, 2.0 / mesh.dz

    def ddx(a):  # sum_n D[i,n] a[e,k,j,n]
        return np.einsum("in,ekjn->ekji", D, a) * sx

    def ddy(a):  # sum_n D[j,n] a[e,k,n,i]
        return np.einsum("jn,ekni->ekji", D, a) * sy

    def ddz(a):  # sum_n D[k,n] a[e,n,j,i]
        return np.einsum("kn,enji->ekji", D, a) * sz

    def adv(a):
        return u * ddx(a) + v * ddy(a) + w * ddz(a)

    div_u = ddx(u) + ddy(v) + ddz(w)
    t_rho = -(adv(rho_p) + w * drho0 + rho * div_u)
    t_u = -(adv(u) + ddx(Pp) / rho)
    t_v = -(adv(v) + ddy(Pp) / rho)
    t_w = -(adv(w) + ddz(Pp) / rho + GRAV * rho_p / rho)
    t_th = -(adv(th_p) + w * dtheta0)

    out = np.stack([mesh.dss(t, l2g, mass) for t in (t_rho, t_u, t_v, t_w, t_th)])
    apply_wall_bc(mesh, out)
    return out


def wall_masks(mesh):
    """Boolean masks over global nodes: on an x-wall, a y-wall, a z-wall."""
    ix = np.arange(mesh.nxg)
    iy = np.arange(mesh.nyg)
    izz = np.arange(mesh.M)
    onx = ((ix == 0) | (ix == mesh.nxg - 1))[None, :, None]
    ony = ((iy == 0) | (iy == mesh.nyg - 1))[:, None, None]
    onz = ((izz == 0) | (izz == mesh.M - 1))[None, None, :]
    shape = (mesh.nyg, mesh.nxg, mesh.M)
    return (np.broadcast_to(onx, shape).ravel(), np.broadcast_to(ony, shape).ravel(),
            np.broadcast_to(onz, shape).ravel())


def apply_wall_bc(mesh, t):
    """Zero the wall-normal velocity component of t (5, nnode) in place."""
    mx, my, mz = wall_masks(mesh)
    t[1, mx] = 0.0
    t[2, my] = 0.0
    t[3, mz] = 0.0
    return t
