"""Pins of the oracle's explicit right-hand side R(q) (not GPU)."""
import numpy as np

from oracle.column import Column
from oracle.mesh import BoxMesh
from oracle.reference import GRAV
from oracle.rhs import rhs, wall_masks
import synthetic


def _setup(nex=3, ney=3, nez=3, N=4, L=(30e3, 30e3, 10e3), n_bv=0.0):
    m = BoxMesh(nex, ney, nez, N, *L)
    return m, Column(m, 300.0, n_bv)


def _lattice(m):
    xg, yg, zg = m.coords()
    shape = (m.nyg, m.nxg, m.M)
    X = np.broadcast_to(xg[None, :, None], shape).ravel()
    Y = np.broadcast_to(yg[:, None, None], shape).ravel()
    Z = np.broadcast_to(zg[None, None, :], shape).ravel()
    return X, Y, Z


def test_rest_state_gives_zero():
    m, col = _setup()
    R = rhs(m, col, np.zeros((5, m.nnode)))
    assert np.abs(R).max() == 0.0               # P' = 0 exactly at rest


def test_pressure_perturbation_is_the_eos_difference():
    from oracle.reference import pressure, pressure_perturbation
    m, col = _setup()
    rng = np.random.default_rng(4)
    rp = 1e-2 * rng.standard_normal(m.M) * col.rho0
    tp = 2.0 * rng.standard_normal(m.M)
    direct = pressure(col.rho0 + rp, col.theta0 + tp) - col.P0
    stable = pressure_perturbation(rp, tp, col.rho0, col.theta0, col.P0)
    np.testing.assert_allclose(stable, direct, rtol=1e-9, atol=1e-9)


def test_balanced_state_gives_pure_buoyancy():
    m, col = _setup()
    xg, yg, zg = m.coords()
    q = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Ly, m.Lz, col.rho0, col.theta0, 7)
    R = rhs(m, col, q)
    rho = np.tile(col.rho0, m.ncol) + q[0]
    _, _, mz = wall_masks(m)
    expect = -GRAV * q[0] / rho
    np.testing.assert_allclose(R[3][~mz], expect[~mz], rtol=1e-9, atol=1e-12)
    assert np.abs(R[3][mz]).max() == 0.0
    assert np.abs(R[0]).max() == 0.0 and np.abs(R[4]).max() == 0.0
    assert np.abs(R[1:3]).max() < 1e-9 * np.abs(R[3]).max()


def test_polynomial_velocity_field_is_exact():
    """rho' = theta' = 0 and velocities polynomial of degree <= N in each direction:
    the discrete derivatives are exact, so R equals the analytic tendencies."""
    m, col = _setup(n_bv=0.01)
    X, Y, Z = _lattice(m)
    x, y, z = X / 1e4, Y / 1e4, Z / 1e4
    u = 1.0 + 0.5 * x - 0.3 * y * z + 0.2 * x * x
    v = -0.4 + 0.7 * y + 0.1 * x * z
    w = 0.3 * z - 0.2 * x * y + 0.05 * z * z
    dudx, dudy, dudz = (0.5 + 0.4 * x) / 1e4, (-0.3 * z) / 1e4, (-0.3 * y) / 1e4
    dvdx, dvdy, dvdz = (0.1 * z) / 1e4, 0.7 / 1e4, (0.1 * x) / 1e4
    dwdx, dwdy, dwdz = (-0.2 * y) / 1e4, (-0.2 * x) / 1e4, (0.3 + 0.1 * z) / 1e4
    q = np.zeros((5, m.nnode))
    q[1], q[2], q[3] = u, v, w
    R = rhs(m, col, q)
    rho0 = np.tile(col.rho0, m.ncol)
    drho0 = np.tile(col.drho0, m.ncol)
    dth0 = np.tile(col.dtheta0, m.ncol)
    mx, my, mz = wall_masks(m)
    np.testing.assert_allclose(R[0], -(w * drho0 + rho0 * (dudx + dvdy + dwdz)), rtol=1e-9, atol=1e-16)
    Ru = -(u * dudx + v * dudy + w * dudz)
    Rv = -(u * dvdx + v * dvdy + w * dvdz)
    Rw = -(u * dwdx + v * dwdy + w * dwdz)
    np.testing.assert_allclose(R[1][~mx], Ru[~mx], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(R[2][~my], Rv[~my], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(R[3][~mz], Rw[~mz], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(R[4], -w * dth0, rtol=1e-9, atol=1e-16)
    assert np.all(R[1][mx] == 0) and np.all(R[2][my] == 0) and np.all(R[3][mz] == 0)


def test_isentropic_reference_gradient_is_zero():
    m, col = _setup()
    assert np.all(col.dtheta0 == 0.0)


def test_pressure_gradient_against_finite_differences():
    """u = 0, rho' = 0, smooth theta': R_u = -dP'/dx / rho0 etc. (P' through the EOS).
    The LGL derivative of the non-polynomial P' is only spectrally accurate (8 elements
    per wavelength, N=4): 2e-4 of the largest term."""
    m, col = _setup(nex=8, ney=8, nez=6, L=(20e3, 20e3, 10e3))
    X, Y, Z = _lattice(m)

    def th(x, y, z):
        return 0.5 * np.cos(2 * np.pi * x / 20e3) * np.cos(2 * np.pi * y / 20e3) * np.sin(np.pi * z / 10e3)

    from oracle.reference import pressure, reference_profile

    def Pp(x, y, z):
        r = reference_profile(z, 300.0)
        return pressure(r["rho0"], r["theta0"] + th(x, y, z)) - r["P0"]

    q = np.zeros((5, m.nnode))
    q[4] = th(X, Y, Z)
    R = rhs(m, col, q)
    h = 1.0
    rho0 = np.tile(col.rho0, m.ncol)
    dPx = (Pp(X + h, Y, Z) - Pp(X - h, Y, Z)) / (2 * h)
    dPy = (Pp(X, Y + h, Z) - Pp(X, Y - h, Z)) / (2 * h)
    dPz = (Pp(X, Y, Z + h) - Pp(X, Y, Z - h)) / (2 * h)
    mx, my, mz = wall_masks(m)
    scale = np.abs(dPz / rho0).max()
    assert np.abs(R[1][~mx] + (dPx / rho0)[~mx]).max() < 2e-4 * scale
    assert np.abs(R[2][~my] + (dPy / rho0)[~my]).max() < 2e-4 * scale
    assert np.abs(R[3][~mz] + (dPz / rho0)[~mz]).max() < 2e-4 * scale
    assert np.abs(R[0]).max() == 0.0 and np.abs(R[4]).max() == 0.0


def test_horizontally_uniform_state_has_no_horizontal_tendency():
    m, col = _setup()
    xg, yg, zg = m.coords()
    q = synthetic.balanced_state(xg, yg, zg, m.Lx, m.Ly, m.Lz, col.rho0, col.theta0, 9, uniform=True)
    q = q.reshape(5, m.nyg, m.nxg, m.M)
    q[3] = 0.3 * np.sin(np.pi * zg / m.Lz)[None, None, :]
    R = rhs(m, col, q.reshape(5, -1)).reshape(5, m.nyg, m.nxg, m.M)
    assert np.abs(R[1:3]).max() < 1e-10 * np.abs(R[3]).max()
    for f in (0, 3, 4):
        spread = np.abs(R[f] - R[f][:1, :1, :]).max()
        assert spread <= 1e-10 * (np.abs(R[f]).max() + 1e-300)


def test_linearisation_matches_vertical_operator():
    """Horizontally uniform, u = v = 0: R(eps q) / eps -> L_V(q) as eps -> 0."""
    m, col = _setup(n_bv=0.01)
    zg = m.coords()[2]
    rng = np.random.default_rng(5)
    prof = rng.standard_normal((3, m.M))
    prof[1, 0] = prof[1, -1] = 0.0
    q = np.zeros((5, m.ncol, m.M))
    q[0] = 1e-3 * prof[0] * col.rho0
    q[3] = prof[1]
    q[4] = prof[2]
    eps = 1e-6
    R = rhs(m, col, eps * q.reshape(5, -1)).reshape(5, m.ncol, m.M) / eps
    Lr, Lw, Lt = col.L_V(q[0][0], q[3][0], q[4][0])
    for got, ref in ((R[0][7], Lr), (R[3][7], Lw), (R[4][7], Lt)):
        assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


def test_all_fields_nonzero_against_closed_forms():
    """rho', u, v, w and theta' all nonzero together, each a polynomial of degree <= N = 4
    along every axis.  Their LGL derivatives are then exact, so the continuity and theta'
    tendencies have closed forms (u.grad rho', rho div u with rho = rho0 + rho', u.grad
    theta').  P' is not a polynomial (equation of state over a z-dependent reference): its
    gradient is a centred difference of the EOS, and the momentum tendencies
    -(u.grad u + grad P' / rho + g rho' / rho z_hat) are checked to the spectral accuracy of
    the mesh.  rho' is 1-8 % of rho0, so reading rho0 for rho anywhere (in rho div u, in
    grad P' / rho or in the buoyancy) moves a tendency far outside these bounds; the test
    checks that margin too."""
    from oracle.reference import pressure, reference_profile
    m, col = _setup(nex=8, ney=8, nez=6, L=(20e3, 20e3, 10e3))
    X, Y, Z = _lattice(m)

    def fields(X, Y, Z):
        x, y, z = X / 1e4, Y / 1e4, Z / 1e4
        rp = 0.02 * (1.0 + 0.3 * x - 0.2 * y + 0.1 * z + 0.05 * x * y)
        u = 1.0 + 0.5 * x - 0.3 * y * z + 0.2 * x * x
        v = -0.4 + 0.7 * y + 0.1 * x * z
        w = 0.3 * z - 0.2 * x * y + 0.05 * z * z
        tp = 0.5 * (1.0 + 0.2 * x + 0.3 * y * z - 0.1 * z * z)
        return rp, u, v, w, tp

    rp, u, v, w, tp = fields(X, Y, Z)
    x, y, z = X / 1e4, Y / 1e4, Z / 1e4
    s = 1e-4
    drx, dry, drz = 0.02 * (0.3 + 0.05 * y) * s, 0.02 * (-0.2 + 0.05 * x) * s, 0.002 * s
    dudx, dudy, dudz = (0.5 + 0.4 * x) * s, (-0.3 * z) * s, (-0.3 * y) * s
    dvdx, dvdy, dvdz = (0.1 * z) * s, 0.7 * s, (0.1 * x) * s
    dwdx, dwdy, dwdz = (-0.2 * y) * s, (-0.2 * x) * s, (0.3 + 0.1 * z) * s
    dtx, dty, dtz = 0.1 * s + 0 * x, 0.15 * z * s, 0.5 * (0.3 * y - 0.2 * z) * s
    q = np.stack([rp, u, v, w, tp])
    R = rhs(m, col, q)

    rho0 = np.tile(col.rho0, m.ncol)
    drho0 = np.tile(col.drho0, m.ncol)
    dth0 = np.tile(col.dtheta0, m.ncol)
    assert 0.005 < (rp / rho0).min() and (rp / rho0).max() < 0.1
    rho = rho0 + rp
    div = dudx + dvdy + dwdz
    adv = lambda fx, fy, fz: u * fx + v * fy + w * fz
    R_rho = -(adv(drx, dry, drz) + w * drho0 + rho * div)
    R_th = -(adv(dtx, dty, dtz) + w * dth0)
    np.testing.assert_allclose(R[0], R_rho, rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(R[4], R_th, rtol=1e-9, atol=1e-16)
    # the exact tendencies tell rho from rho0 in rho div u: by far more than the bound
    assert np.abs(rp * div).max() > 1e3 * 1e-9 * np.abs(R_rho).max()

    def Pp(X, Y, Z):
        r = reference_profile(Z, 300.0)
        a = fields(X, Y, Z)
        return pressure(r["rho0"] + a[0], r["theta0"] + a[4]) - r["P0"]

    h = 1.0
    dPx = (Pp(X + h, Y, Z) - Pp(X - h, Y, Z)) / (2 * h)
    dPy = (Pp(X, Y + h, Z) - Pp(X, Y - h, Z)) / (2 * h)
    dPz = (Pp(X, Y, Z + h) - Pp(X, Y, Z - h)) / (2 * h)
    mx, my, mz = wall_masks(m)
    Ru = -(adv(dudx, dudy, dudz) + dPx / rho)
    Rv = -(adv(dvdx, dvdy, dvdz) + dPy / rho)
    Rw = -(adv(dwdx, dwdy, dwdz) + dPz / rho + GRAV * rp / rho)
    tol = 2e-4
    for got, ref, mask in ((R[1], Ru, mx), (R[2], Rv, my), (R[3], Rw, mz)):
        scale = np.abs(ref[~mask]).max()
        assert np.abs(got[~mask] - ref[~mask]).max() < tol * scale
        assert np.all(got[mask] == 0.0)
    # rho0 in place of rho in grad P' / rho and in the buoyancy would miss by > 5x the bound
    Rw_wrong = -(adv(dwdx, dwdy, dwdz) + dPz / rho0 + GRAV * rp / rho0)
    Ru_wrong = -(adv(dudx, dudy, dudz) + dPx / rho0)
    assert np.abs((Rw_wrong - Rw)[~mz]).max() > 5 * tol * np.abs(Rw[~mz]).max()
    assert np.abs((Ru_wrong - Ru)[~mx]).max() > 5 * tol * np.abs(Ru[~mx]).max()
