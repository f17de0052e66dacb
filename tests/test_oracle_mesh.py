"""Pins of the oracle's box mesh, element-to-global map and DSS (not GPU)."""
import numpy as np

from oracle.mesh import BoxMesh


def _mesh():
    return BoxMesh(3, 2, 2, 3, 3.0e3, 2.5e3, 1.5e3)


def test_l2g_covers_every_node_with_closed_form_multiplicity():
    m = _mesh()
    l2g = m.l2g()
    mult = m.multiplicity(l2g)
    assert mult.min() >= 1
    assert mult.sum() == m.nelem * m.Nq ** 3

    def axis_mult(n_nodes, N):
        i = np.arange(n_nodes)
        return np.where((i % N == 0) & (i > 0) & (i < n_nodes - 1), 2, 1)

    mx, my, mz = axis_mult(m.nxg, m.N), axis_mult(m.nyg, m.N), axis_mult(m.M, m.N)
    expect = (my[:, None, None] * mx[None, :, None] * mz[None, None, :]).ravel()
    np.testing.assert_array_equal(mult, expect)


def test_l2g_brute_force_coordinates():
    m = _mesh()
    l2g = m.l2g()
    xg, yg, zg = m.coords()
    X = np.broadcast_to(xg[None, :, None], (m.nyg, m.nxg, m.M)).ravel()
    Y = np.broadcast_to(yg[:, None, None], (m.nyg, m.nxg, m.M)).ravel()
    Z = np.broadcast_to(zg[None, None, :], (m.nyg, m.nxg, m.M)).ravel()
    for e in range(m.nelem):
        ex, ey, ez = e % m.nex, (e // m.nex) % m.ney, e // (m.nex * m.ney)
        for k in range(m.Nq):
            for j in range(m.Nq):
                for i in range(m.Nq):
                    g = l2g[e, k, j, i]
                    assert abs(X[g] - (ex * m.dx + (1 + m.xi[i]) * m.dx / 2)) < 1e-9
                    assert abs(Y[g] - (ey * m.dy + (1 + m.xi[j]) * m.dy / 2)) < 1e-9
                    assert abs(Z[g] - (ez * m.dz + (1 + m.xi[k]) * m.dz / 2)) < 1e-9


def test_total_mass_is_volume():
    m = _mesh()
    assert abs(m.global_mass().sum() - m.Lx * m.Ly * m.Lz) < 1e-9 * m.Lx * m.Ly * m.Lz


def test_dss_identity_on_continuous_field_and_conservation():
    m = _mesh()
    l2g = m.l2g()
    mass = m.global_mass(l2g)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(m.nnode)
    np.testing.assert_allclose(m.dss(g[l2g], l2g, mass), g, rtol=1e-14, atol=1e-14)
    f = rng.standard_normal(l2g.shape)            # discontinuous element-local field
    lhs = (mass * m.dss(f, l2g, mass)).sum()
    rhs = (np.broadcast_to(m.local_weights(), l2g.shape) * f).sum()
    assert abs(lhs - rhs) < 1e-9 * np.abs(rhs) + 1e-6
