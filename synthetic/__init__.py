"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds no arithmetic of the method: it evaluates seeded Fourier sums at node
coordinates that the caller supplies, and builds the initial state from reference
profiles that the caller supplies.  It imports neither the oracle nor the CUDA library.

Layout of every state: float64 array (5, ncol*M) in the order (rho', u, v, w, theta'),
global id g = (iy*nxg + ix)*M + iz (columns consecutive).

Recipe (perturbation of a hydrostatic rest state):
* theta' = sum_{m=1..8} a_m cos(2 pi kx_m x/Lx + phi_m) cos(2 pi ky_m y/Ly + psi_m)
  sin(pi kz_m z/Lz), kx, ky in {1,2,3}, kz in {1,2}, phases U[0, 2 pi), a_m in U[0.5, 1],
  rescaled so that max |theta'| over the nodes equals ``amp`` (K).  ``uniform=True``
  sets kx = ky = 0 (a horizontally uniform state).
* rho' = rho0 (theta0 / (theta0 + theta') - 1), so that rho theta = rho0 theta0 and the
  initial pressure perturbation vanishes; u = v = w = 0.
* ``random_state`` additionally draws smooth velocities (amplitude ``vel`` m/s) that
  vanish on the walls they are normal to, for tests that exercise every term.
Seeds: numpy PCG64(seed).
"""
import numpy as np


def _modes(rng, n_modes, uniform):
    kx = np.zeros(n_modes, dtype=np.int64) if uniform else rng.integers(1, 4, n_modes)
    ky = np.zeros(n_modes, dtype=np.int64) if uniform else rng.integers(1, 4, n_modes)
    kz = rng.integers(1, 3, n_modes)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    psi = rng.uniform(0.0, 2.0 * np.pi, n_modes)
    a = rng.uniform(0.5, 1.0, n_modes)
    return kx, ky, kz, phi, psi, a


def fourier_theta(xg, yg, zg, Lx, Ly, Lz, rng, amp, n_modes=8, uniform=False):
    """theta' on the (nyg, nxg, M) node lattice given the 1D coordinate arrays."""
    kx, ky, kz, phi, psi, a = _modes(rng, n_modes, uniform)
    X = xg[None, :, None]
    Y = yg[:, None, None]
    Z = zg[None, None, :]
    th = np.zeros((yg.size, xg.size, zg.size))
    for m in range(n_modes):
        th += (a[m] * np.cos(2 * np.pi * kx[m] * X / Lx + phi[m])
               * np.cos(2 * np.pi * ky[m] * Y / Ly + psi[m])
               * np.sin(np.pi * kz[m] * Z / Lz))
    mx = np.max(np.abs(th))
    return th * (amp / mx) if mx > 0 else th


def balanced_state(xg, yg, zg, Lx, Ly, Lz, rho0_lev, theta0_lev, seed, amp=0.5,
                   uniform=False):
    """Initial state (5, nnode): theta' from the Fourier recipe, rho' balancing it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = fourier_theta(xg, yg, zg, Lx, Ly, Lz, rng, amp, uniform=uniform)
    rho0 = np.asarray(rho0_lev)[None, None, :]
    theta0 = np.asarray(theta0_lev)[None, None, :]
    rho_p = rho0 * (theta0 / (theta0 + th) - 1.0)
    q = np.zeros((5,) + th.shape)
    q[0] = rho_p
    q[4] = th
    return q.reshape(5, -1)


def random_state(xg, yg, zg, Lx, Ly, Lz, rho0_lev, theta0_lev, seed, amp=0.5, vel=5.0,
                 rho_amp=2e-3):
    """A smooth state with every field non-zero (wall-normal velocities vanish on walls)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = balanced_state(xg, yg, zg, Lx, Ly, Lz, rho0_lev, theta0_lev,
                       int(rng.integers(1 << 30)), amp).reshape(5, yg.size, xg.size, zg.size)
    X = xg[None, :, None] / Lx
    Y = yg[:, None, None] / Ly
    Z = zg[None, None, :] / Lz

    def smooth(nonzero_axis=None):
        f = np.zeros(q.shape[1:])
        for _ in range(4):
            k = rng.integers(1, 3, 3)
            ph = rng.uniform(0, 2 * np.pi, 3)
            gx = np.sin(np.pi * k[0] * X) if nonzero_axis == 0 else np.cos(2 * np.pi * k[0] * X + ph[0])
            gy = np.sin(np.pi * k[1] * Y) if nonzero_axis == 1 else np.cos(2 * np.pi * k[1] * Y + ph[1])
            gz = np.sin(np.pi * k[2] * Z) if nonzero_axis == 2 else np.cos(2 * np.pi * k[2] * Z + ph[2])
            f += rng.uniform(0.5, 1.0) * gx * gy * gz
        return f / np.max(np.abs(f))

    q[1] = vel * smooth(0)
    q[2] = vel * smooth(1)
    q[3] = 0.5 * vel * smooth(2)
    q[0] += rho_amp * np.asarray(rho0_lev)[None, None, :] * smooth()
    return q.reshape(5, -1)
