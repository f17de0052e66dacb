"""Physical constants, equation of state and the hydrostatic reference state.

Test infrastructure (oracle).  Sec. "Equation Set2NC":

* equation of state  P = p00 (rho R theta / p00)^gamma, R = c_p - c_v, gamma = c_p / c_v
  (the paper writes the constant as "P_0"; it is the reference surface pressure p00,
  not the background field P_0(x));
* background state in hydrostatic balance, dP0/dz = -rho0 g.

Constants.  R and c_p are pinned by the sound speed the paper quotes in
Sec. "Acoustic wave problem": sqrt(gamma p / rho) = 347.32 m/s for theta0 = 300 K at
the surface.  The paper does not state g; g = 9.80616 m/s^2 is a reading.

Reference profile for a given surface potential temperature theta_s and Brunt-Vaisala
frequency n_bv (n_bv = 0: isentropic, theta0 = theta_s):

* theta0(z) = theta_s exp(n_bv^2 z / g)
* Exner pi0 from d(pi0)/dz = -g / (c_p theta0), pi0(0) = 1:
    isentropic:  pi0 = 1 - g z / (c_p theta_s)
    stratified:  pi0 = 1 + g^2 / (c_p theta_s n_bv^2) (exp(-n_bv^2 z / g) - 1)
* P0 = p00 pi0^(c_p/R);  rho0 = P0 / (R pi0 theta0)
* G0 = gamma P0 / rho0,  H0 = gamma P0 / theta0   (Eq. 2ncp)
"""
import numpy as np

P00 = 1.0e5
R_GAS = 287.17
CP = 1004.67
CV = CP - R_GAS
GAMMA = CP / CV
GRAV = 9.80616


def reference_profile(z, theta_s=300.0, n_bv=0.0):
    """Nodal reference fields at heights z (any shape).  Returns a dict of arrays."""
    z = np.asarray(z, dtype=np.float64)
    if n_bv == 0.0:
        theta0 = np.full_like(z, theta_s)
        pi0 = 1.0 - GRAV * z / (CP * theta_s)
    else:
        s = n_bv * n_bv / GRAV
        theta0 = theta_s * np.exp(s * z)
        pi0 = 1.0 + GRAV * GRAV / (CP * theta_s * n_bv * n_bv) * (np.exp(-s * z) - 1.0)
    P0 = P00 * pi0 ** (CP / R_GAS)
    rho0 = P0 / (R_GAS * pi0 * theta0)
    return {
        "theta0": theta0,
        "pi0": pi0,
        "P0": P0,
        "rho0": rho0,
        "G0": GAMMA * P0 / rho0,
        "H0": GAMMA * P0 / theta0,
    }


def pressure(rho, theta):
    """Equation of state P = p00 (rho R theta / p00)^gamma."""
    return P00 * (rho * R_GAS * theta / P00) ** GAMMA


def pressure_perturbation(rho_p, theta_p, rho0, theta0, P0):
    """P' = P(rho0 + rho', theta0 + theta') - P0 without cancellation.

    With a = rho'/rho0 and b = theta'/theta0 the equation of state gives
    P / P0 = ((1 + a)(1 + b))^gamma, so P' = P0 ((1 + x)^gamma - 1), x = a + b + a b,
    evaluated as P0 expm1(gamma log1p(x)).  This is P - P0 exactly in real arithmetic;
    the direct difference of two ~1e5 Pa pressures would carry ~1e-11 Pa of rounding
    noise, which is the whole of P' in a balanced state (the perturbation split exists
    for numerical accuracy: Sec. "Equation Set2NC").
    """
    a = rho_p / rho0
    b = theta_p / theta0
    x = a + b + a * b
    return P0 * np.expm1(GAMMA * np.log1p(x))


def sound_speed(P, rho):
    """a = sqrt(gamma P / rho) (Sec. "Acoustic wave problem")."""
    return np.sqrt(GAMMA * P / rho)
