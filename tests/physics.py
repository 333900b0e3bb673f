"""Closed forms and statistics used by the tests (independent of the oracle).

Everything here is derived from SI constants (CODATA 2018) and textbook
kinetics, not from the oracle's or the library's literals.
"""
import math

import numpy as np

E_CHARGE = 1.602176634e-19       # C (exact)
M_ELECTRON = 9.1093837015e-31    # kg
Q_OVER_M = E_CHARGE / M_ELECTRON  # C/kg

# unit conversions: cm, ns, V/cm, T
ACCEL_PER_VCM = Q_OVER_M * 100.0 * 1e-16     # (m/s^2 per V/m)*(V/m per V/cm)*(cm/ns^2 per m/s^2)
OMEGA_PER_T = Q_OVER_M * 1e-9                # rad/ns per T


def speed_sq(eps_ev):
    """v^2 in cm^2/ns^2 of an electron with kinetic energy eps (eV)."""
    v_si_sq = 2.0 * eps_ev * E_CHARGE / M_ELECTRON   # m^2/s^2
    return v_si_sq * 1e-14                          # (cm/ns)^2 = (m/s)^2 * 1e4 / 1e18


def drift_velocity(e_vcm, nu):
    """Mean drift speed eE/(m nu) (cm/ns) for constant collision rate nu (1/ns)
    and isotropic elastic scattering without loss."""
    return ACCEL_PER_VCM * e_vcm / nu


def transverse_msd(e_vcm, nu, n_coll, eps0):
    """E[x^2] (cm^2) after n_coll flights for the constant-rate elastic gas
    without loss and E along z.

    x = sum_i s_i n_ix tau_i; the cross terms vanish because each direction
    n_j is isotropic and independent of everything before it, so
    E[x^2] = sum_i E[s_i^2] E[n_ix^2] E[tau_i^2] with E[n_ix^2] = 1/3,
    E[tau^2] = 2/nu^2 and, since the field work is the only energy change
    and E[dz per flight] = a/nu^2, E[s_i^2] = v0^2 + 2 i a^2/nu^2.  Summed:
    (2/(3 nu^2)) (N v0^2 + a^2 N (N-1)/nu^2)."""
    a = ACCEL_PER_VCM * e_vcm
    n = float(n_coll)
    return 2.0 / (3.0 * nu * nu) * (n * speed_sq(eps0) + a * a * n * (n - 1.0) / (nu * nu))


def langevin_drift(e_vec_vcm, b_vec_t, nu):
    """Steady mean velocity of an electron with constant collision rate nu
    (isotropic, speed-preserving collisions): nu v = a + v x w with
    a = -(e/m) E and w = -(e/m) B.  Solved as a 3x3 linear system."""
    a = -ACCEL_PER_VCM * np.asarray(e_vec_vcm, float)
    w = -OMEGA_PER_T * np.asarray(b_vec_t, float)
    # v x w = M v with M = [[0, w2, -w1], [-w2, 0, w0], [w1, -w0, 0]]
    M = np.array([[0.0, w[2], -w[1]], [-w[2], 0.0, w[0]], [w[1], -w[0], 0.0]])
    return np.linalg.solve(nu * np.eye(3) - M, a)


def within_sigma(value, expect, se, k=3.0):
    return abs(value - expect) <= k * se


def geometric_cdf(k, p):
    """P(N <= k) for N ~ Geometric(p) on {1, 2, ...}."""
    return 1.0 - (1.0 - p) ** np.asarray(k, float)


def ramp_first_collision_survival(t, eps0, cos_a, e_vcm, c):
    """P(no real collision before t) for an electron starting with energy
    eps0 (eV) at angle acos(cos_a) to its acceleration a = (e/m)|E| in a
    gas whose total rate is nu(eps) = c * eps (1/ns per eV), with no
    magnetic field.

    v(s) = v0 + a s, so eps(s) = |v(s)|^2 / (2 a_1) with a_1 the acceleration
    per V/cm, and the survival is exp(-int_0^t c eps(s) ds) with
    int_0^t |v0 + a s|^2 ds = |v0|^2 t + (v0.a) t^2 + |a|^2 t^3 / 3."""
    a1 = ACCEL_PER_VCM
    a = a1 * e_vcm
    v0 = np.sqrt(speed_sq(np.asarray(eps0, float)))
    t = np.asarray(t, float)
    integral = v0 * v0 * t + v0 * a * np.asarray(cos_a, float) * t * t + a * a * t ** 3 / 3.0
    return np.exp(-c * integral / (2.0 * a1))


def screened_coulomb_cdf(mu, xi):
    """P(cos chi <= mu) for the density (1 - xi^2) / (2 (1 - xi mu)^2) on
    [-1, 1] (xi != 0)."""
    mu = np.asarray(mu, float)
    return (1.0 - xi * xi) / (2.0 * xi) * (1.0 / (1.0 - xi * mu) - 1.0 / (1.0 + xi))


def screened_coulomb_mean_cos(xi):
    """<cos chi> of that density, by quadrature."""
    from scipy import integrate
    val, _ = integrate.quad(lambda m: m * (1.0 - xi * xi) / (2.0 * (1.0 - xi * m) ** 2), -1.0, 1.0)
    return val


def birth_death(lam, mu, t):
    """Linear birth-death process started from one individual (Kendall 1948):
    mean population at t and the probability of extinction by t."""
    g = math.exp((lam - mu) * t)
    return g, mu * (g - 1.0) / (lam * g - mu)


def opb_cdf(x, w, rest):
    """P(share <= x) for the density proportional to 1 / (1 + (x/w)^2) on
    [0, rest / 2]."""
    return np.arctan(np.asarray(x, float) / w) / math.atan(rest / (2.0 * w))
