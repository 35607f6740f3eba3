"""Wetting theory of the ternary model, written out plainly (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the independent
checker of the product's host-side contact-angle functions.

Follows Sec. Surface Thermodynamics and Sec. Inverting the contact angle
relations of arXiv:1511.02155 step by step, without the simplified closed form:
- wall values of C_m from the Cahn condition with Noether's invariant: the
  majority root C_max = (1 + sqrt(1 + 4h/(alpha kappa)))/2 and the minority root
  C_min = (1 - sqrt(1 - 4h/(alpha kappa)))/2;
- I_m = -h_m C_max + int_{C_max}^{1} alpha kappa_m C (1 - C) dC (majority phase m),
  J_n = -h_n C_min - int_{C_min}^{0} alpha kappa_n C (1 - C) dC (minority phase n),
  the integrals taken by numerical quadrature;
- gamma_sm = I_m + sum_{n != m} J_n (Eq. solidST), gamma_mn = alpha (kappa_m + kappa_n)/6
  (Eq. SurfTens), and Young's equation cos theta_mn = (gamma_sn - gamma_sm)/gamma_mn
  (Eq. contact angle), theta_mn measured through fluid m;
- the inverse problem solved numerically on Young's equation itself with the
  gauge sum_m h_m / kappa_m = 0 (Eq. Redundancy).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, optimize

PAIRS = ((0, 1), (1, 2), (2, 0))  # theta_12, theta_23, theta_31


def wall_roots(kappa_m: float, alpha: float, h_m: float):
    """(C_max, C_min) at the wall for component m (Sec. Surface Thermodynamics)."""
    r = 4.0 * h_m / (alpha * kappa_m)
    if not abs(r) < 1.0:
        raise ValueError("|4 h / (alpha kappa)| must be < 1")
    return 0.5 * (1.0 + np.sqrt(1.0 + r)), 0.5 * (1.0 - np.sqrt(1.0 - r))


def _integral(kappa_m, alpha, a, b):
    val, _ = integrate.quad(lambda C: alpha * kappa_m * C * (1.0 - C), a, b, epsabs=1e-15, epsrel=1e-13)
    return val


def majority_term(kappa_m, alpha, h_m):
    """I_m: surface energy of component m where it is the bulk phase."""
    cmax, _ = wall_roots(kappa_m, alpha, h_m)
    return -h_m * cmax + _integral(kappa_m, alpha, cmax, 1.0)


def minority_term(kappa_n, alpha, h_n):
    """J_n: surface energy of component n where it is absent in the bulk."""
    _, cmin = wall_roots(kappa_n, alpha, h_n)
    return -h_n * cmin - _integral(kappa_n, alpha, cmin, 0.0)


def solid_tensions(kappa, alpha, h):
    """(gamma_s1, gamma_s2, gamma_s3) = I_m + sum_{n != m} J_n."""
    out = []
    for m in range(3):
        g = majority_term(kappa[m], alpha, h[m])
        g += sum(minority_term(kappa[n], alpha, h[n]) for n in range(3) if n != m)
        out.append(g)
    return tuple(out)


def fluid_tension(kappa, alpha, m, n):
    """gamma_mn = alpha (kappa_m + kappa_n) / 6 (Eq. SurfTens)."""
    return alpha * (kappa[m] + kappa[n]) / 6.0


def contact_cosines(kappa, alpha, h):
    """(cos theta_12, cos theta_23, cos theta_31) from Young's equation."""
    gs = solid_tensions(kappa, alpha, h)
    return tuple((gs[n] - gs[m]) / fluid_tension(kappa, alpha, m, n) for m, n in PAIRS)


def contact_angles(kappa, alpha, h):
    """(theta_12, theta_23, theta_31) in degrees."""
    return tuple(float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))) for c in contact_cosines(kappa, alpha, h))


def wetting_from_angles(kappa, alpha, theta12, theta13):
    """h with theta_12 and theta_13 (through fluid 1, degrees) and sum h_m/kappa_m = 0,
    by a numerical root of Young's equation.  None when no admissible h exists:
    the solver finds no root with |4 h_m| < alpha kappa_m, or the third pair would
    have no contact angle (|cos theta_23| >= 1: one fluid wets completely)."""
    c12 = np.cos(np.radians(theta12))
    c13 = np.cos(np.radians(theta13))  # theta_13 = 180 - theta_31

    def h_of(u):  # every u maps to an admissible h_m = (alpha kappa_m / 4) tanh(u_m)
        return tuple(alpha * kappa[m] / 4.0 * np.tanh(u[m]) for m in range(3))

    def F(u):
        h = h_of(u)
        c = contact_cosines(kappa, alpha, h)
        return [c[0] - c12, -c[2] - c13, sum(h[m] / kappa[m] for m in range(3)) / (alpha / 4.0)]

    try:
        sol = optimize.root(F, [0.0, 0.0, 0.0], method="hybr", tol=1e-14)
    except ValueError:  # the search reached |tanh u| = 1 in floating point: the edge of the range
        return None
    if max(abs(v) for v in F(sol.x)) > 1e-12:  # judged by the residual, not the solver's flag
        return None
    h = tuple(float(v) for v in h_of(sol.x))
    if not abs(contact_cosines(kappa, alpha, h)[1]) < 1.0:
        return None
    return h
