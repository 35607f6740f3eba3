"""Physics pins of the full oracle step against the paper's closed forms.

- A flat m/n interface relaxes to C = (1 + tanh(x / 2 alpha)) / 2 (Eq. tanh);
  the lattice error falls roughly as 1/alpha^2 when alpha doubles, and the
  relaxed profile satisfies the first integral of Eq. invariant.
- A drop of fluid m in fluid n obeys the 2-D Laplace law dp = gamma_mn / R with
  gamma_mn = alpha (kappa_m + kappa_n) / 6 (Eq. SurfTens), for all three pairs
  (the paper reports the Laplace test, data not shown).
- Next to a wall, the concentrations approach the wall values
  C_m|s = (1 +- sqrt(1 +- 4 h_m / (alpha kappa_m))) / 2 of the surface
  thermodynamics section (majority: larger root, minority: smaller root).
"""
import numpy as np
import pytest

import oracle
from paper_1511_02155_gb300 import workloads as W

KAPPA = (0.01, 0.02, 0.03)


def _relax(p, C, steps, solid=None):
    rho, phi, psi = W.to_aux(*C)
    if solid is not None:
        for a in (rho, phi, psi):
            a[solid != 0] = 0.0
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    oracle.step(p, f, g, k, steps, solid)
    return oracle.fields(p, f, g, k, solid)


def _slab(m, n, nx, width):
    x = np.arange(nx, dtype=float)
    prof = 0.5 * (np.tanh((x - nx / 4) / (2 * width)) - np.tanh((x - 3 * nx / 4) / (2 * width)))
    C = [np.zeros((2, nx)) for _ in range(3)]
    C[m][:] = prof
    C[n][:] = 1 - prof
    return C


def _tanh_slab(nx, alpha):
    x = np.arange(nx, dtype=float)
    return 0.5 * (np.tanh((x - nx / 4) / (2 * alpha)) - np.tanh((x - 3 * nx / 4) / (2 * alpha)))


@pytest.mark.parametrize("m,n", [(0, 1), (0, 2), (1, 2)])
def test_flat_interface_tanh_profile_and_first_integral(m, n):
    errs = {}
    for alpha in (1.0, 2.0):
        nx = int(64 * alpha)
        p = oracle.make_params(9, nx, 2, 1, KAPPA, alpha, tau_f=1.0, M_phi=0.5, M_psi=0.5)
        C1, C2, C3, rho, u = _relax(p, _slab(m, n, nx, alpha), 4000)
        Cm = [C1, C2, C3][m].reshape(2, nx)[0]
        errs[alpha] = np.abs(Cm - _tanh_slab(nx, alpha)).max()
        assert np.abs(u).max() < 1e-6
        assert np.abs(rho - 1).max() < 1e-3
        if alpha == 2.0:
            # first integral kappa/2 C^2 (1-C)^2 = alpha^2 kappa/2 |C'|^2 (Eq. invariant),
            # C' by a fourth-order central difference
            dC = (-np.roll(Cm, -2) + 8 * np.roll(Cm, -1) - 8 * np.roll(Cm, 1) + np.roll(Cm, 2)) / 12
            lhs = Cm ** 2 * (1 - Cm) ** 2
            rhs = alpha ** 2 * dC ** 2
            assert np.abs(lhs - rhs).max() < 0.03 * lhs.max()
    assert errs[1.0] < 1e-2
    assert errs[2.0] < errs[1.0] / 3.0


def test_sharp_interface_relaxes_towards_tanh():
    nx, alpha = 64, 1.0
    p = oracle.make_params(9, nx, 2, 1, KAPPA, alpha, tau_f=1.0, M_phi=0.5, M_psi=0.5)
    rho, phi, psi = W.to_aux(*_slab(0, 1, nx, 0.5 * alpha))
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi)
    want = _tanh_slab(nx, alpha)
    errs = []
    for _ in range(3):
        oracle.step(p, f, g, k, 4000)
        C1 = oracle.fields(p, f, g, k)[0].reshape(2, nx)[0]
        errs.append(np.abs(C1 - want).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1.5e-2


@pytest.mark.parametrize("m,n", [(0, 1), (2, 0), (1, 2)])
def test_laplace_law_gives_surface_tension(m, n):
    nx = ny = 64
    radii = (10.0, 14.0, 18.0)
    dps = []
    for R in radii:
        p = oracle.make_params(9, nx, ny, 1, KAPPA, 1.0, tau_f=1.0, M_phi=0.5, M_psi=0.5)
        C1, C2, C3, rho, u = _relax(p, W.drop(nx, ny, R, m, n), 3000)

        def pb(r):
            X = np.array([rho[r], C1[r] - C2[r], C3[r]])
            return oracle.thermo_node(p, X, np.zeros(3))[2]

        dps.append(pb((ny // 2) * nx + nx // 2) - pb(0))
        assert np.abs(u).max() < 1e-4
    gamma = 1.0 * (KAPPA[m] + KAPPA[n]) / 6.0
    for R, dp in zip(radii, dps):
        assert abs(dp - gamma / R) < 0.1 * gamma / R
    inv = 1.0 / np.array(radii)
    slope = float(np.dot(inv, dps) / np.dot(inv, inv))  # least squares through the origin
    assert abs(slope - gamma) < 0.05 * gamma, (slope, gamma)


@pytest.mark.parametrize("h", [(-0.001, 0.002, 0.0), (0.0005, -0.001, 0.0)])
def test_wall_concentrations_match_cahn_roots(h):
    nx, ny, alpha = 4, 48, 1.0
    solid = W.walls_y(nx, ny, 1, 1)
    C = [np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))]
    p = oracle.make_params(9, nx, ny, 1, KAPPA, alpha, tau_f=1.0, M_phi=0.5, M_psi=0.5, h=h)
    C1, C2, C3, rho, u = _relax(p, C, 20000, solid)
    # wall value: mean of the ghost (solid row 0) and the first fluid row
    R, Ph, Ps = rho.copy(), (C1 - C2).copy(), C3.copy()
    oracle.ghosts(p, R, Ph, Ps, solid)
    Cg = [(R + Ph - Ps) / 2, (R - Ph - Ps) / 2, Ps]
    Cf = [C1, C2, C3]
    wall = [0.5 * (Cg[m].reshape(ny, nx)[0, 0] + Cf[m].reshape(ny, nx)[1, 0]) for m in range(3)]
    roots = [0.5 * (1 + np.sqrt(1 + 4 * h[0] / (alpha * KAPPA[0]))),   # fluid 1 majority
             0.5 * (1 - np.sqrt(1 - 4 * h[1] / (alpha * KAPPA[1]))),   # minorities
             0.5 * (1 - np.sqrt(1 - 4 * h[2] / (alpha * KAPPA[2])))]
    bulk = [1.0, 0.0, 0.0]
    for m in range(3):
        assert abs(wall[m] - roots[m]) <= 0.1 * abs(roots[m] - bulk[m]) + 2e-3, (m, wall, roots)
    assert np.abs(u).max() < 1e-6
