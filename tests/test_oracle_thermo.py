"""Pins of the oracle's local thermodynamics (chemical potentials, bulk pressure).

The chemical potentials are functional derivatives of the free energy
(Eq. energy_functional_general, rewritten in rho, phi, psi as
Eq. functional_newvar).  The test writes down a discrete free energy on a small
periodic lattice - bulk terms plus a lattice gradient energy whose variation is
the isotropic Laplacian - differentiates it with torch autograd, and compares
with the oracle's mu_rho, mu_phi, mu_psi.  The bulk pressure is pinned by the
thermodynamic identity p_b = sum_X X df_b/dX - f_b + rho c_s^2 that the
pressure-tensor condition of the Equations-of-Motion section implies.
The printed mu_phi, mu_psi are checked as printed; the printed mu_rho and p_b
carry misprints, and the tests record exactly what differs.
"""
import numpy as np
import pytest
import torch

import oracle

torch.set_default_dtype(torch.float64)


def _conc(rho, phi, psi):
    return [(rho + phi - psi) / 2, (rho - phi - psi) / 2, psi]


def _free_energy(X, kappa, alpha, e, w, shape):
    """Discrete F = sum_r [ sum_m kappa_m/2 C_m^2 (1-C_m)^2
                            + sum_m alpha^2 kappa_m/2 * (1/c_s^2) sum_i w_i (C_m(r+e_i)-C_m(r))^2 ]."""
    rho, phi, psi = X
    C = _conc(rho, phi, psi)
    F = sum(kappa[m] / 2 * C[m] ** 2 * (1 - C[m]) ** 2 for m in range(3)).sum()
    dims = len(shape)  # arrays are [z][y][x] or [y][x]
    for m in range(3):
        for i in range(1, len(w)):
            shifts, axes = [], []
            for a in range(dims):
                comp = e[i][a]
                if comp:
                    shifts.append(-int(comp))
                    axes.append(dims - 1 - a)
            nb = torch.roll(C[m], shifts=tuple(shifts), dims=tuple(axes)) if shifts else C[m]
            F = F + alpha ** 2 * kappa[m] / 2 * 3.0 * w[i] * ((nb - C[m]) ** 2).sum()
    return F


@pytest.mark.parametrize("Q,shape", [(9, (10, 12)), (19, (4, 5, 6))])
@pytest.mark.parametrize("alpha", [1.0, 1.5])
def test_chemical_potentials_are_functional_derivatives(Q, shape, alpha):
    rng = np.random.default_rng(7)
    kappa = (0.013, 0.021, 0.034)
    e, w, _, _ = oracle.lattice(Q)
    nz, ny, nx = (1,) + shape if len(shape) == 2 else shape
    p = oracle.make_params(Q, nx, ny, nz, kappa, alpha)
    # smooth-ish random fields around a ternary mixture
    base = [rng.uniform(0.9, 1.1, shape), rng.uniform(-0.6, 0.6, shape), rng.uniform(0.0, 0.5, shape)]
    X = [torch.tensor(b, requires_grad=True) for b in base]
    F = _free_energy(X, kappa, alpha, e, w, shape)
    F.backward()
    N = int(np.prod(shape))
    laps = [oracle.derivatives(p, b.reshape(N))[1] for b in base]
    worst = 0.0
    for r in range(N):
        Xr = np.array([base[c].reshape(N)[r] for c in range(3)])
        lr = np.array([laps[c][r] for c in range(3)])
        _, mu, _ = oracle.thermo_node(p, Xr, lr)
        want = np.array([X[c].grad.reshape(N)[r].item() for c in range(3)])
        worst = max(worst, float(np.max(np.abs(mu - want))))
    assert worst < 1e-13, worst


def _fb_torch(rho, phi, psi, kappa):
    C = _conc(rho, phi, psi)
    return sum(kappa[m] / 2 * C[m] ** 2 * (1 - C[m]) ** 2 for m in range(3))


def test_bulk_pressure_thermodynamic_identity():
    rng = np.random.default_rng(3)
    kappa = (0.011, 0.027, 0.019)
    p = oracle.make_params(9, 4, 4, 1, kappa, 1.0)
    for _ in range(200):
        x = rng.uniform([-0.2, -1.2, -0.2], [1.3, 1.2, 1.2])
        X = torch.tensor(x, requires_grad=True)
        fb = _fb_torch(X[0], X[1], X[2], kappa)
        (g,) = torch.autograd.grad(fb, X)
        want = float(((X * g).sum() - fb + X[0] / 3.0).detach())
        _, _, pb = oracle.thermo_node(p, x, np.zeros(3))
        assert abs(pb - want) < 1e-15 * max(1.0, abs(want)) + 1e-16


def _printed_pb(r, f, s, k1, k2, k3):
    """Bulk pressure polynomial exactly as printed in the Equations-of-Motion section."""
    A = (3 / 32 * r**4 + 3 / 32 * f**4 + 9 / 16 * r**2 * f**2 + 9 / 16 * r**2 * s**2
         + 9 / 16 * f**2 * s**2 - 3 / 8 * r**3 * s - 3 / 8 * r * s**3 + 3 / 4 * r**2 * s
         - 3 / 4 * r * f**2 - 3 / 4 * r * s**2 + 3 / 4 * f**2 * s - 1 / 4 * r**3 + 1 / 8 * r**2
         + 1 / 8 * f**2 - 1 / 4 * r * s - 9 / 8 * r * f**2 * s)
    B = (3 / 8 * r**3 * f + 3 / 8 * r * f**3 - 3 / 8 * f**3 * s - 3 / 8 * f * s**3 - 1 / 4 * f**3
         - 3 / 4 * r**2 * f - 3 / 4 * f * s**2 + 1 / 4 * r * f - 1 / 4 * f * s
         + 9 / 8 * r * f * s**2 - 9 / 8 * r**2 * f * s + 3 / 2 * r * f * s)
    return (r / 3 + (k1 + k2) * A + (k1 - k2) * B + 1 / 4 * (k1 + k2 - 8 * k3) * s**3
            + (k1 + k2 + 16 * k3) * (3 / 32 * s**4 + 1 / 8 * s**2))


def test_printed_bulk_pressure_differs_by_psi_squared_term():
    """The printed p_b exceeds the identity by exactly 3 kappa_3 psi^2 / 2."""
    rng = np.random.default_rng(4)
    kappa = (0.01, 0.02, 0.03)
    p = oracle.make_params(9, 4, 4, 1, kappa, 1.0)
    for _ in range(100):
        x = rng.uniform([0.8, -1.0, 0.0], [1.2, 1.0, 1.0])
        _, _, pb = oracle.thermo_node(p, x, np.zeros(3))
        printed = _printed_pb(*x, *kappa)
        assert abs(printed - 1.5 * kappa[2] * x[2] ** 2 - pb) < 1e-14


def test_printed_mu_phi_mu_psi_and_corrected_mu_rho():
    rng = np.random.default_rng(5)
    k1, k2, k3 = 0.012, 0.023, 0.031
    a = 1.3
    p = oracle.make_params(9, 4, 4, 1, (k1, k2, k3), a)
    misprint_gap = 0.0
    for _ in range(100):
        r, f, s = rng.uniform([0.8, -1.0, 0.0], [1.2, 1.0, 1.0])
        lr, lf, ls = rng.uniform(-0.1, 0.1, 3)
        _, mu, _ = oracle.thermo_node(p, np.array([r, f, s]), np.array([lr, lf, ls]))
        P1 = (r + f - s) * (r + f - s - 2) * (r + f - s - 1)
        P2 = (r - f - s) * (r - f - s - 2) * (r - f - s - 1)
        mu_phi = k1 / 8 * P1 - k2 / 8 * P2 + a**2 / 4 * ((k2 - k1) * (lr - ls) - (k1 + k2) * lf)
        mu_psi = (-k1 / 8 * P1 - k2 / 8 * P2 + k3 * s * (s - 1) * (2 * s - 1)
                  + a**2 / 4 * ((k1 + k2) * lr - (k2 - k1) * lf - (k2 + k1 + 4 * k3) * ls))
        assert abs(mu[1] - mu_phi) < 1e-15
        assert abs(mu[2] - mu_psi) < 1e-15
        # mu_rho as dF/drho: the printed form has -kappa_2 instead of +kappa_2 on the
        # bulk term and a permuted Laplacian part.
        mu_rho = k1 / 8 * P1 + k2 / 8 * P2 - a**2 / 4 * ((k1 + k2) * lr + (k1 - k2) * lf - (k1 + k2) * ls)
        assert abs(mu[0] - mu_rho) < 1e-15
        printed = k1 / 8 * P1 - k2 / 8 * P2 + a**2 / 4 * ((k1 + k2) * (ls - lf) + (k2 - k1) * lr)
        misprint_gap = max(misprint_gap, abs(printed - mu_rho))
    assert misprint_gap > 1e-3


def test_pure_phases_have_zero_potentials_and_ideal_pressure():
    p = oracle.make_params(9, 4, 4, 1, (0.01, 0.02, 0.03), 1.0)
    for C in ([1, 0, 0], [0, 1, 0], [0, 0, 1]):
        X = np.array([sum(C), C[0] - C[1], C[2]], dtype=float)
        Cout, mu, pb = oracle.thermo_node(p, X, np.zeros(3))
        assert np.allclose(Cout, C, atol=0, rtol=0)
        assert np.all(mu == 0.0)
        assert pb == 1.0 / 3.0
