"""Pins of the oracle's equilibria through the moments the paper requires of them.

The equilibria of the LBM section must satisfy (Chapman-Enskog requirements,
mass constraints that close the section):
  sum_i f_eq = rho,  sum_i f_eq e = rho v,  sum_i f_eq e e = P + rho v v,
  sum_i g_eq = phi,  sum_i g_eq e = phi v,  sum_i g_eq e e = Gamma_phi mu_phi I + phi v v,
and likewise for k_eq with psi, mu_psi.  P is the pressure tensor of the
Equations-of-Motion section.  The test builds P itself: mixing coefficients
from the quadratic form of the gradient energy under C = A X (Sec. Auxiliary
variables), p_b and mu from autograd of the bulk free energy.  Nothing here
reuses the oracle's own formulas.
"""
import numpy as np
import pytest
import torch

import oracle

torch.set_default_dtype(torch.float64)

A = np.array([[0.5, 0.5, -0.5], [0.5, -0.5, -0.5], [0.0, 0.0, 1.0]])  # C = A @ (rho, phi, psi)


def _mixing(kappa):
    return sum(kappa[m] * np.outer(A[m], A[m]) for m in range(3))


def _bulk_parts(X, kappa):
    Xt = torch.tensor(X, requires_grad=True)
    C = [sum(A[m, c] * Xt[c] for c in range(3)) for m in range(3)]
    fb = sum(kappa[m] / 2 * C[m] ** 2 * (1 - C[m]) ** 2 for m in range(3))
    (g,) = torch.autograd.grad(fb, Xt)
    g = g.detach().numpy()
    pb = float(np.dot(X, g) - fb.item() + X[0] / 3.0)
    return g, pb


@pytest.mark.parametrize("Q,D", [(9, 2), (19, 3)])
@pytest.mark.parametrize("alpha", [1.0, 1.7])
def test_equilibrium_moments(Q, D, alpha):
    rng = np.random.default_rng(11 + Q)
    kappa = (0.013, 0.029, 0.017)
    gam = (0.7, 1.3)
    p = oracle.make_params(Q, 4, 4, 1 if Q == 9 else 4, kappa, alpha, tau_f=0.9,
                           gamma_phi=gam[0], gamma_psi=gam[1])
    e, _, _, _ = oracle.lattice(Q)
    K = _mixing(kappa)
    a2 = alpha * alpha
    for _ in range(40):
        X = rng.uniform([0.9, -1.0, 0.0], [1.1, 1.0, 1.0])
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.05, 0.05, D)
        j = X[0] * u
        grad = np.zeros((3, 3))
        grad[:, :D] = rng.uniform(-0.2, 0.2, (3, D))
        lap = rng.uniform(-0.05, 0.05, 3)
        feq, geq, keq = oracle.equilibrium_node(p, X, j, grad, lap)
        dfb, pb = _bulk_parts(X, kappa)
        mu = dfb - a2 * K @ lap  # mu_X = df_b/dX - alpha^2 sum_Y K_XY lap Y
        # pressure tensor (Equations-of-Motion section), symmetric sum over X, Y
        P = pb * np.eye(3)
        for x in range(3):
            for y in range(3):
                P += a2 * K[x, y] * (np.outer(grad[x], grad[y])
                                     - 0.5 * np.dot(grad[x], grad[y]) * np.eye(3)
                                     - X[x] * lap[y] * np.eye(3))
        M0 = lambda d: d.sum()
        M1 = lambda d: e.T.astype(float) @ d
        M2 = lambda d: np.einsum("i,ia,ib->ab", d, e.astype(float), e.astype(float))
        sl = slice(0, D)
        assert abs(M0(feq) - X[0]) < 1e-14
        assert np.allclose(M1(feq), j, atol=1e-14, rtol=0)
        assert np.allclose(M2(feq)[sl, sl], (P + X[0] * np.outer(u, u))[sl, sl], atol=1e-13, rtol=0)
        for d_, val, mu_x, G in ((geq, X[1], mu[1], gam[0]), (keq, X[2], mu[2], gam[1])):
            assert abs(M0(d_) - val) < 1e-14
            assert np.allclose(M1(d_), val * u, atol=1e-14, rtol=0)
            want = G * mu_x * np.eye(3) + val * np.outer(u, u)
            assert np.allclose(M2(d_)[sl, sl], want[sl, sl], atol=1e-13, rtol=0)


def test_equilibrium_at_rest_uniform_is_weighted_density():
    """A uniform pure phase at rest has f_eq = w_i rho (p_b = rho c_s^2); with zero
    chemical potential g_eq and k_eq vanish at i > 0 and the rest population
    carries all of phi and psi."""
    for Q in (9, 19):
        e, w, _, _ = oracle.lattice(Q)
        p = oracle.make_params(Q, 4, 4, 1 if Q == 9 else 4, (0.01, 0.02, 0.03), 1.0)
        for C in ([1, 0, 0], [0, 1, 0], [0, 0, 1]):
            X = np.array([sum(C), C[0] - C[1], C[2]], dtype=float)
            feq, geq, keq = oracle.equilibrium_node(p, X, np.zeros(3), np.zeros((3, 3)), np.zeros(3))
            assert np.allclose(feq, w * X[0], atol=1e-15, rtol=0)
            assert np.allclose(geq[1:], 0.0, atol=1e-16) and abs(geq[0] - X[1]) < 1e-15
            assert np.allclose(keq[1:], 0.0, atol=1e-16) and abs(keq[0] - X[2]) < 1e-15
