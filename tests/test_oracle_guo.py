"""Pins of the oracle's forcing coupling (orc_step_guo): the body-force
alternative to the pressure-tensor coupling that Sec. Equations of Motion
names (Guo forcing).  The force is the divergence of the paper's pressure
tensor minus the ideal-gas pressure, F_a = -d_b (P_ab - rho c_s^2 delta_ab),
which the paper's identity makes -(rho grad mu_rho + phi grad mu_phi + psi
grad mu_psi) in the continuum; the source is that of Guo, Zheng and Shi (2002).

- one step in exact rational arithmetic (an independent restatement in Python
  fractions) equals the C oracle to rounding;
- the force equals the analytic -(sum_X X grad mu_X) for smooth periodic
  fields (calculus on trigonometric fields against the discrete stencils,
  O(k^2) apart), which pins the identity and the pressure tensor together;
- every step conserves sum rho, sum phi, sum psi, changes the total momentum
  by exactly the total force (the half-force velocity shift and the source
  together), and the total force vanishes (the divergence form);
- a flat 1/2 interface relaxes to the same profile as under the
  pressure-tensor coupling, within the lattice error of Eq. tanh, and a lens
  to nearly the same fields (both minimise the same free energy).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_1511_02155_gb300 import workloads as W
from test_oracle_exact import CS2, Exact, _random_state


def exact_step_guo(ex, pops):
    """One forcing-coupling step of Exact's lattice (periodic) in fractions."""
    Q, N, e, w = ex.Q, ex.N, ex.e, ex.w
    X = [[sum((pops[s][i][r] for i in range(Q)), Fr(0)) for r in range(N)] for s in range(3)]
    j = [[sum((pops[0][i][r] * e[i][a] for i in range(Q)), Fr(0)) for a in range(3)] for r in range(N)]

    def lap(field, r):
        return 2 * sum((w[i] * (field[ex.nb(r, i)] - field[r]) for i in range(1, Q)), Fr(0)) / CS2

    def grad(field, r):
        return [sum((w[i] * e[i][a] * field[ex.nb(r, i)] for i in range(1, Q)), Fr(0)) / CS2 for a in range(3)]

    mu = [[Fr(0)] * N for _ in range(3)]
    for r in range(N):
        rho, phi, psi = X[0][r], X[1][r], X[2][r]
        L = [lap(X[s], r) for s in range(3)]
        C = [(rho + phi - psi) / 2, (rho - phi - psi) / 2, psi]
        lC = [(L[0] + L[1] - L[2]) / 2, (L[0] - L[1] - L[2]) / 2, L[2]]
        m = [ex.kap[c] * C[c] * (1 - C[c]) * (1 - 2 * C[c]) - ex.a2 * ex.kap[c] * lC[c] for c in range(3)]
        mu[0][r], mu[1][r], mu[2][r] = (m[0] + m[1]) / 2, (m[0] - m[1]) / 2, m[2] - (m[0] + m[1]) / 2
    # non-ideal pressure tensor P_ab - rho c_s^2 delta_ab at every node, from the
    # printed tensor (alpha^2 on the gradient terms, symmetric cross terms)
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]
    Pi = [[Fr(0)] * N for _ in range(6)]
    for r in range(N):
        gX = [grad(X[s], r) for s in range(3)]
        LX = [lap(X[s], r) for s in range(3)]
        rho, phi, psi = X[0][r], X[1][r], X[2][r]
        C = [(rho + phi - psi) / 2, (rho - phi - psi) / 2, psi]
        pb = rho * CS2 + sum((ex.kap[m] / 2 * C[m] ** 2 * (1 - C[m]) * (1 - 3 * C[m]) for m in range(3)), Fr(0))
        for c, (al, be) in enumerate(comps):
            v = (pb - rho * CS2) if al == be else Fr(0)
            for (x, y), kxy in ex.K.items():
                if x == y:
                    v += ex.a2 * kxy * (gX[x][al] * gX[x][be])
                    if al == be:
                        v -= ex.a2 * kxy * (sum((gX[x][d] ** 2 for d in range(3)), Fr(0)) / 2 + X[x][r] * LX[x])
                else:
                    v += ex.a2 * kxy * (gX[x][al] * gX[y][be] + gX[y][al] * gX[x][be])
                    if al == be:
                        v -= ex.a2 * kxy * (sum((gX[x][d] * gX[y][d] for d in range(3)), Fr(0))
                                            + X[x][r] * LX[y] + X[y][r] * LX[x])
            Pi[c][r] = v
    idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (1, 2): 4, (2, 1): 4, (2, 0): 5, (0, 2): 5}
    post = [[[Fr(0)] * N for _ in range(Q)] for _ in range(3)]
    for r in range(N):
        F = [-sum((grad(Pi[idx[(a, b)]], r)[b] for b in range(3)), Fr(0)) for a in range(3)]
        rho = X[0][r]
        u = [(j[r][a] + F[a] / 2) / rho for a in range(3)]
        uu = sum((ua * ua for ua in u), Fr(0))
        eq = [[Fr(0)] * Q for _ in range(3)]
        for i in range(1, Q):
            eu = sum((e[i][a] * u[a] for a in range(3)), Fr(0))
            quad = (eu * eu - CS2 * uu) / (2 * CS2 * CS2)
            eq[0][i] = w[i] * rho * (1 + eu / CS2 + quad)
            eq[1][i] = w[i] * (ex.gam[0] * mu[1][r] / CS2 + X[1][r] * eu / CS2 + X[1][r] * quad)
            eq[2][i] = w[i] * (ex.gam[1] * mu[2][r] / CS2 + X[2][r] * eu / CS2 + X[2][r] * quad)
        for s in range(3):
            eq[s][0] = X[s][r] - sum(eq[s][1:], Fr(0))
        pref = 1 - 1 / (2 * ex.tau[0])
        for i in range(Q):
            eu = sum((e[i][a] * u[a] for a in range(3)), Fr(0))
            eF = sum((e[i][a] * F[a] for a in range(3)), Fr(0))
            uF = sum((u[a] * F[a] for a in range(3)), Fr(0))
            S = pref * w[i] * ((eF - uF) / CS2 + eu * eF / (CS2 * CS2))
            for s in range(3):
                x = pops[s][i][r]
                post[s][i][r] = x - (x - eq[s][i]) / ex.tau[s] + (S if s == 0 else 0)
    return [[[post[s][i][ex.nb(r, i, -1)] for r in range(N)] for i in range(Q)] for s in range(3)]


@pytest.mark.parametrize("Q,shape,kappa,seed", [(9, (4, 4, 1), (0.1, 0.2, 0.3), 21),
                                                (19, (3, 3, 3), (0.1, 0.2, 0.3), 22)])
def test_guo_step_equals_exact_rational_step(Q, shape, kappa, seed):
    nx, ny, nz = shape
    p = oracle.make_params(Q, nx, ny, nz, kappa, 1.0, 0.9, 0.1, 0.15)
    N = nx * ny * nz
    f, g, k = _random_state(Q, N, None, seed)
    want = exact_step_guo(Exact(Q, shape, p), [[[Fr(float(v)) for v in a[i]] for i in range(Q)] for a in (f, g, k)])
    oracle.step_guo(p, f, g, k, 1)
    worst = max(abs(a[i][r] - float(want[s][i][r])) for s, a in enumerate((f, g, k)) for i in range(Q)
                for r in range(N))
    print("max |oracle - exact| =", worst)
    assert worst <= 1e-14


def test_force_equals_analytic_value_for_smooth_fields():
    """rho, phi, psi varying as cosines along x on a 256-long periodic lattice:
    mu_m and its gradient in closed form (second and third derivatives of the
    trigonometric C_m), against the oracle's discrete force."""
    n, ny = 256, 4
    kap, alpha = (0.02, 0.03, 0.05), 1.3
    kx = 2 * np.pi / n
    x = np.arange(n, dtype=np.float64)
    amp = {"rho": (1.0, 0.01, 0.0), "phi": (0.1, 0.4, 0.3), "psi": (0.3, 0.25, -0.2)}

    def field(name, d=0):
        c0, a, b = amp[name]  # c0 + a cos(kx) + b sin(kx) and its d-th derivative
        v = [a * np.cos(kx * x) + b * np.sin(kx * x), -a * kx * np.sin(kx * x) + b * kx * np.cos(kx * x)]
        v += [-kx * kx * v[0], -kx * kx * v[1]]
        return (c0 if d == 0 else 0.0) + v[d]

    X = [np.stack([field(nm, d) for d in range(4)]) for nm in ("rho", "phi", "psi")]
    C = [(X[0] + X[1] - X[2]) / 2, (X[0] - X[1] - X[2]) / 2, X[2]]
    dmu = []
    for m in range(3):
        c, c1, c3 = C[m][0], C[m][1], C[m][3]
        # mu_m = kappa (c - 3c^2 + 2c^3) - alpha^2 kappa c''  ->  d/dx
        dmu.append(kap[m] * (1 - 6 * c + 6 * c * c) * c1 - alpha ** 2 * kap[m] * c3)
    dmu_rho = (dmu[0] + dmu[1]) / 2
    dmu_phi = (dmu[0] - dmu[1]) / 2
    dmu_psi = dmu[2] - (dmu[0] + dmu[1]) / 2
    Fx = -(X[0][0] * dmu_rho + X[1][0] * dmu_phi + X[2][0] * dmu_psi)
    p = oracle.make_params(9, n, ny, 1, kap, alpha)
    F = oracle.force(p, *[np.tile(Xc[0], (ny, 1)) for Xc in X])
    got = F[0].reshape(ny, n)
    scale = np.abs(Fx).max()
    assert np.abs(got - Fx[None, :]).max() <= 2e-3 * scale
    assert np.abs(F[1]).max() <= 1e-15 and np.abs(F[2]).max() == 0.0


@pytest.mark.parametrize("Q,shape", [(9, (24, 18, 1)), (19, (8, 7, 6))])
def test_guo_step_conserves_mass_and_balances_momentum(Q, shape):
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    C = W.spinodal(sh, seed=31, amp=0.2)
    p = oracle.make_params(Q, nx, ny, nz, (0.05, 0.08, 0.06), 1.0, 0.8, 0.2, 0.3)
    f, g, k = oracle.init_equilibrium_guo(p, *W.to_aux(*C))
    m0 = oracle.mass(p, f, g, k)
    for _ in range(5):
        rho, j, phi, psi = oracle.moments(p, f, g, k)
        F = oracle.force(p, rho, phi, psi)
        oracle.step_guo(p, f, g, k, 1)
        j1 = oracle.moments(p, f, g, k)[1]
        for a in range(3):
            assert abs(j1[a].sum() - j[a].sum() - F[a].sum()) <= 1e-13 * max(1.0, np.abs(F[a]).sum())
            assert abs(F[a].sum()) <= 1e-13 * max(1.0, np.abs(F[a]).sum())
    assert np.allclose(oracle.mass(p, f, g, k), m0, rtol=0, atol=1e-12 * np.prod(shape))


def test_guo_flat_interface_relaxes_to_tanh():
    """Started from a profile twice as sharp, the flat interface relaxes toward
    Eq. tanh exactly as under the pressure-tensor coupling (same discrete
    equilibrium to 1e-4); started from Eq. tanh it stays within the lattice
    error of the pressure-tensor pin (1e-2 at alpha = 1)."""
    nx, ny, alpha = 64, 4, 1.0
    C = W.flat_interfaces(nx, ny, 0, 1, alpha)
    C0 = W.flat_interfaces(nx, ny, 0, 1, alpha / 2)
    p = oracle.make_params(9, nx, ny, 1, (0.01, 0.01, 0.01), alpha, 1.0, 0.5, 0.5)
    a = oracle.init_equilibrium_guo(p, *W.to_aux(*C0))
    b = oracle.init_equilibrium(p, *W.to_aux(*C0))
    oracle.step_guo(p, *a, 6000)
    oracle.step(p, *b, 6000)
    ca = oracle.fields(p, *a)[0].reshape(ny, nx)[0]
    cb = oracle.fields(p, *b)[0].reshape(ny, nx)[0]
    assert np.abs(ca - cb).max() <= 1e-4
    assert np.abs(ca - C[0][0]).max() < 0.2 * np.abs(C0[0][0] - C[0][0]).max()
    f, g, k = oracle.init_equilibrium_guo(p, *W.to_aux(*C))
    oracle.step_guo(p, f, g, k, 4000)
    C1 = oracle.fields(p, f, g, k)[0]
    assert np.abs(C1.reshape(ny, nx)[0] - C[0][0]).max() <= 1e-2
    # the fluid velocity under Guo forcing is (j + F/2)/rho: at rest the
    # stored momentum balances half the force and the velocity vanishes
    rho, j, phi, psi = oracle.moments(p, f, g, k)
    F = oracle.force(p, rho, phi, psi)
    u = (np.asarray(j) + np.asarray(F) / 2) / rho
    print("flat interface max |u| =", np.abs(u).max(), "max |F| =", np.abs(F).max())
    assert np.abs(u).max() < 1e-7 and np.abs(F).max() > 1e-5


def test_guo_lens_matches_pressure_tensor_lens():
    kap = (0.01, 0.02, 0.03)
    C = W.lens(48, 40, 8.0, 1.0, 10.0, 30.0, (24.0, 30.0))
    p = oracle.make_params(9, 48, 40, 1, kap, 1.0, 1.0, 0.1, 0.1)
    r = W.to_aux(*C)
    a = oracle.init_equilibrium_guo(p, *r)
    b = oracle.init_equilibrium(p, *r)
    oracle.step_guo(p, *a, 3000)
    oracle.step(p, *b, 3000)
    Ca, Cb = oracle.fields(p, *a), oracle.fields(p, *b)
    d = max(float(np.abs(x - y).max()) for x, y in zip(Ca[:3], Cb[:3]))
    print("max |C(guo) - C(pressure tensor)| =", d, "max |u|", np.abs(Ca[4]).max())
    assert d <= 1e-2
    assert np.abs(Ca[4]).max() < 1e-3
