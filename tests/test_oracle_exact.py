"""Brute-force pins of the oracle's whole step in exact rational arithmetic.

A second, independent restatement of one time step, written directly from the
paper's printed equations in Python ``fractions`` (no floating point), is run
on tiny lattices -- a 4x4 D2Q9 lattice with a solid wall row (wetting ghosts,
halfway bounce-back) and a periodic 3x3x3 D3Q19 lattice -- from populations
that are exactly the doubles the C oracle receives.  The C oracle's FP64 step
must agree with the exact result to rounding (1e-14 absolute on O(1) values),
which pins its stencils, equilibria, collision and streaming node by node: a
dropped term, a wrong sign, a swapped index or a transposed operand changes
the result by many orders of magnitude more.  The oracle's mass totals are
pinned against correctly rounded direct sums (math.fsum).

Equations restated (the paper's sections):
- moments: Eq. lbconstraint;
- C_1, C_2, C_3 from rho, phi, psi: Sec. Auxiliary variables;
- mu_m = kappa_m C_m (1 - C_m)(1 - 2 C_m) - alpha^2 kappa_m lap C_m
  (bulk and gradient terms of the free energy); mu_phi = (mu_1 - mu_2)/2,
  mu_psi = mu_3 - (mu_1 + mu_2)/2 (Sec. Equations of Motion);
- p_b = rho c_s^2 + sum_m kappa_m/2 C_m^2 (1 - C_m)(1 - 3 C_m) (the bulk
  pressure identity; the printed polynomial carries an extra 3 kappa_3 psi^2/2);
- kappa_XY mixing coefficients as printed under the pressure tensor;
- f_eq, g_eq, k_eq for i > 0: Eq. eqdistfbinary term by term (alpha^2 on the
  gradient terms, cross terms in their symmetric form); rest populations from
  the mass constraints; the D3Q19 weight table as printed;
- BGK: Eq. latboltCollision; propagation: Eq. latboltPropagation (pull form)
  with halfway bounce-back at solid nodes;
- wetting ghosts on solid nodes: mean over fluid axis neighbours of X(n) - G_X
  with G_X the wall-normal gradients of Sec. Auxiliary variables;
- derivatives: d_a X = (1/c_s^2) sum_i w_i e_ia X(r + e_i),
  lap X = (2/c_s^2) sum_i w_i (X(r + e_i) - X(r)).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

CS2 = Fr(1, 3)


def d2q9():
    e = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (1, 1, 0), (-1, -1, 0), (-1, 1, 0), (1, -1, 0)]
    w = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
    # components xx yy zz xy yz zx; axis link along a: w^aa = 1/9, w^bb = -1/18;
    # diagonal link: w^xx = w^yy = -1/72, w^xy = e_x e_y / 12
    t = []
    for (x, y, _) in e:
        if x == 0 and y == 0:
            t.append([Fr(0)] * 6)
        elif x * y == 0:
            t.append([Fr(1, 9) if x else Fr(-1, 18), Fr(1, 9) if y else Fr(-1, 18), 0, 0, 0, 0])
        else:
            t.append([Fr(-1, 72), Fr(-1, 72), 0, Fr(x * y, 12), 0, 0])
    return e, w, [[Fr(v) for v in row] for row in t]


def d3q19():
    e = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0),
         (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1),
         (1, 0, 1), (1, 0, -1), (-1, 0, 1), (-1, 0, -1)]
    w = [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12
    t = [[Fr(0)] * 6 for _ in range(19)]
    XX, YY, ZZ, XY, YZ, ZX = range(6)

    def put(c, idx, v):
        for i in idx:
            t[i][c] = Fr(v)
    # the weight table as printed
    put(XX, [1, 2], Fr(5, 36)); put(YY, [3, 4], Fr(5, 36)); put(ZZ, [5, 6], Fr(5, 36))
    put(XX, [3, 4, 5, 6], Fr(-1, 9)); put(YY, [1, 2, 5, 6], Fr(-1, 9)); put(ZZ, [1, 2, 3, 4], Fr(-1, 9))
    put(XX, list(range(7, 11)) + list(range(15, 19)), Fr(-1, 72))
    put(YY, range(7, 15), Fr(-1, 72)); put(ZZ, range(11, 19), Fr(-1, 72))
    put(XX, range(11, 15), Fr(1, 36)); put(YY, range(15, 19), Fr(1, 36)); put(ZZ, range(7, 11), Fr(1, 36))
    put(XY, [7, 10], Fr(1, 12)); put(YZ, [11, 14], Fr(1, 12)); put(ZX, [15, 18], Fr(1, 12))
    put(XY, [8, 9], Fr(-1, 12)); put(YZ, [12, 13], Fr(-1, 12)); put(ZX, [16, 17], Fr(-1, 12))
    return e, w, t


def opposite(e, i):
    return e.index(tuple(-c for c in e[i]))


class Exact:
    """One step of the method in exact arithmetic on an nx x ny x nz lattice."""

    def __init__(self, Q, shape, p, solid=None):
        self.e, self.w, self.t = d2q9() if Q == 9 else d3q19()
        self.Q = Q
        self.nx, self.ny, self.nz = shape
        self.N = self.nx * self.ny * self.nz
        self.solid = [False] * self.N if solid is None else [bool(s) for s in np.asarray(solid).reshape(-1)]
        self.kap = [Fr(p.kappa[m]) for m in range(3)]
        self.a2 = Fr(p.alpha) * Fr(p.alpha)
        self.tau = [Fr(p.tau[s]) for s in range(3)]
        self.gam = [Fr(p.gamma[0]), Fr(p.gamma[1])]
        h = [Fr(p.h[m]) for m in range(3)]
        q = [h[m] / (self.a2 * self.kap[m]) for m in range(3)]
        self.G = [-q[0] - q[1] - q[2], -q[0] + q[1], -q[2]]  # d_n rho, phi, psi at the wall
        k1, k2, k3 = self.kap
        self.K = {(0, 0): (k1 + k2) / 4, (1, 1): (k1 + k2) / 4, (2, 2): (k1 + k2 + 4 * k3) / 4,
                  (0, 1): (k1 - k2) / 4, (1, 2): -(k1 - k2) / 4, (0, 2): -(k1 + k2) / 4}

    def nb(self, r, i, sign=+1):
        x, rest = r % self.nx, r // self.nx
        y, z = rest % self.ny, rest // self.ny
        ex, ey, ez = self.e[i]
        return ((x + sign * ex) % self.nx) + self.nx * (((y + sign * ey) % self.ny) + self.ny * ((z + sign * ez) % self.nz))

    def step(self, pops):
        Q, N, e, w, t = self.Q, self.N, self.e, self.w, self.t
        fluid = [not s for s in self.solid]
        # moments
        X = [[Fr(0)] * N for _ in range(3)]
        j = [[Fr(0)] * 3 for _ in range(N)]
        for r in range(N):
            if not fluid[r]:
                continue
            for s in range(3):
                X[s][r] = sum((pops[s][i][r] for i in range(Q)), Fr(0))
            for a in range(3):
                j[r][a] = sum((pops[0][i][r] * e[i][a] for i in range(Q)), Fr(0))
        # wetting ghosts: mean over fluid axis neighbours of X(n) - G_X
        naxis = 4 if Q == 9 else 6
        for r in range(N):
            if fluid[r]:
                continue
            ns = [self.nb(r, i) for i in range(1, naxis + 1) if fluid[self.nb(r, i)]]
            for s in range(3):
                X[s][r] = (sum((X[s][n] - self.G[s] for n in ns), Fr(0)) / len(ns)) if ns else Fr(0)
        # collision at fluid nodes
        post = [[[Fr(0)] * N for _ in range(Q)] for _ in range(3)]
        for r in range(N):
            if not fluid[r]:
                continue
            grad = [[sum((w[i] * e[i][a] * X[s][self.nb(r, i)] for i in range(1, Q)), Fr(0)) / CS2
                     for a in range(3)] for s in range(3)]
            lap = [2 * sum((w[i] * (X[s][self.nb(r, i)] - X[s][r]) for i in range(1, Q)), Fr(0)) / CS2
                   for s in range(3)]
            rho, phi, psi = X[0][r], X[1][r], X[2][r]
            u = [j[r][a] / rho for a in range(3)]
            C = [(rho + phi - psi) / 2, (rho - phi - psi) / 2, psi]
            lC = [(lap[0] + lap[1] - lap[2]) / 2, (lap[0] - lap[1] - lap[2]) / 2, lap[2]]
            mu = [self.kap[m] * C[m] * (1 - C[m]) * (1 - 2 * C[m]) - self.a2 * self.kap[m] * lC[m] for m in range(3)]
            mu_phi = (mu[0] - mu[1]) / 2
            mu_psi = mu[2] - (mu[0] + mu[1]) / 2
            pb = rho * CS2 + sum((self.kap[m] / 2 * C[m] ** 2 * (1 - C[m]) * (1 - 3 * C[m]) for m in range(3)), Fr(0))
            comp = {"xx": (0, 0), "yy": (1, 1), "zz": (2, 2), "xy": (0, 1), "yz": (1, 2), "zx": (2, 0)}
            cidx = {"xx": 0, "yy": 1, "zz": 2, "xy": 3, "yz": 4, "zx": 5}
            eq = [[Fr(0)] * Q for _ in range(3)]
            for i in range(1, Q):
                eu = sum((e[i][a] * u[a] for a in range(3)), Fr(0))
                uu = sum((u[a] * u[a] for a in range(3)), Fr(0))
                vv = [eu * eu - CS2 * uu]  # v_a v_b (e_a e_b - c_s^2 delta_ab)
                fe = w[i] * (pb / CS2 + rho * eu / CS2 + rho * vv[0] / (2 * CS2 * CS2))
                # Eq. eqdistfbinary, pair by pair (X, Y), with alpha^2 on every gradient term
                for (a_, b_), kXY in self.K.items():
                    Xa, Xb = X[a_][r], X[b_][r]
                    if a_ == b_:
                        fe -= self.a2 * w[i] / CS2 * kXY * Xa * lap[a_]
                        for c, (p1, p2) in comp.items():
                            fe += self.a2 * kXY / CS2 * t[i][cidx[c]] * grad[a_][p1] * grad[a_][p2]
                    else:
                        fe -= self.a2 * w[i] / CS2 * kXY * (Xa * lap[b_] + Xb * lap[a_])
                        for c in ("xx", "yy", "zz"):
                            p1 = comp[c][0]
                            fe += self.a2 * 2 * kXY / CS2 * t[i][cidx[c]] * grad[a_][p1] * grad[b_][p1]
                        for c in ("xy", "yz", "zx"):
                            p1, p2 = comp[c]
                            fe += self.a2 * kXY / CS2 * t[i][cidx[c]] * (grad[a_][p1] * grad[b_][p2] +
                                                                          grad[a_][p2] * grad[b_][p1])
                ge = w[i] * (self.gam[0] * mu_phi / CS2 + phi * eu / CS2 + phi * vv[0] / (2 * CS2 * CS2))
                ke = w[i] * (self.gam[1] * mu_psi / CS2 + psi * eu / CS2 + psi * vv[0] / (2 * CS2 * CS2))
                eq[0][i], eq[1][i], eq[2][i] = fe, ge, ke
            for s, M in enumerate((rho, phi, psi)):
                eq[s][0] = M - sum(eq[s][1:], Fr(0))
                for i in range(Q):
                    x = pops[s][i][r]
                    post[s][i][r] = x - (x - eq[s][i]) / self.tau[s]
        # propagation (pull) with halfway bounce-back
        out = [[[Fr(0)] * N for _ in range(Q)] for _ in range(3)]
        for r in range(N):
            if not fluid[r]:
                continue
            for i in range(Q):
                src = self.nb(r, i, -1)
                for s in range(3):
                    out[s][i][r] = post[s][i][src] if fluid[src] else post[s][opposite(e, i)][r]
        return out


def _random_state(Q, N, solid, seed):
    rng = np.random.default_rng(seed)
    _, w, _ = d2q9() if Q == 9 else d3q19()
    w = np.array([float(v) for v in w])
    f = w[:, None] * (1.0 + rng.uniform(-0.2, 0.2, (Q, N)))
    g = w[:, None] * rng.uniform(-0.5, 0.5, (Q, N))
    k = w[:, None] * (0.3 + rng.uniform(-0.2, 0.2, (Q, N)))
    if solid is not None:
        for a in (f, g, k):
            a[:, np.asarray(solid).reshape(-1) != 0] = 0.0
    return [np.ascontiguousarray(a) for a in (f, g, k)]


CASES = [
    # Q, shape, kappa, h, solid rows (y indices), seed
    (9, (4, 4, 1), (0.1, 0.2, 0.3), (0.004, -0.012, 0.02), [0], 1),
    (9, (4, 4, 1), (0.05, 0.2, 0.15), (0.0, 0.0, 0.0), None, 2),
    (19, (3, 3, 3), (0.1, 0.2, 0.3), (0.0, 0.0, 0.0), None, 3),
]


@pytest.mark.parametrize("Q,shape,kappa,h,rows,seed", CASES)
def test_oracle_step_equals_exact_rational_step(Q, shape, kappa, h, rows, seed):
    nx, ny, nz = shape
    solid = None
    if rows is not None:
        solid = np.zeros((nz, ny, nx), dtype=np.uint8)
        for y in rows:
            solid[:, y, :] = 1
    p = oracle.make_params(Q, nx, ny, nz, kappa, 1.0, 0.9, 0.1, 0.15, h)
    N = nx * ny * nz
    f, g, k = _random_state(Q, N, solid, seed)
    exact_in = [[[Fr(float(v)) for v in a[i]] for i in range(Q)] for a in (f, g, k)]
    want = Exact(Q, shape, p, solid).step(exact_in)
    oracle.step(p, f, g, k, 1, solid)
    worst = 0.0
    for s, got in enumerate((f, g, k)):
        for i in range(Q):
            for r in range(N):
                worst = max(worst, abs(got[i][r] - float(want[s][i][r])))
    print("max |oracle - exact| =", worst)
    assert worst <= 1e-14


def test_exact_step_sees_a_planted_mistake():
    """The comparison above has teeth: the exact step with one gradient-term
    coefficient changed by 1 % (kappa_rho_phi) differs from the oracle far beyond
    the 1e-14 bound."""
    Q, shape = 9, (4, 4, 1)
    p = oracle.make_params(Q, *shape, (0.1, 0.2, 0.3), 1.0, 0.9, 0.1, 0.15)
    f, g, k = _random_state(Q, 16, None, 5)
    ex = Exact(Q, shape, p)
    ex.K[(0, 1)] *= Fr(101, 100)
    want = ex.step([[[Fr(float(v)) for v in a[i]] for i in range(Q)] for a in (f, g, k)])
    oracle.step(p, f, g, k, 1)
    worst = max(abs(f[i][r] - float(want[0][i][r])) for i in range(Q) for r in range(16))
    assert worst > 1e-9


@pytest.mark.parametrize("walls", [False, True])
def test_oracle_mass_equals_direct_sum(walls):
    Q, nx, ny = 9, 23, 17
    solid = None
    if walls:
        solid = np.zeros((ny, nx), dtype=np.uint8)
        solid[0, :] = solid[-1, :] = 1
        solid[5:9, 4:11] = 1
    p = oracle.make_params(Q, nx, ny, 1, (0.01, 0.02, 0.03))
    f, g, k = _random_state(Q, nx * ny, solid, 11)
    # nonzero populations on solid nodes must not count
    if solid is not None:
        m = solid.reshape(-1) != 0
        for a in (f, g, k):
            a[:, m] = 7.0
    got = oracle.mass(p, f, g, k, solid)
    keep = np.ones(nx * ny, bool) if solid is None else solid.reshape(-1) == 0
    for s, a in enumerate((f, g, k)):
        want = math.fsum(float(v) for v in a[:, keep].reshape(-1))
        assert abs(got[s] - want) <= 4 * np.spacing(abs(want)), (s, got[s], want)
