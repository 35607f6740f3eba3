"""Differentiable FP64 restatement of the oracle's step, for checking adjoints.

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The same step as ``tlbm_oracle.c`` (moments, wetting ghosts, isotropic
derivatives, thermodynamics, equilibria, BGK, pull streaming with halfway
bounce-back; conventional populations f_i(r, t)), written with plain PyTorch
CPU tensor operations in float64 so that torch.autograd gives the exact
gradient of a loss with respect to kappa_m, the wetting parameters h_m and the
initial fields.  Every formula is the one the C oracle uses (same readings);
the C oracle's forward result pins this one (tests), and central finite
differences of the C oracle pin the gradients.

Loss used throughout: L = sum over fluid nodes of (C_3(r, T) - target(r))^2
after T steps from the equilibrium of the initial fields (u = 0).
"""
from __future__ import annotations

import numpy as np
import torch

from . import lattice as _lattice

_DT = torch.float64


class Geometry:
    """Neighbour tables and wetting-ghost stencils of one lattice + solid mask."""

    def __init__(self, Q, nx, ny, nz, solid=None):
        self.Q, self.nx, self.ny, self.nz = Q, nx, ny, nz
        self.N = N = nx * ny * nz
        e, w, t, opp = _lattice(Q)
        self.e = e
        self.w = torch.tensor(w, dtype=_DT)
        self.t = torch.tensor(t, dtype=_DT)
        self.opp = np.asarray(opp)
        r = np.arange(N)
        x, y, z = r % nx, (r // nx) % ny, r // (nx * ny)

        def idx(dx, dy, dz):
            return ((x + dx) % nx) + nx * (((y + dy) % ny) + ny * ((z + dz) % nz))

        self.nb = np.stack([idx(*e[i]) for i in range(Q)])        # r + e_i
        self.src = np.stack([idx(*(-e[i])) for i in range(Q)])    # r - e_i
        s = np.zeros(N, dtype=bool) if solid is None else (np.asarray(solid).reshape(-1) != 0)
        self.solid = s
        self.fluid_t = torch.tensor(~s, dtype=_DT)
        # halfway bounce-back: population i of r comes from r - e_i, or from opp(i) at r
        self.bounce = np.stack([s[self.src[i]] for i in range(Q)])
        # wetting ghosts: X(s) = sum_b c_sb X(b) - g_s G, over fluid axis neighbours b
        # (coefficient 1/n), else over fluid diagonal neighbours (g_s = sqrt 2)
        naxis = 4 if Q == 9 else 6
        S, B, C = [], [], []
        gs = np.zeros(N)
        for rr in np.nonzero(s)[0]:
            nbs = [self.nb[i][rr] for i in range(1, naxis + 1) if not s[self.nb[i][rr]]]
            coef = 1.0
            if not nbs:
                nbs = [self.nb[i][rr] for i in range(naxis + 1, Q) if not s[self.nb[i][rr]]]
                coef = np.sqrt(2.0)
            if nbs:
                for b in nbs:
                    S.append(rr)
                    B.append(b)
                    C.append(1.0 / len(nbs))
                gs[rr] = coef
        self.gS = torch.tensor(S, dtype=torch.long)
        self.gB = torch.tensor(B, dtype=torch.long)
        self.gC = torch.tensor(C, dtype=_DT)
        self.gcoef = torch.tensor(gs, dtype=_DT)


def _mixing(kappa):
    k1, k2, k3 = kappa[0], kappa[1], kappa[2]
    return [[(k1 + k2) / 4, (k1 - k2) / 4, -(k1 + k2) / 4],
            [(k1 - k2) / 4, (k1 + k2) / 4, -(k1 - k2) / 4],
            [-(k1 + k2) / 4, -(k1 - k2) / 4, (k1 + k2 + 4 * k3) / 4]]


def wetting_gradients(kappa, h, alpha):
    """G_rho, G_phi, G_psi (Sec. Auxiliary variables, wall-normal gradients)."""
    a2 = alpha * alpha
    q = [h[m] / (a2 * kappa[m]) for m in range(3)]
    return [-q[0] - q[1] - q[2], -q[0] + q[1], -q[2]]


def ghosts(G: Geometry, X, Gw):
    """X (fluid values, zeros on solids) with ghost values on solid nodes."""
    if len(G.gS) == 0:
        return X
    out = []
    for c in range(3):
        v = torch.zeros(G.N, dtype=_DT).index_add(0, G.gS, G.gC * X[c][G.gB])
        out.append(X[c] + v - G.gcoef * Gw[c])
    return out


def derivatives(G: Geometry, Xc):
    """(grad[3], lap) of one field: 3 sum w_i e_i X(r+e_i), 6 sum w_i (X(r+e_i) - X(r))."""
    grad = [torch.zeros(G.N, dtype=_DT) for _ in range(3)]
    lap = torch.zeros(G.N, dtype=_DT)
    for i in range(1, G.Q):
        xn = Xc[G.nb[i]]
        for a in range(3):
            if G.e[i][a]:
                grad[a] = grad[a] + G.w[i] * G.e[i][a] * xn
        lap = lap + G.w[i] * (xn - Xc)
    return [3.0 * g for g in grad], 6.0 * lap


def equilibria(G: Geometry, kappa, alpha, gamma, X, j):
    """feq, geq, keq ([Q] lists of [N]) at every node from X (with ghosts) and j."""
    cs2 = 1.0 / 3.0
    a2 = alpha * alpha
    rho, phi, psi = X
    der = [derivatives(G, X[c]) for c in range(3)]
    grad = [d[0] for d in der]
    lap = [d[1] for d in der]
    C = [(rho + phi - psi) / 2, (rho - phi - psi) / 2, psi]
    lC = [(lap[0] + lap[1] - lap[2]) / 2, (lap[0] - lap[1] - lap[2]) / 2, lap[2]]
    muC = [kappa[m] * C[m] * (1 - C[m]) * (1 - 2 * C[m]) - a2 * kappa[m] * lC[m] for m in range(3)]
    mu_phi = (muC[0] - muC[1]) / 2
    mu_psi = muC[2] - (muC[0] + muC[1]) / 2
    pb = rho / 3
    for m in range(3):
        pb = pb + kappa[m] / 2 * C[m] * C[m] * (1 - C[m]) * (1 - 3 * C[m])
    K = _mixing(kappa)
    safe = torch.where(G.fluid_t > 0, rho, torch.ones_like(rho))
    u = [j[a] / safe for a in range(3)]
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    Lap = 0.0
    for a in range(3):
        Lap = Lap + K[a][a] * X[a] * lap[a]
        for b in range(a + 1, 3):
            Lap = Lap + K[a][b] * (X[a] * lap[b] + X[b] * lap[a])
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
    Gt = []
    for al, be in pairs:
        s = 0.0
        for x in range(3):
            s = s + K[x][x] * grad[x][al] * grad[x][be]
            for y in range(x + 1, 3):
                s = s + K[x][y] * (grad[x][al] * grad[y][be] + grad[x][be] * grad[y][al])
        Gt.append(s)
    feq, geq, keq = [None] * G.Q, [None] * G.Q, [None] * G.Q
    sf = sg = sk = 0.0
    for i in range(1, G.Q):
        eu = sum(float(G.e[i][a]) * u[a] for a in range(3) if G.e[i][a])
        quad = (eu * eu - cs2 * uu) / (2 * cs2 * cs2)
        tg = sum(G.t[i][c] * Gt[c] for c in range(6) if G.t[i][c] != 0)
        wi = G.w[i]
        feq[i] = wi * (pb / cs2 + rho * eu / cs2 + rho * quad) - wi / cs2 * a2 * Lap + a2 / cs2 * tg
        geq[i] = wi * (gamma[0] * mu_phi / cs2 + phi * eu / cs2 + phi * quad)
        keq[i] = wi * (gamma[1] * mu_psi / cs2 + psi * eu / cs2 + psi * quad)
        sf, sg, sk = sf + feq[i], sg + geq[i], sk + keq[i]
    feq[0], geq[0], keq[0] = rho - sf, phi - sg, psi - sk
    fl = G.fluid_t
    return [[v * fl for v in s] for s in (feq, geq, keq)]


def init_equilibrium(G: Geometry, kappa, h, alpha, gamma, rho, phi, psi):
    """Conventional populations at equilibrium with the fields (u = 0)."""
    fl = G.fluid_t
    X = [rho * fl, phi * fl, psi * fl]
    X = ghosts(G, X, wetting_gradients(kappa, h, alpha))
    zero = torch.zeros(G.N, dtype=_DT)
    return equilibria(G, kappa, alpha, gamma, X, [zero, zero, zero])


def step(G: Geometry, kappa, h, alpha, tau, gamma, pops):
    """One step of conventional populations pops = [f, g, k], each a list of Q [N] tensors."""
    fl = G.fluid_t
    f, g, k = pops
    rho = sum(f) * fl
    phi = sum(g) * fl
    psi = sum(k) * fl
    j = []
    for a in range(3):
        s = torch.zeros(G.N, dtype=_DT)
        for i in range(G.Q):
            if G.e[i][a]:
                s = s + float(G.e[i][a]) * f[i]
        j.append(s * fl)
    X = ghosts(G, [rho, phi, psi], wetting_gradients(kappa, h, alpha))
    eq = equilibria(G, kappa, alpha, gamma, X, j)
    out = []
    for s_, (x, xe) in enumerate(zip(pops, eq)):
        post = [(x[i] - (x[i] - xe[i]) / tau[s_]) * fl for i in range(G.Q)]
        streamed = []
        for i in range(G.Q):
            pulled = post[i][G.src[i]]
            bb = post[G.opp[i]]
            v = torch.where(torch.as_tensor(G.bounce[i]), bb, pulled)
            streamed.append(v * fl)
        out.append(streamed)
    return out


def c3_misfit(G: Geometry, kappa, h, alpha, tau, gamma, rho0, phi0, psi0, target, nsteps):
    """Loss sum_fluid (C_3(T) - target)^2 after nsteps from the initial fields."""
    pops = init_equilibrium(G, kappa, h, alpha, gamma, rho0, phi0, psi0)
    for _ in range(nsteps):
        pops = step(G, kappa, h, alpha, tau, gamma, pops)
    psi = sum(pops[2])
    d = (psi - target) * G.fluid_t
    return (d * d).sum(), pops


def gradients(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, h, rho0, phi0, psi0, target, nsteps,
              solid=None, gamma=(1.0, 1.0)):
    """(loss, dL/dkappa[3], dL/dh[3], dL/drho0, dL/dphi0, dL/dpsi0) by autograd, FP64."""
    G = Geometry(Q, nx, ny, nz, solid)
    kap = torch.tensor(kappa, dtype=_DT, requires_grad=True)
    hh = torch.tensor(h, dtype=_DT, requires_grad=True)
    fields = [torch.tensor(np.asarray(a, dtype=np.float64).reshape(-1), requires_grad=True)
              for a in (rho0, phi0, psi0)]
    tau = (tau_f, 0.5 + M_phi / gamma[0], 0.5 + M_psi / gamma[1])
    tgt = torch.tensor(np.asarray(target, dtype=np.float64).reshape(-1))
    loss, _ = c3_misfit(G, [kap[0], kap[1], kap[2]], [hh[0], hh[1], hh[2]], alpha, tau, gamma,
                        *fields, tgt, nsteps)
    loss.backward()
    def grad_of(t):  # a leaf the loss does not depend on (h without walls) has no gradient: 0
        return t.grad.numpy().copy() if t.grad is not None else np.zeros(tuple(t.shape))

    return (float(loss.detach()), grad_of(kap), grad_of(hh), *[grad_of(f) for f in fields])


def forward_pops(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, h, rho0, phi0, psi0, nsteps,
                 solid=None, gamma=(1.0, 1.0)):
    """Conventional populations ([3][Q][N] numpy) after nsteps, no gradient."""
    G = Geometry(Q, nx, ny, nz, solid)
    tau = (tau_f, 0.5 + M_phi / gamma[0], 0.5 + M_psi / gamma[1])
    with torch.no_grad():
        f = [torch.tensor(np.asarray(a, dtype=np.float64).reshape(-1)) for a in (rho0, phi0, psi0)]
        pops = init_equilibrium(G, list(kappa), list(h), alpha, gamma, *f)
        for _ in range(nsteps):
            pops = step(G, list(kappa), list(h), alpha, tau, gamma, pops)
    return np.stack([np.stack([v.numpy() for v in s]) for s in pops])
