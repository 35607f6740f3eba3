"""Pins of the oracle's stencils, wetting ghosts, streaming, collision and conservation.

- Stencils: on a field that varies along one lattice axis, the isotropic
  gradient and Laplacian have the textbook symbols sin(k) cos(kx) and
  2 (cos k - 1) sin(kx); on a linear ramp the gradient is exact.
- Ghosts: the wall-normal difference between a fluid node and its solid
  neighbour equals the gradient the wetting condition prescribes
  (Sec. Auxiliary variables, conditions on rho, phi, psi).
- Streaming: Eq. latboltPropagation moves a population one link along e_i;
  at a wall, halfway bounce-back returns it reversed to the same node.
- Collision: Eq. latboltCollision relaxes the non-equilibrium part by 1 - 1/tau.
- Conservation: the mass constraints that close the LBM section make every
  step conserve sum rho, sum phi, sum psi; on a periodic lattice total momentum
  is conserved too, since the thermodynamic force enters as a pressure tensor.
"""
import numpy as np
import pytest

import oracle
from paper_1511_02155_gb300 import workloads as W


def test_gradient_and_laplacian_symbols():
    for Q, shape in ((9, (1, 8, 32)), (19, (4, 6, 32))):
        nz, ny, nx = shape
        p = oracle.make_params(Q, nx, ny, nz)
        x = np.arange(nx, dtype=float)
        for kk in (1, 3, 5):
            k = 2 * np.pi * kk / nx
            X = np.broadcast_to(np.sin(k * x), shape).reshape(-1).copy()
            grad, lap = oracle.derivatives(p, X)
            want_g = np.broadcast_to(np.sin(k) * np.cos(k * x), shape).reshape(-1)
            want_l = np.broadcast_to(2 * (np.cos(k) - 1) * np.sin(k * x), shape).reshape(-1)
            assert np.allclose(grad[0], want_g, atol=1e-14, rtol=0)
            assert np.allclose(grad[1:], 0.0, atol=1e-14)
            assert np.allclose(lap, want_l, atol=1e-14, rtol=0)
        # the same field along y and z gives the same symbols on those axes
        for ax in range(1, 3 if Q == 19 else 2):
            n = shape[2 - ax]
            c = np.arange(n, dtype=float)
            k = 2 * np.pi / n
            prof = np.sin(k * c)
            sh = [1, 1, 1]
            sh[2 - ax] = n
            X = np.broadcast_to(prof.reshape(sh), shape).reshape(-1).copy()
            grad, lap = oracle.derivatives(p, X)
            want_g = np.broadcast_to((np.sin(k) * np.cos(k * c)).reshape(sh), shape).reshape(-1)
            want_l = np.broadcast_to((2 * (np.cos(k) - 1) * prof).reshape(sh), shape).reshape(-1)
            assert np.allclose(grad[ax], want_g, atol=1e-14, rtol=0)
            assert np.allclose(lap, want_l, atol=1e-14, rtol=0)


def test_gradient_exact_on_linear_ramp_and_diagonal_isotropy():
    nx = ny = 16
    p = oracle.make_params(9, nx, ny, 1)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    X = (0.3 * x - 0.2 * y).reshape(-1)
    grad, lap = oracle.derivatives(p, X)
    inner = ((x > 0) & (x < nx - 1) & (y > 0) & (y < ny - 1)).reshape(-1)
    assert np.allclose(grad[0][inner], 0.3, atol=1e-14)
    assert np.allclose(grad[1][inner], -0.2, atol=1e-14)
    assert np.allclose(lap[inner], 0.0, atol=1e-14)
    # quadratic: the Laplacian of x^2 + 2 y^2 is 6 exactly in the interior
    X = (x ** 2 + 2 * y ** 2).reshape(-1)
    _, lap = oracle.derivatives(p, X)
    assert np.allclose(lap[inner], 6.0, atol=1e-12)


def test_ghost_rule_on_flat_wall_and_corner():
    nx, ny = 8, 8
    kappa = (0.01, 0.02, 0.03)
    h = (0.0012, -0.0008, 0.0005)
    p = oracle.make_params(9, nx, ny, 1, kappa, 1.3, h=h)
    G = oracle.wetting_gradients(p)
    a2 = 1.3 ** 2
    # the wetting conditions on rho, phi, psi
    assert np.isclose(G[0], -(h[0] / (a2 * kappa[0]) + h[1] / (a2 * kappa[1]) + h[2] / (a2 * kappa[2])))
    assert np.isclose(G[1], -h[0] / (a2 * kappa[0]) + h[1] / (a2 * kappa[1]))
    assert np.isclose(G[2], -h[2] / (a2 * kappa[2]))
    rng = np.random.default_rng(1)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1                 # flat walls at the bottom and top rows
    solid[ny - 1, :] = 1
    solid[4:, 4:] = 1               # a solid block in the upper-right quadrant
    fields = [rng.uniform(0.5, 1.0, (ny, nx)) for _ in range(3)]
    for f in fields:
        f[solid != 0] = 0.0
    F = [f.reshape(-1).copy() for f in fields]
    oracle.ghosts(p, F[0], F[1], F[2], solid)
    F = [f.reshape(ny, nx) for f in F]
    # wall node (x=1, y=0): its only fluid axis neighbour is (1,1) above
    for c in range(3):
        assert np.isclose(F[c][1, 1] - F[c][0, 1], G[c], atol=1e-15)
    # block corner node (5,5) inside the block has no fluid neighbour -> 0
    for c in range(3):
        assert F[c][6, 6] == 0.0
    # convex corner of the block at (x=4, y=4): fluid at (3,4) [axis -x] and (4,3)
    # [axis -y] -> mean of two axis neighbours
    for c in range(3):
        want = ((fields[c][4, 3] - G[c]) + (fields[c][3, 4] - G[c])) / 2
        assert np.isclose(F[c][4, 4], want, atol=1e-15)


def test_ghost_diagonal_only_neighbour():
    nx = ny = 6
    p = oracle.make_params(9, nx, ny, 1, (0.01, 0.02, 0.03), 1.0, h=(0.001, 0.0, -0.0004))
    G = oracle.wetting_gradients(p)
    solid = np.ones((ny, nx), np.uint8)
    solid[2, 2] = 0  # single fluid node; (3,3) touches it only diagonally
    F = [np.zeros(nx * ny) for _ in range(3)]
    for c in range(3):
        F[c][2 * nx + 2] = 0.7 + 0.1 * c
    oracle.ghosts(p, *F, solid)
    for c in range(3):
        assert np.isclose(F[c][3 * nx + 3], 0.7 + 0.1 * c - np.sqrt(2) * G[c], atol=1e-15)
        assert np.isclose(F[c][2 * nx + 3], 0.7 + 0.1 * c - G[c], atol=1e-15)


def test_streaming_moves_along_links_and_bounces_back():
    for Q, shape in ((9, (1, 6, 7)), (19, (5, 6, 7))):
        nz, ny, nx = shape
        N = nx * ny * nz
        p = oracle.make_params(Q, nx, ny, nz)
        e, _, _, opp = oracle.lattice(Q)
        r0 = (2, 3, 3)  # (z, y, x) or y, x for 2-D
        if Q == 9:
            r0 = (0, 3, 3)
        idx = lambda z, y, x: (x % nx) + nx * ((y % ny) + ny * (z % nz))
        xs = np.zeros((Q, N))
        for i in range(Q):
            xs[i, idx(*r0)] = 1.0 + i
        x = oracle.stream(p, xs)
        for i in range(Q):
            z, y, xx = r0
            dst = idx(z + e[i][2], y + e[i][1], xx + e[i][0])
            assert x[i, dst] == 1.0 + i
            assert np.count_nonzero(x[i]) == 1
        # a wall one link in +x of r0: the +x population comes back as -x at r0
        solid = np.zeros(N, np.uint8)
        z, y, xx = r0
        solid[idx(z, y, xx + 1)] = 1
        xs2 = xs.copy()
        xs2[:, idx(z, y, xx + 1)] = 0.0
        x = oracle.stream(p, xs2, solid)
        for i in range(Q):
            if e[i][0] == 1 and e[i][1] == 0 and e[i][2] == 0:
                assert x[opp[i], idx(*r0)] == 1.0 + i
        assert np.all(x[:, idx(z, y, xx + 1)] == 0.0)
        assert np.isclose(x.sum(), xs2.sum())


@pytest.mark.parametrize("Q", [9, 19])
def test_bgk_relaxes_nonequilibrium_part(Q):
    """Uniform state f = f_eq + d with d carrying no mass or momentum: one step
    (streaming a uniform state is the identity) gives f_eq + (1 - 1/tau) d."""
    nz = 1 if Q == 9 else 3
    p = oracle.make_params(Q, 4, 3, nz, (0.01, 0.02, 0.03), 1.0, tau_f=0.8, M_phi=0.3, M_psi=0.05)
    e, w, _, _ = oracle.lattice(Q)
    N = 4 * 3 * nz
    X = np.array([1.02, 0.3, 0.2])
    u = np.array([0.02, -0.01, 0.015 if Q == 19 else 0.0])
    feq, geq, keq = oracle.equilibrium_node(p, X, X[0] * u, np.zeros((3, 3)), np.zeros(3))
    rng = np.random.default_rng(2)
    E = np.vstack([np.ones(Q), e.T.astype(float)])
    d = rng.uniform(-1e-3, 1e-3, (3, Q))
    for s in range(3):  # project out mass and momentum
        d[s] -= E.T @ np.linalg.lstsq(E.T, d[s], rcond=None)[0]
    f = np.repeat((feq + d[0])[:, None], N, axis=1)
    g = np.repeat((geq + d[1])[:, None], N, axis=1)
    k = np.repeat((keq + d[2])[:, None], N, axis=1)
    oracle.step(p, f, g, k, 1)
    taus = p.tau
    for arr, eq, dd, t in ((f, feq, d[0], taus[0]), (g, geq, d[1], taus[1]), (k, keq, d[2], taus[2])):
        assert np.allclose(arr, (eq + (1 - 1 / t) * dd)[:, None], atol=1e-15, rtol=0)


def _run(Q, nx, ny, nz, C, steps, solid=None, **kw):
    p = oracle.make_params(Q, nx, ny, nz, **kw)
    rho, phi, psi = W.to_aux(*C)
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    return p, f, g, k


def test_mass_and_momentum_conservation_periodic():
    C = W.lens(48, 40, 9.0, 1.0, 10.0, 30.0, (24.0, 30.0))
    p, f, g, k = _run(9, 48, 40, 1, C, 0, kappa=(0.01, 0.02, 0.03), M_phi=0.2, M_psi=0.1)
    m0 = oracle.mass(p, f, g, k)
    oracle.step(p, f, g, k, 400)
    m1 = oracle.mass(p, f, g, k)
    N = 48 * 40
    assert np.all(np.abs(m1 - m0) <= 1e-12 * N)
    _, j, _, _ = oracle.moments(p, f, g, k)
    assert np.all(np.abs(j.sum(axis=1)) < 1e-12 * N)
    # 3-D spinodal mixture
    C = W.spinodal((6, 7, 8), seed=9)
    p, f, g, k = _run(19, 8, 7, 6, C, 0, kappa=(0.01, 0.01, 0.01), tau_f=0.8)
    m0 = oracle.mass(p, f, g, k)
    oracle.step(p, f, g, k, 60)
    m1 = oracle.mass(p, f, g, k)
    assert np.all(np.abs(m1 - m0) <= 1e-12 * 336)
    _, j, _, _ = oracle.moments(p, f, g, k)
    assert np.all(np.abs(j.sum(axis=1)) < 1e-12 * 336)


def test_mass_conservation_with_walls_and_wetting():
    C, solid = W.sessile_drop(40, 30, 8.0, m=2, n=0, alpha=1.0)
    h = (0.0005, -0.0008, 0.001)
    p = oracle.make_params(9, 40, 30, 1, (0.01, 0.02, 0.03), 1.0, h=h)
    rho, phi, psi = W.to_aux(*C)
    rho[solid != 0] = 0
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    m0 = oracle.mass(p, f, g, k, solid)
    oracle.step(p, f, g, k, 300, solid)
    m1 = oracle.mass(p, f, g, k, solid)
    assert np.all(np.abs(m1 - m0) <= 1e-12 * 1200)
    assert np.all(f[:, solid.reshape(-1) != 0] == 0)


@pytest.mark.parametrize("Q", [9, 19])
def test_uniform_state_is_steady(Q):
    nz = 1 if Q == 9 else 4
    C = [np.full((nz, 5, 6) if Q == 19 else (5, 6), v) for v in (0.2, 0.5, 0.3)]
    p = oracle.make_params(Q, 6, 5, nz, (0.01, 0.02, 0.03), 1.0)
    rho, phi, psi = W.to_aux(*C)
    u = [np.full(rho.shape, 0.01), np.full(rho.shape, -0.02), np.full(rho.shape, 0.005 if Q == 19 else 0.0)]
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, u=u)
    f0, g0, k0 = f.copy(), g.copy(), k.copy()
    oracle.step(p, f, g, k, 5)
    assert np.allclose(f, f0, atol=1e-15) and np.allclose(g, g0, atol=1e-15) and np.allclose(k, k0, atol=1e-15)
