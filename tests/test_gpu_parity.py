"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle.

Tolerances
- FP64 storage: every field (C_1, C_2, C_3, rho) and every population set within
  a relative 1e-12 of the oracle after the stated number of steps, relative to
  max(largest magnitude of the field, 1) -- concentrations and densities are
  O(1) by construction, and a field that is identically zero (a fluid absent
  from the geometry) is compared on that O(1) scale, not on its rounding
  noise; velocities within 1e-14 absolute.
- FP32 storage: max |dC_m| <= 1e-4 against the FP64 oracle.
- Full-size lattices: the GPU state after T steps is read back in patches;
  the oracle advances each patch one step (periodic wrap inside the patch,
  so only nodes at least three links from the patch edge are compared) and the
  GPU's own next step must match it within 2e-6 absolute per population
  (FP32 rounding of one step).
"""
import numpy as np
import pytest

import oracle
import paper_1511_02155_gb300 as tl
from paper_1511_02155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _setup(Q, shape, C, precision, kernel="auto", solid=None, kappa=(0.01, 0.02, 0.03), alpha=1.0,
           tau_f=1.0, M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), u=None):
    nx, ny, nz = shape
    eng = tl.TernaryLB(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, h, solid, precision)
    if kernel != "auto":
        eng.set_kernel(kernel)
    p = oracle.make_params(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, h)
    rho, phi, psi = W.to_aux(*C)
    if solid is not None:
        for a in (rho, phi, psi):
            a[np.asarray(solid) != 0] = 0.0
    eng.init_fields(rho, phi, psi, u)
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, u=u, solid=solid)
    return eng, p, (f, g, k)


def _rel(a, b):
    scale = max(np.abs(b).max(), 1.0)
    return np.abs(a - b).max() / scale


def _compare_fp64(eng, p, pops, solid=None, tol=1e-12):
    f, g, k = pops
    C1, C2, C3, rho, u = oracle.fields(p, f, g, k, solid)
    got = eng.fields()
    for name, want in (("C1", C1), ("C2", C2), ("C3", C3), ("rho", rho)):
        assert _rel(got[name], want) <= tol, (name, _rel(got[name], want))
    assert np.abs(got["u"] - u).max() <= 1e-14
    P = eng.get_populations()
    for s, want in enumerate((f, g, k)):
        assert _rel(P[s], want) <= tol, ("set", s, _rel(P[s], want))


# --------------------------------------------------------------- FP64 parity

@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_lens_64x64_fp64_2000_steps(kernel):
    """Plain-FP64 D2Q9 lens, 64x64 periodic, 2000 steps, against the oracle."""
    cfg = W.lens_64_fp64()
    shape = (cfg["nx"], cfg["ny"], 1)
    eng, p, pops = _setup(9, shape, cfg["C"], "fp64", kernel, kappa=cfg["kappa"], M_phi=cfg["M_phi"],
                          M_psi=cfg["M_psi"], tau_f=cfg["tau_f"])
    m0 = eng.mass()
    eng.step(2000)
    oracle.step(p, *pops, 2000)
    _compare_fp64(eng, p, pops)
    m1 = eng.mass()
    assert np.all(np.abs(m1 - m0) <= 1e-12 * 4096)
    assert np.allclose(m1, oracle.mass(p, *pops), rtol=0, atol=1e-10)


SMALL = [
    (9, (37, 29, 1)),    # ragged against every tile
    (9, (5, 3, 1)),      # smaller than a tile
    (9, (16, 1, 1)),     # one row: the y neighbours are the node itself
    (9, (130, 7, 1)),    # one tile plus a 2-node tail
    (19, (19, 13, 11)),
    (19, (3, 2, 2)),
    (19, (33, 9, 1)),    # a single plane
]


@pytest.mark.parametrize("kernel", ["fused", "split"])
@pytest.mark.parametrize("Q,shape", SMALL)
def test_fp64_parity_periodic(Q, shape, kernel):
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    C = W.spinodal(sh, seed=11, amp=0.2)
    rng = np.random.default_rng(3)
    u = [rng.uniform(-0.02, 0.02, sh) for _ in range(3)]
    if Q == 9:
        u[2][:] = 0.0
    eng, p, pops = _setup(Q, shape, C, "fp64", kernel, kappa=(0.012, 0.02, 0.031), tau_f=0.8,
                          M_phi=0.15, M_psi=0.1, u=u)
    _compare_fp64(eng, p, pops, tol=1e-13)       # equilibrium initialisation
    eng.step(60)
    oracle.step(p, *pops, 60)
    _compare_fp64(eng, p, pops)


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp64_parity_walls_and_wetting_d2q9(kernel):
    C, solid = W.sessile_drop(40, 30, 8.0, m=2, n=0)
    h = (0.0005, -0.0008, 0.001)
    eng, p, pops = _setup(9, (40, 30, 1), C, "fp64", kernel, solid=solid, h=h)
    assert eng.kernel == kernel
    _compare_fp64(eng, p, pops, solid=solid, tol=1e-13)
    eng.step(150)
    oracle.step(p, *pops, 150, solid)
    _compare_fp64(eng, p, pops, solid=solid)


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp64_parity_square_well_with_corners(kernel):
    C, solid = W.square_well(48, 40, width=14, depth=10, floor=6)
    h = (-0.0006, 0.0009, 0.0004)
    eng, p, pops = _setup(9, (48, 40, 1), C, "fp64", kernel, solid=solid, h=h, kappa=(0.01, 0.012, 0.015))
    eng.step(120)
    oracle.step(p, *pops, 120, solid)
    _compare_fp64(eng, p, pops, solid=solid)


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp64_parity_walls_d3q19(kernel):
    nx, ny, nz = 12, 10, 9
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    solid[3:6, 1:3, 4:7] = 1  # a block on the bottom wall (edges and corners)
    C = W.spinodal((nz, ny, nx), seed=5, amp=0.2)
    h = (0.0004, -0.0006, 0.0002)
    eng, p, pops = _setup(19, (nx, ny, nz), C, "fp64", kernel, solid=solid, h=h)
    eng.step(40)
    oracle.step(p, *pops, 40, solid.reshape(-1))
    _compare_fp64(eng, p, pops, solid=solid.reshape(-1))


# --------------------------------------------------------------- FP32 parity

@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp32_lens_against_fp64_oracle(kernel):
    C = W.lens(96, 80, 14.0, 1.0, 20.0, 60.0, (48.0, 60.0))
    eng, p, pops = _setup(9, (96, 80, 1), C, "fp32", kernel, kappa=(0.01, 0.02, 0.03))
    eng.step(1000)
    oracle.step(p, *pops, 1000)
    C1, C2, C3, _, _ = oracle.fields(p, *pops)
    got = eng.fields()
    for name, want in (("C1", C1), ("C2", C2), ("C3", C3)):
        assert np.abs(got[name] - want).max() <= 1e-4, name


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp32_spinodal_3d_against_fp64_oracle(kernel):
    n = 20
    C = W.spinodal((n, n, n), seed=3)
    eng, p, pops = _setup(19, (n, n, n), C, "fp32", kernel, kappa=(0.01, 0.01, 0.01), tau_f=0.8)
    eng.step(200)
    oracle.step(p, *pops, 200)
    C1, C2, C3, _, _ = oracle.fields(p, *pops)
    got = eng.fields()
    for name, want in (("C1", C1), ("C2", C2), ("C3", C3)):
        assert np.abs(got[name] - want).max() <= 1e-4, name


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_fp32_walls_against_fp64_oracle(kernel):
    C, solid = W.sessile_drop(64, 40, 12.0, m=2, n=0)
    h = (0.0004, -0.0006, 0.0008)
    eng, p, pops = _setup(9, (64, 40, 1), C, "fp32", kernel, solid=solid, h=h)
    eng.step(500)
    oracle.step(p, *pops, 500, solid)
    C1, C2, C3, _, _ = oracle.fields(p, *pops, solid)
    got = eng.fields()
    for name, want in (("C1", C1), ("C2", C2), ("C3", C3)):
        assert np.abs(got[name] - want).max() <= 1e-4, name


# ------------------------------------------------ full sizes, sampled patches

def _patch_step_check(eng, p_full, solid_full, centres, B, tol):
    """Oracle one step on patches of the GPU state vs the GPU's next step."""
    nx, ny, nz = eng.shape
    Q = eng.Q
    before = []
    for c in centres:
        x0, y0 = c[0] - B // 2, c[1] - B // 2
        z0 = c[2] - B // 2 if Q == 19 else 0
        bz = B if Q == 19 else 1
        before.append((x0, y0, z0, bz, eng.get_populations_box(x0, y0, z0, B, B, bz)))
    eng.step(1)
    worst = 0.0
    for x0, y0, z0, bz, pops in before:
        after = eng.get_populations_box(x0, y0, z0, B, B, bz)
        p = oracle.make_params(Q, B, B, bz, tuple(p_full.kappa), p_full.alpha, p_full.tau[0],
                               p_full.tau[1] - 0.5, p_full.tau[2] - 0.5, tuple(p_full.h))
        sol = None
        if solid_full is not None:
            sf = solid_full.reshape(nz, ny, nx)
            zi = (np.arange(bz) + z0) % nz
            yi = (np.arange(B) + y0) % ny
            xi = (np.arange(B) + x0) % nx
            sol = np.ascontiguousarray(sf[np.ix_(zi, yi, xi)]).reshape(-1)
        f, g, k = (np.ascontiguousarray(pops[s].reshape(Q, -1)) for s in range(3))
        oracle.step(p, f, g, k, 1, sol)
        m = 3
        sl = (slice(None), slice(m, bz - m) if Q == 19 else slice(None), slice(m, B - m), slice(m, B - m))
        for s, want in enumerate((f, g, k)):
            w = want.reshape(Q, bz, B, B)[sl]
            gpu = after[s][sl]
            worst = max(worst, float(np.abs(gpu - w).max()))
    assert worst <= tol, worst


def test_full_size_lens_512x256_fp32_sampled_step():
    cfg = W.lens_512x256()
    nx, ny = cfg["nx"], cfg["ny"]
    eng = tl.TernaryLB(9, nx, ny, 1, cfg["kappa"], 1.0, cfg["tau_f"], cfg["M_phi"], cfg["M_psi"],
                       precision="fp32")
    eng.init_fields(*W.to_aux(*cfg["C"]))
    eng.step(300)
    p = oracle.make_params(9, nx, ny, 1, cfg["kappa"], 1.0, cfg["tau_f"], cfg["M_phi"], cfg["M_psi"])
    rng = np.random.default_rng(0)
    centres = [(int(rng.integers(nx)), int(rng.integers(ny)), 0) for _ in range(6)]
    centres += [(256, 128, 0), (316, 128, 0), (0, 0, 0), (nx - 1, ny - 1, 0)]  # triple line, wrap
    _patch_step_check(eng, p, None, centres, 16, 2e-6)


def test_full_size_spinodal_256_cubed_fp32_sampled_step():
    """The benchmark's D3Q19 256^3 workload, in the benchmark's launch configuration."""
    n = 256
    C = W.spinodal((n, n, n), seed=3)
    eng = tl.TernaryLB(19, n, n, n, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1, precision="fp32")
    assert eng.kernel == "fused"
    eng.init_fields(*W.to_aux(*C))
    del C
    m0 = eng.mass()
    eng.step(20)
    p = oracle.make_params(19, n, n, n, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1)
    rng = np.random.default_rng(1)
    centres = [tuple(int(v) for v in rng.integers(n, size=3)) for _ in range(4)]
    centres += [(0, 0, 0), (255, 128, 255)]
    _patch_step_check(eng, p, None, centres, 12, 2e-6)
    m1 = eng.mass()
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0).max())


def test_full_size_wells_4096_fp32_sampled_step():
    """The benchmark's walls-and-wetting workload (D2Q9 4096x2048, 32 wells), in
    the benchmark's launch configuration (solid-aware fused kernel): patches
    over wells, walls, the lid and the 1/2 interface."""
    cfg = W.wells_2d()
    nx, ny = cfg["nx"], cfg["ny"]
    solid = cfg["solid"]
    rho, phi, psi = W.to_aux(*cfg["C"])
    for a in (rho, phi, psi):
        a[solid != 0] = 0.0
    eng = tl.TernaryLB(9, nx, ny, 1, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"], cfg["M_psi"],
                       cfg["h"], solid.reshape(-1), "fp32")
    assert eng.kernel == "fused"
    eng.init_fields(rho, phi, psi)
    eng.step(200)
    p = oracle.make_params(9, nx, ny, 1, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"], cfg["M_psi"],
                           cfg["h"])
    pitch = nx // 32
    centres = [(k * pitch + pitch // 2, 40, 0) for k in (0, 7, 19, 31)]      # inside / at the rim of wells
    centres += [(k * pitch + 5, 30, 0) for k in (3, 12)]                      # well side walls and corners
    centres += [(1000, ny - 6, 0), (2500, 48 + (ny - 49) // 2, 0), (nx - 2, 50, 0)]  # lid, interface, wrap
    _patch_step_check(eng, p, solid.reshape(-1), centres, 24, 2e-6)


def test_full_size_2d_probe_8192_fp32_sampled_step():
    n = 8192
    C = W.spinodal((n, n), seed=5)
    eng = tl.TernaryLB(9, n, n, 1, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1, precision="fp32")
    eng.init_fields(*W.to_aux(*C))
    del C
    eng.step(10)
    p = oracle.make_params(9, n, n, 1, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1)
    centres = [(0, 0, 0), (4096, 17, 0), (8191, 8191, 0), (1234, 5678, 0)]
    _patch_step_check(eng, p, None, centres, 16, 2e-6)


# --------------------------------------------------- invariants and edge cases

def test_tile_variants_are_bitwise_identical():
    n = 40
    C = W.spinodal((n, n, n), seed=8, amp=0.05)
    ref = None
    for variant, chunk in ((0, 0), (1, 8), (2, 3), (3, 40), (1, 1), (4, 0), (5, 7), (6, 0), (3, 13), (4, 6),
                           (7, 0), (7, 5), (5, 0)):
        eng = tl.TernaryLB(19, n, n, n, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1, precision="fp32")
        eng.set_tile(variant, chunk)
        eng.init_fields(*W.to_aux(*C))
        eng.step(7)
        P = eng.get_populations()
        if ref is None:
            ref = P
        else:
            assert np.array_equal(P, ref), (variant, chunk)
        eng.close()
    # whole and single tiles along a, ragged b and marching extents
    for shape in ((64, 21, 19), (32, 13, 11)):
        nx, ny, nz = shape
        C3 = W.spinodal((nz, ny, nx), seed=9, amp=0.05)
        ref = None
        for variant, chunk in ((0, 0), (5, 0), (6, 5), (3, 1), (4, 0), (7, 3)):
            eng = tl.TernaryLB(19, nx, ny, nz, (0.01, 0.02, 0.015), 1.0, 0.8, 0.1, 0.1, precision="fp32")
            eng.set_tile(variant, chunk)
            eng.init_fields(*W.to_aux(*C3))
            eng.step(6)
            P = eng.get_populations()
            if ref is None:
                ref = P
            else:
                assert np.array_equal(P, ref), (shape, variant, chunk)
            eng.close()
    C2 = W.spinodal((200, 300), seed=8, amp=0.05)
    ref = None
    for variant, chunk in ((0, 0), (1, 5), (2, 64), (3, 1), (4, 0), (5, 3), (1, 0)):
        eng = tl.TernaryLB(9, 300, 200, 1, (0.01, 0.01, 0.01), 1.0, 0.8, 0.1, 0.1, precision="fp32")
        eng.set_tile(variant, chunk)
        eng.init_fields(*W.to_aux(*C2))
        eng.step(5)
        P = eng.get_populations()
        if ref is None:
            ref = P
        else:
            assert np.array_equal(P, ref), (variant, chunk)
        eng.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_tile_variants_are_bitwise_identical_16bit(precision):
    """The staging orders and tiles of the 16-bit D3Q19 kernels (paired lane
    words) give bitwise the same state on a ragged lattice."""
    nx, ny, nz = 45, 13, 11
    C = W.spinodal((nz, ny, nx), seed=10, amp=0.05)
    ref = None
    for variant, chunk in ((0, 0), (4, 0), (5, 3), (6, 0), (7, 1), (3, 0), (1, 2)):
        eng = tl.TernaryLB(19, nx, ny, nz, (0.01, 0.02, 0.015), 1.0, 0.8, 0.1, 0.1, precision=precision)
        eng.set_tile(variant, chunk)
        eng.init_fields(*W.to_aux(*C))
        eng.step(6)
        P = eng.get_populations()
        if ref is None:
            ref = P
        else:
            assert np.array_equal(P, ref), (variant, chunk)
        eng.close()


@pytest.mark.parametrize("Q,shape", [(9, (150, 37, 1)), (19, (37, 13, 11))])
def test_fused_walls_ragged_fp64(Q, shape):
    """Solid geometry on lattices that are ragged against every tile: walls, a
    block with edges and corners, and wetting on all three fluids."""
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    solid = np.zeros(sh, np.uint8)
    if Q == 9:
        solid[0, :] = 1
        solid[ny - 1, :] = 1
        solid[1:6, 20:31] = 1
    else:
        solid[:, 0, :] = 1
        solid[:, ny - 1, :] = 1
        solid[2:6, 1:4, 10:17] = 1
    C = W.spinodal(sh, seed=12, amp=0.2)
    h = (0.0006, -0.0004, 0.0003)
    eng, p, pops = _setup(Q, shape, C, "fp64", "fused", solid=solid, h=h)
    eng.step(30)
    oracle.step(p, *pops, 30, solid.reshape(-1))
    _compare_fp64(eng, p, pops, solid=solid.reshape(-1))


def test_fused_and_split_agree_fp32():
    C = W.lens(64, 48, 10.0, 1.0, 12.0, 36.0, (32.0, 36.0))
    out = []
    for kind in ("fused", "split"):
        eng, _, _ = _setup(9, (64, 48, 1), C, "fp32", kind)
        eng.step(300)
        out.append(eng.fields())
    for name in ("C1", "C2", "C3", "rho"):
        assert np.abs(out[0][name] - out[1][name]).max() <= 1e-5


def test_checkpoint_resume_is_bitwise_and_runs_repeat():
    C = W.spinodal((24, 28, 20), seed=2, amp=0.05)
    eng, _, _ = _setup(19, (20, 28, 24), C, "fp32")
    eng.step(5)
    state = eng.get_state()
    eng.step(9)
    a = eng.get_populations()
    ma = eng.mass()
    eng.set_state(state)
    eng.step(9)
    b = eng.get_populations()
    assert np.array_equal(a, b)
    assert np.array_equal(ma, eng.mass())  # fixed-order reduction: bitwise repeatable


def test_set_and_get_populations_round_trip():
    C = W.lens(30, 20, 5.0, 1.0, 5.0, 15.0, (15.0, 15.0))
    solid = W.walls_y(30, 20, 1, 1)
    eng, p, pops = _setup(9, (30, 20, 1), C, "fp64", solid=solid, h=(0.0003, 0.0, -0.0002))
    P = np.stack(pops)
    rng = np.random.default_rng(4)
    P = P + rng.uniform(-1e-3, 1e-3, P.shape)
    P[:, :, solid.reshape(-1) != 0] = 0.0
    eng.set_populations(P)
    assert np.array_equal(eng.get_populations(), P)
    eng.step(3)
    f, g, k = (np.ascontiguousarray(P[s]) for s in range(3))
    oracle.step(p, f, g, k, 3, solid)
    _compare_fp64(eng, p, (f, g, k), solid=solid)


def test_zero_steps_and_uniform_state():
    C = [np.full((6, 7), v) for v in (0.2, 0.5, 0.3)]
    u = [np.full((6, 7), 0.01), np.full((6, 7), -0.02), np.zeros((6, 7))]
    eng, p, pops = _setup(9, (7, 6, 1), C, "fp64", u=u)
    P0 = eng.get_populations()
    eng.step(0)
    assert np.array_equal(eng.get_populations(), P0)
    eng.step(10)
    assert np.abs(eng.get_populations() - P0).max() < 1e-14  # steady up to FP64 rounding


def test_nonfinite_is_detected_from_a_host_made_fault():
    """A NaN planted in the populations on the host: the in-step FP64 totals flag it."""
    C = W.lens(32, 24, 5.0, 1.0, 6.0, 18.0, (16.0, 18.0))
    eng, p, pops = _setup(9, (32, 24, 1), C, "fp32")
    P = np.stack(pops)
    P[0, 3, 100] = np.nan
    eng.set_populations(P)
    eng.step(2)
    with pytest.raises(tl.TLBMError) as e:
        eng.step_mass()
    assert e.value.status == 5
    with pytest.raises(tl.TLBMError) as e:
        eng.mass()
    assert e.value.status == 5
    # a fresh initialisation clears the flag
    eng.init_fields(*W.to_aux(*C))
    eng.step(1)
    assert np.all(np.isfinite(eng.step_mass()))


def test_step_mass_matches_mass_of_previous_state():
    C = W.lens(48, 40, 8.0, 1.0, 10.0, 30.0, (24.0, 30.0))
    for kind in ("fused", "split"):
        eng, p, pops = _setup(9, (48, 40, 1), C, "fp64", kind)
        eng.step(4)
        m = eng.mass()
        eng.step(1)
        assert np.allclose(eng.step_mass(), m, rtol=0, atol=1e-11)


def test_launch_counts():
    C = W.lens(32, 24, 5.0, 1.0, 6.0, 18.0, (16.0, 18.0))
    eng, _, _ = _setup(9, (32, 24, 1), C, "fp32")
    assert eng.kernel == "fused" and eng.launches_per_step == 2
    eng.set_kernel("split")
    assert eng.launches_per_step == 3
    solid = W.walls_y(32, 24)
    eng2, _, _ = _setup(9, (32, 24, 1), C, "fp32", solid=solid)
    assert eng2.kernel == "fused" and eng2.launches_per_step == 2
    eng2.set_kernel("split")
    assert eng2.launches_per_step == 4


@pytest.mark.parametrize("Q,shape,walls", [(19, (37, 13, 11), False), (19, (37, 13, 11), True),
                                           (9, (150, 37, 1), False), (9, (150, 37, 1), True)])
def test_bounds_checked_step_records_nothing_and_matches(Q, shape, walls):
    """The bounds-checked kernels (every population address against the buffer
    and its chunk layout, every moment-ring and mask index against its extent)
    record no violation on lattices ragged against the tiles, with and without
    walls, and give bitwise the results of the unchecked kernels."""
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    C = W.spinodal(sh, seed=12, amp=0.05)
    solid = None
    if walls:
        solid = np.zeros(sh, dtype=np.uint8)
        if Q == 9:
            solid[0, :] = solid[-1, :] = 1
            solid[9:15, 40:70] = 1
        else:
            solid[:, 0, :] = solid[:, -1, :] = 1
            solid[3:7, 4:8, 10:20] = 1
    out = []
    for checked in (False, True):
        eng, _, _ = _setup(Q, shape, C, "fp32", solid=solid, h=(0.0005, -0.0004, 0.0003))
        eng.set_bounds_check(checked)
        eng.step(5)
        assert eng.bounds_check_word() == 0
        out.append(eng.get_state())
        eng.close()
    assert np.array_equal(out[0], out[1])
