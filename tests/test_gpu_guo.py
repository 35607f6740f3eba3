"""GPU parity of the forcing (Guo) coupling against the oracle's orc_step_guo,
for both of its kernels: the marching kernel (one launch per step, the
default) and the split step (three launches).

Tolerances
- FP64 storage: populations and fields within a relative 1e-12 of the oracle
  (same arithmetic, other summation orders; the FP64 units do not contract
  multiply-adds), the fluid velocity (j + F/2)/rho within 1e-14 absolute.
- FP32 storage: max |dC_m| <= 1e-4 against the FP64 oracle (the bound of the
  pressure-tensor coupling's FP32 tests); FP16/BF16 storage within 1e-2 / 5e-2.
- Full size: the 256^3 D3Q19 spinodal state is read back in 16^3 patches, the
  oracle advances each patch one step (periodic wrap inside the patch) and
  nodes four links or more from the patch edge (the step's dependence radius
  is three: pull, Pi at r + e, moments at r + e + e') must match the GPU's
  own next step within 2e-6 per population (FP32 rounding of one step).
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


def _engine(Q, shape, kappa, alpha, tau_f, M_phi, M_psi, precision, C, kernel="auto"):
    nx, ny, nz = shape
    eng = tl.TernaryLB(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi, precision=precision)
    eng.set_coupling("forcing")
    if kernel != "auto":
        eng.set_kernel(kernel)
    assert eng.coupling == "forcing" and eng.kernel == ("fused" if kernel == "auto" else kernel)
    r = W.to_aux(*C)
    eng.init_fields(*r)
    p = oracle.make_params(Q, nx, ny, nz, kappa, alpha, tau_f, M_phi, M_psi)
    f, g, k = oracle.init_equilibrium_guo(p, *r)
    return eng, p, (f, g, k)


def _velocity(p, pops):
    rho, j, phi, psi = oracle.moments(p, *pops)
    F = oracle.force(p, rho, phi, psi)
    return (np.asarray(j) + np.asarray(F) / 2) / rho


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


CASES = [
    (9, (40, 33, 1), (0.05, 0.08, 0.06), 1.0, 0.8, 0.2, 0.3),   # ragged 32-node chunks
    (19, (12, 10, 9), (0.01, 0.02, 0.03), 1.0, 1.0, 0.1, 0.1),
]


@pytest.mark.parametrize("kernel", ["fused", "split"])
@pytest.mark.parametrize("Q,shape,kappa,alpha,tau_f,Mp,Ms", CASES)
def test_guo_fp64_matches_oracle(Q, shape, kappa, alpha, tau_f, Mp, Ms, kernel):
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    C = W.spinodal(sh, seed=17, amp=0.2)
    eng, p, pops = _engine(Q, shape, kappa, alpha, tau_f, Mp, Ms, "fp64", C, kernel)
    P = eng.get_populations()
    for s in range(3):
        assert _rel(np.ravel(P[s]), np.ravel(pops[s])) <= 1e-12, ("init set", s)
    m0 = eng.mass()
    eng.step(60)
    oracle.step_guo(p, *pops, 60)
    P = eng.get_populations()
    for s in range(3):
        assert _rel(np.ravel(P[s]), np.ravel(pops[s])) <= 1e-12, ("set", s)
    got = eng.fields()
    C1, C2, C3, rho, _ = oracle.fields(p, *pops)
    for name, want in (("C1", C1), ("C2", C2), ("C3", C3), ("rho", rho)):
        assert _rel(got[name], want) <= 1e-12, name
    u = _velocity(p, pops)
    assert np.abs(got["u"] - u.reshape(got["u"].shape)).max() <= 1e-14
    assert np.abs(u).max() > 1e-6  # the comparison is not of zeros
    assert np.all(np.abs(eng.mass() - m0) <= 1e-12 * np.prod(shape))


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_guo_total_momentum_is_conserved_fp64(kernel):
    """sum_r F = 0 on a periodic lattice: the total momentum j stays at its
    initial zero through many steps of a coarsening spinodal mixture."""
    C = W.spinodal((64, 64), seed=5, amp=0.3)
    eng, p, pops = _engine(9, (64, 64, 1), (0.01, 0.02, 0.03), 1.0, 1.0, 0.1, 0.1, "fp64", C, kernel)
    eng.step(500)
    P = eng.get_populations()
    f, g, k = (np.ascontiguousarray(P[s].reshape(9, -1)) for s in range(3))
    _, j, _, _ = oracle.moments(p, f, g, k)  # the oracle's lattice, same population order
    jx, jy = float(np.sum(j[0])), float(np.sum(j[1]))
    assert np.abs(j).max() > 1e-8  # there is flow to sum
    assert abs(jx) <= 1e-11 and abs(jy) <= 1e-11, (jx, jy)


@pytest.mark.parametrize("kernel", ["fused", "split"])
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp16", 1e-2), ("bf16", 5e-2)])
def test_guo_lens_reduced_precision_against_fp64_oracle(precision, tol, kernel):
    kappa = (0.01, 0.02, 0.03)
    C = W.lens(48, 40, 8.0, 1.0, 10.0, 30.0, (24.0, 30.0))
    eng, p, pops = _engine(9, (48, 40, 1), kappa, 1.0, 1.0, 0.1, 0.1, precision, C, kernel)
    m0 = eng.mass()
    eng.step(1000)
    oracle.step_guo(p, *pops, 1000)
    got = eng.fields()
    want = oracle.fields(p, *pops)
    d = max(float(np.abs(got[n] - want[i]).max()) for i, n in enumerate(("C1", "C2", "C3")))
    print(kernel, precision, "max |dC| =", d)
    assert d <= tol
    if precision == "fp32":
        # per-node exact rest update: totals stay within FP32 rounding of the sums
        assert np.all(np.abs(eng.mass() - m0) <= 1e-6 * np.abs(m0).max())


@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_guo_full_size_spinodal_256_cubed_fp32_sampled_step(kernel):
    """The forcing coupling on the benchmark's D3Q19 256^3 workload, in the
    launch configuration of bench.py --coupling forcing (fused) and split."""
    n = 256
    kappa = (0.01, 0.01, 0.01)
    C = W.spinodal((n, n, n), seed=3)
    eng = tl.TernaryLB(19, n, n, n, kappa, 1.0, 0.8, 0.1, 0.1, precision="fp32")
    eng.set_coupling("forcing")
    eng.set_kernel(kernel)
    eng.init_fields(*W.to_aux(*C))
    del C
    eng.step(20)
    B, m = 16, 4
    rng = np.random.default_rng(2)
    centres = [tuple(int(v) for v in rng.integers(n, size=3)) for _ in range(3)] + [(0, 0, 0)]
    before = [(c, eng.get_populations_box(c[0] - B // 2, c[1] - B // 2, c[2] - B // 2, B, B, B))
              for c in centres]
    eng.step(1)
    p = oracle.make_params(19, B, B, B, kappa, 1.0, 0.8, 0.1, 0.1)
    worst = 0.0
    for c, pops in before:
        after = eng.get_populations_box(c[0] - B // 2, c[1] - B // 2, c[2] - B // 2, B, B, B)
        f, g, k = (np.ascontiguousarray(pops[s].reshape(19, -1)) for s in range(3))
        oracle.step_guo(p, f, g, k, 1)
        sl = (slice(None), slice(m, B - m), slice(m, B - m), slice(m, B - m))
        for s, want in enumerate((f, g, k)):
            worst = max(worst, float(np.abs(after[s][sl] - want.reshape(19, B, B, B)[sl]).max()))
    assert worst <= 2e-6, worst


def test_guo_refusals_and_launch_count():
    kappa = (0.01, 0.02, 0.03)
    solid = np.zeros((8, 16), np.uint8)
    solid[0] = 1
    walls = tl.TernaryLB(9, 16, 8, 1, kappa, 1.0, 1.0, 0.1, 0.1, solid=solid.reshape(-1), precision="fp32")
    with pytest.raises(tl.TLBMError, match="UNSUPPORTED"):
        walls.set_coupling("forcing")
    assert walls.coupling == "pressure_tensor"
    eng = tl.TernaryLB(9, 16, 8, 1, kappa, 1.0, 1.0, 0.1, 0.1, precision="fp32")
    eng.set_coupling("forcing")
    assert eng.kernel == "fused" and eng.launches_per_step == 2
    eng.set_kernel("split")
    assert eng.kernel == "split" and eng.launches_per_step == 4
    eng.set_kernel("auto")
    with pytest.raises(tl.TLBMError, match="UNSUPPORTED"):
        tl.TernaryBatch([eng])
    eng.init_fields(*W.to_aux(*W.spinodal((8, 16), seed=1)))
    with pytest.raises(tl.TLBMError, match="UNSUPPORTED"):
        eng.adjoint_c3_misfit(3, 1, np.zeros(128))
    # back to the pressure tensor
    eng.set_coupling("pressure_tensor")
    assert eng.kernel == "fused" and eng.coupling == "pressure_tensor"


@pytest.mark.parametrize("Q,shape", [(9, (37, 29, 1)), (19, (21, 13, 11))])
def test_guo_fused_and_split_agree_fp32(Q, shape):
    """Both kernels of the forcing coupling on ragged lattices and chunkings,
    FP32: the same arithmetic in other summation orders (derivatives from the
    shared-memory ring against the node arrays), within FP32 rounding."""
    nx, ny, nz = shape
    sh = (ny, nx) if Q == 9 else (nz, ny, nx)
    C = W.spinodal(sh, seed=23, amp=0.2)
    out = []
    for kernel, chunk in (("split", 0), ("fused", 0), ("fused", 1), ("fused", 5)):
        eng = tl.TernaryLB(Q, nx, ny, nz, (0.01, 0.02, 0.015), 1.0, 0.8, 0.1, 0.1, precision="fp32")
        eng.set_coupling("forcing")
        eng.set_kernel(kernel)
        eng.set_tile(0, chunk)
        eng.init_fields(*W.to_aux(*C))
        eng.step(40)
        out.append(eng.get_populations())
        eng.close()
    for P in out[1:]:
        assert np.abs(P - out[0]).max() <= 2e-6
    for P in out[2:]:  # chunkings of the fused kernel: the same per-node arithmetic
        assert np.array_equal(P, out[1])
