"""16-bit population storage (FP16 / BF16, computed in FP32) against the FP64 oracle.

Format: f kept as its deviation f_i - w_i from the rest state, g and k as they
are; the moving populations i >= 1 in 16 bits, the rest populations in FP32.
- Round trip: populations written through tlbm_set_populations read back
  exactly as a numpy replica of that encoding predicts.
- One step: from the same (decoded) state, the GPU's next state agrees with the
  oracle's within the rounding of the 16-bit outputs: 2^-p |x - bias| plus 5e-7
  (p = 11 for FP16, 8 for BF16) for a moving population; the rest population
  (FP32) absorbs the rounding of the node's moving ones (it is the moment minus
  the stored moving populations), so its bound is their sum.
- Conservation: with that rest population, 16-bit rounding never changes a
  node's rho, phi or psi; the FP64 totals drift only by FP32 rounding.
- Longer runs: the concentration error against the FP64 oracle and the drift of
  the FP64 mass totals stay within the bounds stated in each test (measured on
  GB300 and recorded in the benchmark's error report).
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

P_BITS = {"fp16": 11, "bf16": 8}


def _bf16_round(x32):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _encode(P, Q, prec):
    """What the packed 16-bit format stores for conventional populations P[3][Q][N]."""
    e, w, _, _ = oracle.lattice(Q)
    out = np.empty_like(P)
    for s in range(3):
        for i in range(Q):
            v = P[s, i].astype(np.float32)
            bias = np.float32(w[i]) if s == 0 else np.float32(0.0)
            d = (v - bias).astype(np.float32)
            if i == 0:
                r = d  # FP32 rest population
            else:
                r = d.astype(np.float16).astype(np.float32) if prec == "fp16" else _bf16_round(d)
            out[s, i] = (r + bias).astype(np.float32).astype(np.float64)
    return out


def _setup(Q, shape, C, prec, **kw):
    nx, ny, nz = shape
    par = dict(kappa=(0.01, 0.02, 0.03), alpha=1.0, tau_f=1.0, M_phi=0.1, M_psi=0.1)
    par.update(kw)
    eng = tl.TernaryLB(Q, nx, ny, nz, par["kappa"], par["alpha"], par["tau_f"], par["M_phi"],
                       par["M_psi"], precision=prec)
    p = oracle.make_params(Q, nx, ny, nz, par["kappa"], par["alpha"], par["tau_f"], par["M_phi"], par["M_psi"])
    rho, phi, psi = W.to_aux(*C)
    eng.init_fields(rho, phi, psi)
    return eng, p, oracle.init_equilibrium(p, rho, phi, psi)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("Q", [9, 19])
def test_packed_round_trip_is_the_documented_encoding(prec, Q):
    shape = (37, 5, 1) if Q == 9 else (33, 4, 3)
    sh = (shape[1], shape[0]) if Q == 9 else (shape[2], shape[1], shape[0])
    eng, p, pops = _setup(Q, shape, W.spinodal(sh, seed=4, amp=0.3), prec)
    P = np.stack(pops)
    rng = np.random.default_rng(9)
    P = P + rng.uniform(-2e-3, 2e-3, P.shape)
    eng.set_populations(P)
    got = eng.get_populations()
    assert np.array_equal(got, _encode(P, Q, prec))
    assert eng.state_bytes == (3 * Q + 3) * 64 * ((shape[0] + 31) // 32) * shape[1] * shape[2]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("kernel", ["fused", "split"])
def test_packed_one_step_matches_oracle_within_storage_rounding(prec, kernel):
    C = W.lens(96, 80, 14.0, 1.0, 20.0, 60.0, (48.0, 60.0))
    eng, p, _ = _setup(9, (96, 80, 1), C, prec)
    eng.set_kernel(kernel)
    eng.step(50)
    P0 = eng.get_populations()
    f, g, k = (np.ascontiguousarray(P0[s]) for s in range(3))
    oracle.step(p, f, g, k, 1)
    eng.step(1)
    P1 = eng.get_populations()
    _, w, _, _ = oracle.lattice(9)
    for s, want in enumerate((f, g, k)):
        bias = np.zeros((9, 1))
        if s == 0:
            bias[1:, 0] = w[1:]
        tol = 2.0 ** -P_BITS[prec] * np.abs(want - bias) * 1.01 + 5e-7
        tol[0] = tol[1:].sum(axis=0) + 1e-6 * np.abs(want[0])  # FP32 rest population
        assert np.all(np.abs(P1[s] - want) <= tol), (s, float(np.max(np.abs(P1[s] - want) - tol)))


# error bounds of the longer runs: max |dC| against the FP64 oracle
LENS_BOUND = {"fp16": 2e-4, "bf16": 1e-3}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_packed_lens_error_against_fp64_oracle(prec):
    C = W.lens(96, 80, 14.0, 1.0, 20.0, 60.0, (48.0, 60.0))
    eng, p, pops = _setup(9, (96, 80, 1), C, prec)
    m0 = eng.mass()
    eng.step(1000)
    oracle.step(p, *pops, 1000)
    want = oracle.fields(p, *pops)
    got = eng.fields()
    err = max(float(np.abs(got[n] - w).max()) for n, w in zip(("C1", "C2", "C3"), want[:3]))
    print(f"{prec} lens 96x80, 1000 steps: max|dC| = {err:.3e}")
    assert err <= LENS_BOUND[prec]
    drift = np.abs(eng.mass() - m0).max() / (96 * 80)
    print(f"{prec} lens mass drift per node: {drift:.3e}")
    assert drift <= 1e-7


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_packed_spinodal_3d_error_and_mass(prec):
    n = 24
    C = W.spinodal((n, n, n), seed=3)
    eng, p, pops = _setup(19, (n, n, n), C, prec, kappa=(0.01, 0.01, 0.01), tau_f=0.8)
    m0 = eng.mass()
    eng.step(300)
    oracle.step(p, *pops, 300)
    want = oracle.fields(p, *pops)
    got = eng.fields()
    err = max(float(np.abs(got[nm] - w).max()) for nm, w in zip(("C1", "C2", "C3"), want[:3]))
    print(f"{prec} spinodal 24^3, 300 steps: max|dC| = {err:.3e}")
    assert err <= LENS_BOUND[prec]
    drift = np.abs(eng.mass() - m0).max() / n ** 3
    print(f"{prec} spinodal mass drift per node: {drift:.3e}")
    assert drift <= 1e-7
