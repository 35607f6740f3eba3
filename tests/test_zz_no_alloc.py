"""tlbm_step_noalloc, the allocation-free step for callers that may not allocate
device memory (a plug-in inside a framework that owns every device allocation
through its own pool and budget, or a time-critical loop), against the engine's
own split step through the C ABI, on two calls in a row.

The allocation-free step runs the engine's split-step kernels with the same
parameters, only with its intermediate arrays in a fixed per-device buffer, so
the populations and the FP64 totals of both must agree bitwise in FP64 and in
FP32 (tolerance 0)."""
import ctypes

import numpy as np
import pytest

import paper_1511_02155_gb300 as tl
from paper_1511_02155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _noalloc():
    lib = tl.load_library()
    f = lib.tlbm_step_noalloc
    d = ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, d, d, d, d, dp,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.tlbm_noalloc_last_error.restype = ctypes.c_char_p
    return lib, f


CASES = [
    # lattice, shape, precision, kappa, h, solid builder, tolerance on populations
    (9, (40, 30, 1), "fp64", (0.01, 0.02, 0.03), (0.0005, -0.0008, 0.001), "sessile", 0.0),
    (19, (20, 12, 10), "fp32", (0.012, 0.01, 0.02), (0.0, 0.0, 0.0), None, 0.0),
    (9, (33, 21, 1), "fp32", (0.01, 0.02, 0.03), (0.0005, -0.0008, 0.001), "sessile", 0.0),
]


@pytest.mark.parametrize("Q,shape,prec,kappa,h,solid_kind,tol", CASES)
def test_noalloc_step_matches_engine_on_two_calls(Q, shape, prec, kappa, h, solid_kind, tol):
    lib, step = _noalloc()
    nx, ny, nz = shape
    if solid_kind == "sessile":
        C, solid = W.sessile_drop(nx, ny, 8.0, m=2, n=0)
    else:
        C, solid = W.spinodal((nz, ny, nx), seed=6, amp=0.05), None
    rho, phi, psi = W.to_aux(*C)
    if solid is not None:
        for a in (rho, phi, psi):
            a[solid != 0] = 0.0
    eng = tl.TernaryLB(Q, nx, ny, nz, kappa, 1.0, 0.9, 0.1, 0.15, h, solid, prec)
    eng.set_kernel("split")
    eng.init_fields(rho, phi, psi)
    dtype = np.float64 if prec == "fp64" else np.float32
    state0 = eng.get_state()
    src = torch.from_numpy(state0.copy()).cuda()
    dst = torch.zeros_like(src)
    mass = torch.zeros(3, dtype=torch.float64, device="cuda")
    sol = None if solid is None else torch.from_numpy(np.ascontiguousarray(solid.reshape(-1), dtype=np.uint8)).cuda()
    k = (ctypes.c_double * 3)(*kappa)
    hh = (ctypes.c_double * 3)(*h)
    stream = torch.cuda.current_stream().cuda_stream
    precision = tl.FP64 if prec == "fp64" else tl.FP32
    for call in range(2):
        rc = step(Q, precision, nx, ny, nz, k, 1.0, 0.9, 0.1, 0.15, hh,
                  None if sol is None else sol.data_ptr(), src.data_ptr(), dst.data_ptr(),
                  mass.data_ptr(), stream)
        assert rc == 0, lib.tlbm_noalloc_last_error().decode()
        eng.step(1)
        torch.cuda.synchronize()
        want = eng.get_state().view(dtype)
        got = dst.cpu().numpy().view(dtype)
        assert np.abs(got - want).max() <= tol, (call, np.abs(got - want).max())
        # FP64 totals of each call's input state, summed in the same order
        assert np.array_equal(mass.cpu().numpy(), np.asarray(eng.step_mass()))
        src, dst = dst, src


def test_noalloc_rejects_oversized_lattice_before_any_launch():
    lib, step = _noalloc()
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    k = (ctypes.c_double * 3)(0.01, 0.02, 0.03)
    rc = step(9, tl.FP64, 1024, 1024, 1, k, 1.0, 1.0, 0.1, 0.1, None, None, buf.data_ptr(),
              buf[8:].data_ptr(), None, None)
    assert rc == tl.STATUS.index("TLBM_ERR_ARG")
    assert "too large" in lib.tlbm_noalloc_last_error().decode()


@pytest.mark.parametrize("bad", ["kappa_inf", "tau_inf", "alpha_nan", "mobility_inf", "h_nan"])
def test_noalloc_rejects_non_finite_parameters_before_any_launch(bad):
    lib, step = _noalloc()
    buf = torch.zeros(2 * 9 * 3 * 32 * 8, dtype=torch.uint8, device="cuda")
    half = buf.numel() // 2
    kap = [0.01, 0.02, 0.03]
    h = [0.0, 0.0, 0.0]
    alpha, tau, mphi = 1.0, 1.0, 0.1
    if bad == "kappa_inf":
        kap[1] = float("inf")
    elif bad == "tau_inf":
        tau = float("inf")
    elif bad == "alpha_nan":
        alpha = float("nan")
    elif bad == "mobility_inf":
        mphi = float("inf")
    else:
        h[2] = float("nan")
    rc = step(9, tl.FP64, 4, 4, 1, (ctypes.c_double * 3)(*kap), alpha, tau, mphi, 0.1, (ctypes.c_double * 3)(*h),
              None, buf.data_ptr(), buf[half:].data_ptr(), None, None)
    assert rc == tl.STATUS.index("TLBM_ERR_PARAM"), lib.tlbm_noalloc_last_error().decode()
