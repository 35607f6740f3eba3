"""The GPU adjoint (tlbm_adjoint_c3_misfit) against independent gradients.

- Against the FP64 PyTorch-autograd oracle (oracle/adjoint.py, itself pinned to
  the C oracle's finite differences): D2Q9 32x16 with a bottom wall and a lid
  (wetting on), D3Q19 with walls and a step, periodic D2Q9 and periodic
  D3Q19; loss to 1e-12 relative,
  dL/dkappa and dL/dh to 1e-9 relative, dL/dfields to 1e-9 of their largest
  magnitude.
- Against central finite differences (step 1e-4 relative) of the GPU's own FP64
  forward on the inverse-wetting lattice (D2Q9 256x128, wall at y = 0, lid),
  300 steps: 1e-5 relative.
- The checkpoint interval changes nothing (bitwise), the engine ends at the
  forward state, and the torch.autograd.Function returns the same gradients.
- FP32 storage (adjoint in FP32, loss and parameter gradients summed in FP64)
  against the FP64 adjoint: loss to 1e-5 relative, dL/dkappa and dL/dh to 1e-3
  relative, dL/dfields to 1e-3 of their largest magnitude (D2Q9 with walls,
  20 and 300 steps; FP32 rounding of the forward and backward sweeps).
"""
import numpy as np
import pytest

from oracle import adjoint as OA
import paper_1511_02155_gb300 as tl
from paper_1511_02155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

PAR = dict(alpha=1.0, tau_f=0.9, M_phi=0.3, M_psi=0.2)


def _drop_case(nx, ny, R, seed=3, noise=0.05):
    C, solid = W.sessile_drop(nx, ny, R, m=2, n=0)
    rho, phi, psi = W.to_aux(*C)
    for a in (rho, phi, psi):
        a[solid != 0] = 0.0
    rng = np.random.default_rng(seed)
    target = np.clip(psi + noise * rng.standard_normal(psi.shape), 0, 1)
    return [a.reshape(-1) for a in (rho, phi, psi)], solid.reshape(-1), target.reshape(-1)


def _gpu(Q, shape, kap, h, fields, solid, target, T, K, prec="fp64"):
    eng = tl.TernaryLB(Q, *shape, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], h, solid, prec)
    eng.init_fields(*fields)
    out = eng.adjoint_c3_misfit(T, K, target)
    return eng, out


def _compare(got, want):
    loss, dk, dh, df = got
    wl, wk, wh, *wf = want
    assert loss == pytest.approx(wl, rel=1e-12)
    assert np.allclose(dk, wk, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(wk).max())), (dk, wk)
    assert np.allclose(dh, wh, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(wh).max())), (dh, wh)
    for c in range(3):
        scale = max(np.abs(wf[c]).max(), 1e-30)
        assert np.abs(df[c] - wf[c]).max() <= 1e-9 * scale, (c, np.abs(df[c] - wf[c]).max() / scale)


def test_walls_d2q9_against_autograd_oracle():
    nx, ny = 32, 16
    fields, solid, target = _drop_case(nx, ny, 7.0)
    kap, h = (0.012, 0.02, 0.016), (0.0006, -0.0004, 0.0003)
    T = 20
    want = OA.gradients(9, nx, ny, 1, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], h, *fields,
                        target, T, solid)
    eng, got = _gpu(9, (nx, ny, 1), kap, h, fields, solid, target, T, 7)
    _compare(got, want)
    assert eng.steps_done == T
    eng.close()


def test_periodic_d2q9_and_d3q19_against_autograd_oracle():
    kap = (0.01, 0.015, 0.02)
    C = W.lens(24, 20, 5.0, 1.0, 5.0, 15.0, (12.0, 15.0))
    fields = [a.reshape(-1) for a in W.to_aux(*C)]
    target = np.roll(fields[2], 3)
    want = OA.gradients(9, 24, 20, 1, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], (0, 0, 0),
                        *fields, target, 12)
    eng, got = _gpu(9, (24, 20, 1), kap, (0, 0, 0), fields, None, target, 12, 5)
    _compare(got, want)
    assert np.all(got[2] == 0.0)  # no wall: h does not enter
    eng.close()
    n = (8, 6, 5)
    C = W.spinodal((n[2], n[1], n[0]), seed=4, amp=0.2)
    fields = [a.reshape(-1) for a in W.to_aux(*C)]
    target = np.full(fields[2].shape, 1.0 / 3.0)
    want = OA.gradients(19, *n, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], (0, 0, 0), *fields,
                        target, 4)
    eng, got = _gpu(19, n, kap, (0, 0, 0), fields, None, target, 4, 3)
    _compare(got, want)
    eng.close()


def test_walls_d3q19_against_autograd_oracle():
    nx, ny, nz = 8, 7, 6
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    solid[1:3, 1, 2:4] = 1  # a step on the bottom wall (edges and corners)
    C = W.spinodal((nz, ny, nx), seed=6, amp=0.2)
    rho, phi, psi = W.to_aux(*C)
    for a in (rho, phi, psi):
        a[solid != 0] = 0.0
    fields = [a.reshape(-1) for a in (rho, phi, psi)]
    solid = solid.reshape(-1)
    target = np.full(fields[2].shape, 0.3) * (solid == 0)
    kap, h = (0.012, 0.02, 0.016), (0.0006, -0.0004, 0.0003)
    want = OA.gradients(19, nx, ny, nz, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], h, *fields,
                        target, 5, solid)
    eng, got = _gpu(19, (nx, ny, nz), kap, h, fields, solid, target, 5, 2)
    _compare(got, want)
    eng.close()


def test_checkpoint_interval_changes_nothing_and_engine_ends_forward():
    nx, ny = 32, 16
    fields, solid, target = _drop_case(nx, ny, 7.0)
    kap, h = (0.012, 0.02, 0.016), (0.0006, -0.0004, 0.0003)
    res = []
    for K in (1, 4, 9, 30):
        eng, out = _gpu(9, (nx, ny, 1), kap, h, fields, solid, target, 9, K)
        res.append(out)
        P = eng.get_populations()
        eng.close()
    ref = tl.TernaryLB(9, nx, ny, 1, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], h, solid, "fp64")
    ref.init_fields(*fields)
    ref.step(9)
    assert np.array_equal(P, ref.get_populations())
    ref.close()
    for r in res[1:]:
        assert r[0] == res[0][0]
        for a, b in zip(r[1:], res[0][1:]):
            assert np.array_equal(a, b)


def test_inverse_wetting_lattice_against_finite_differences():
    nx, ny, T = 256, 128, 300
    fields, solid, target = _drop_case(nx, ny, 40.0, noise=0.02)
    kap, h = (0.01, 0.012, 0.014), (0.0005, -0.0003, 0.0002)
    eng, (loss, dk, dh, _) = _gpu(9, (nx, ny, 1), kap, h, fields, solid, target, T, 50)
    eng.close()

    def L(k, hh):
        e = tl.TernaryLB(9, nx, ny, 1, k, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], hh, solid, "fp64")
        e.init_fields(*fields)
        e.step(T)
        C3 = e.fields()["C3"]
        e.close()
        d = (C3 - target) * (solid == 0)
        return float((d * d).sum())

    assert L(kap, h) == pytest.approx(loss, rel=1e-12)
    for m in range(3):
        dkm = 1e-4 * kap[m]
        kp, km = list(kap), list(kap)
        kp[m] += dkm
        km[m] -= dkm
        fd = (L(kp, h) - L(km, h)) / (2 * dkm)
        assert dk[m] == pytest.approx(fd, rel=1e-5), ("kappa", m, dk[m], fd)
        dhm = 1e-4 * max(abs(h[m]), 1e-4)
        hp, hm = list(h), list(h)
        hp[m] += dhm
        hm[m] -= dhm
        fd = (L(kap, hp) - L(kap, hm)) / (2 * dhm)
        assert dh[m] == pytest.approx(fd, rel=1e-5), ("h", m, dh[m], fd)


def test_autograd_function_and_preconditions():
    from paper_1511_02155_gb300.inverse import c3_misfit
    nx, ny = 32, 16
    fields, solid, target = _drop_case(nx, ny, 7.0)
    kap, h = (0.012, 0.02, 0.016), (0.0006, -0.0004, 0.0003)
    tk = torch.tensor(kap, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    tf = [torch.tensor(f, requires_grad=True) for f in fields]
    loss = c3_misfit(tk, th, *tf, torch.tensor(target), nx=nx, ny=ny, solid=solid, nsteps=10,
                     checkpoint_every=4, **PAR)
    (2.0 * loss).backward()
    eng, (l2, dk, dh, df) = _gpu(9, (nx, ny, 1), kap, h, fields, solid, target, 10, 4)
    eng.close()
    assert float(loss.detach()) == l2
    assert np.array_equal(tk.grad.numpy(), 2.0 * dk)
    assert np.array_equal(th.grad.numpy(), 2.0 * dh)
    for c in range(3):
        assert np.array_equal(tf[c].grad.numpy(), 2.0 * df[c])
    # 16-bit storage and a stepped state are refused
    e16 = tl.TernaryLB(9, nx, ny, 1, kap, 1.0, 0.9, 0.3, 0.2, h, solid, "fp16")
    e16.init_fields(*fields)
    with pytest.raises(tl.TLBMError):
        e16.adjoint_c3_misfit(5, 2, target)
    e16.close()
    e64 = tl.TernaryLB(9, nx, ny, 1, kap, 1.0, 0.9, 0.3, 0.2, h, solid, "fp64")
    e64.init_fields(*fields)
    e64.step(1)
    with pytest.raises(tl.TLBMError):
        e64.adjoint_c3_misfit(5, 2, target)
    e64.close()


@pytest.mark.parametrize("shape,T,R", [((32, 16), 20, 7.0), ((256, 128), 300, 40.0)])
def test_fp32_adjoint_against_fp64(shape, T, R):
    nx, ny = shape
    fields, solid, target = _drop_case(nx, ny, R, noise=0.02)
    kap, h = (0.01, 0.012, 0.014), (0.0005, -0.0003, 0.0002)
    out = {}
    for prec in ("fp64", "fp32"):
        eng, out[prec] = _gpu(9, (nx, ny, 1), kap, h, fields, solid, target, T, 50, prec)
        eng.close()
    (l64, k64, h64, f64), (l32, k32, h32, f32) = out["fp64"], out["fp32"]
    print(f"{nx}x{ny} T={T}: loss {l64:.8e} vs {l32:.8e}; dkappa {k64} vs {k32}; dh {h64} vs {h32}")
    assert l32 == pytest.approx(l64, rel=1e-5)
    assert np.allclose(k32, k64, rtol=1e-3, atol=1e-3 * np.abs(k64).max())
    assert np.allclose(h32, h64, rtol=1e-3, atol=1e-3 * np.abs(h64).max())
    for c in range(3):
        assert np.abs(f32[c] - f64[c]).max() <= 1e-3 * np.abs(f64[c]).max()


def test_gradient_descent_recovers_hidden_wetting_parameters():
    """Inverse wetting with the autograd wrapper: a target C_3 field made with
    hidden h*, a start 40 % away (contact angles 3-7 degrees off), and L-BFGS-B
    (scipy) driven by the adjoint's gradient: the misfit falls by 100x and the
    recovered h gives the hidden contact angles to 0.5 degrees.  (h itself is
    determined only up to the direction that leaves every angle unchanged --
    only differences of solid-fluid tensions enter, Sec. Inverting the contact
    angle relations -- so the angles, not h, are compared.)"""
    optimize = pytest.importorskip("scipy.optimize")
    from paper_1511_02155_gb300.inverse import c3_misfit
    nx, ny, T = 64, 32, 400
    fields, solid, _ = _drop_case(nx, ny, 12.0)
    kap = (0.01, 0.012, 0.014)
    h_star = np.array([0.0006, -0.0004, 0.0002])
    eng = tl.TernaryLB(9, nx, ny, 1, kap, PAR["alpha"], PAR["tau_f"], PAR["M_phi"], PAR["M_psi"], tuple(h_star),
                       solid, "fp64")
    eng.init_fields(*fields)
    eng.step(T)
    target = torch.tensor(eng.fields()["C3"] * (solid == 0))
    eng.close()
    tk = torch.tensor(kap, dtype=torch.float64)
    tf = [torch.tensor(f) for f in fields]
    scale = 1e-3  # optimise u = h / scale

    def fun(u):
        h = torch.tensor(u * scale, dtype=torch.float64, requires_grad=True)
        loss = c3_misfit(tk, h, *tf, target, nx=nx, ny=ny, solid=solid, nsteps=T, checkpoint_every=100, **PAR)
        loss.backward()
        return float(loss.detach()), h.grad.numpy() * scale

    u0 = h_star * 1.4 / scale
    l0 = fun(u0)[0]
    bounds = [(-0.2 * k / scale, 0.2 * k / scale) for k in kap]  # |4 h| < 0.8 alpha kappa
    res = optimize.minimize(fun, u0, jac=True, method="L-BFGS-B", bounds=bounds, options={"maxiter": 25})
    h = res.x * scale
    print("loss", l0, "->", res.fun, "h", h, "h*", h_star, "evaluations", res.nfev)
    assert res.fun < 0.01 * l0
    got, want = tl.contact_angles(kap, PAR["alpha"], h), tl.contact_angles(kap, PAR["alpha"], h_star)
    print("angles", got, "hidden", want)
    assert np.max(np.abs(np.subtract(got, want))) <= 0.5
