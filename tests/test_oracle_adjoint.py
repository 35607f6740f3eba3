"""The differentiable oracle (oracle/adjoint.py) pinned to the C oracle.

- Forward: the PyTorch restatement reproduces the C oracle's populations after
  initialisation and several steps (walls with wetting, D2Q9; periodic D3Q19)
  to 1e-12.
- Gradients: autograd's dL/dkappa_m, dL/dh_m and dL/d(initial field at a node)
  agree with central finite differences of the C oracle's loss (step 1e-6 in
  kappa and h, 1e-5 in the fields) to 1e-6 relative -- the finite differences
  use the C code only, so a wrong term anywhere in the restatement or in its
  autograd graph fails here.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as OA
from paper_1511_02155_gb300 import workloads as W

torch = pytest.importorskip("torch")

NX, NY = 20, 12
KAP = (0.012, 0.02, 0.016)
H = (0.0006, -0.0004, 0.0003)
TAU_F, M_PHI, M_PSI, ALPHA = 0.9, 0.3, 0.2, 1.1


def _case():
    C, solid = W.sessile_drop(NX, NY, 5.0, m=2, n=0)
    rho, phi, psi = W.to_aux(*C)
    for a in (rho, phi, psi):
        a[solid != 0] = 0.0
    rng = np.random.default_rng(5)
    target = np.clip(psi + 0.05 * rng.standard_normal(psi.shape), 0, 1)
    return rho.reshape(-1), phi.reshape(-1), psi.reshape(-1), solid.reshape(-1), target.reshape(-1)


def _c_loss(kap, h, rho, phi, psi, solid, target, nsteps):
    p = oracle.make_params(9, NX, NY, 1, kap, ALPHA, TAU_F, M_PHI, M_PSI, h)
    pops = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    oracle.step(p, *pops, nsteps, solid)
    C3 = oracle.fields(p, *pops, solid)[2]
    d = (C3 - target) * (solid == 0)
    return float((d * d).sum())


def test_forward_matches_c_oracle_walls_d2q9():
    rho, phi, psi, solid, _ = _case()
    got = OA.forward_pops(9, NX, NY, 1, KAP, ALPHA, TAU_F, M_PHI, M_PSI, H, rho, phi, psi, 6, solid)
    p = oracle.make_params(9, NX, NY, 1, KAP, ALPHA, TAU_F, M_PHI, M_PSI, H)
    pops = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    oracle.step(p, *pops, 6, solid)
    assert np.abs(got - np.stack(pops)).max() <= 1e-12


def test_forward_matches_c_oracle_periodic_d3q19():
    n = (7, 6, 5)
    C = W.spinodal((n[2], n[1], n[0]), seed=2, amp=0.2)
    rho, phi, psi = (a.reshape(-1) for a in W.to_aux(*C))
    got = OA.forward_pops(19, *n, KAP, ALPHA, TAU_F, M_PHI, M_PSI, (0, 0, 0), rho, phi, psi, 3)
    p = oracle.make_params(19, *n, KAP, ALPHA, TAU_F, M_PHI, M_PSI)
    pops = oracle.init_equilibrium(p, rho, phi, psi)
    oracle.step(p, *pops, 3)
    assert np.abs(got - np.stack(pops)).max() <= 1e-12


def test_gradients_match_central_differences_of_the_c_oracle():
    rho, phi, psi, solid, target = _case()
    T = 8
    loss, dk, dh, drho, dphi, dpsi = OA.gradients(9, NX, NY, 1, KAP, ALPHA, TAU_F, M_PHI, M_PSI, H,
                                                  rho, phi, psi, target, T, solid)
    assert loss == pytest.approx(_c_loss(KAP, H, rho, phi, psi, solid, target, T), rel=1e-12)

    def fd(fun, x0, eps):
        return (fun(x0 + eps) - fun(x0 - eps)) / (2 * eps)

    for m in range(3):
        def fk(v, m=m):
            k = list(KAP)
            k[m] = v
            return _c_loss(k, H, rho, phi, psi, solid, target, T)

        def fh(v, m=m):
            hh = list(H)
            hh[m] = v
            return _c_loss(KAP, hh, rho, phi, psi, solid, target, T)

        assert dk[m] == pytest.approx(fd(fk, KAP[m], 1e-6), rel=1e-6, abs=1e-9)
        assert dh[m] == pytest.approx(fd(fh, H[m], 1e-6), rel=1e-6, abs=1e-9)
    fluid = np.nonzero(solid == 0)[0]
    rng = np.random.default_rng(1)
    for name, arr, grad in (("rho", rho, drho), ("phi", phi, dphi), ("psi", psi, dpsi)):
        for r in rng.choice(fluid, 3, replace=False):
            def ff(v, r=r, name=name):
                a = {"rho": rho.copy(), "phi": phi.copy(), "psi": psi.copy()}
                a[name][r] = v
                return _c_loss(KAP, H, a["rho"], a["phi"], a["psi"], solid, target, T)

            assert grad[r] == pytest.approx(fd(ff, arr[r], 1e-5), rel=1e-6, abs=1e-9), (name, r)
