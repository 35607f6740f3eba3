"""Inverse wetting through the hand-written adjoint: a torch.autograd.Function.

``c3_misfit(kappa, h, rho0, phi0, psi0, target, ...)`` returns the loss
L = sum over fluid nodes of (C_3(T) - target)^2 after T steps of the ternary
LB method from the equilibrium of the initial fields, as a differentiable
torch scalar: its backward hands back dL/dkappa_m, dL/dh_m and dL/d(initial
fields), all computed on the GPU by ``tlbm_adjoint_c3_misfit`` (forward with
checkpoints, adjoint back).  The surface tensions follow kappa
(gamma_mn = alpha (kappa_m + kappa_n) / 6) and the contact angles follow h, so
a gradient-based optimiser over these tensors calibrates them against a
target field.  Only marshalling happens here; there is no CPU path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import TernaryLB


class C3Misfit(torch.autograd.Function):
    """Loss of the C_3 misfit; gradients from the library's adjoint."""

    @staticmethod
    def forward(ctx, kappa, h, rho0, phi0, psi0, target, cfg):
        k = [float(v) for v in kappa.detach().cpu().reshape(-1)]
        hh = [float(v) for v in h.detach().cpu().reshape(-1)]
        eng = TernaryLB(cfg["lattice"], cfg["nx"], cfg["ny"], cfg.get("nz", 1), k, cfg["alpha"], cfg["tau_f"],
                        cfg["M_phi"], cfg["M_psi"], hh, cfg.get("solid"), cfg.get("precision", "fp64"))
        try:
            f = [t.detach().cpu().double().numpy().reshape(-1) for t in (rho0, phi0, psi0)]
            eng.init_fields(*f)
            loss, dk, dh, df = eng.adjoint_c3_misfit(cfg["nsteps"], cfg.get("checkpoint_every", 100),
                                                     target.detach().cpu().double().numpy().reshape(-1))
        finally:
            eng.close()
        ctx.save_for_backward(torch.from_numpy(dk), torch.from_numpy(dh), torch.from_numpy(df))
        ctx.shapes = (kappa.shape, h.shape, rho0.shape)
        ctx.devices = (kappa.device, h.device, rho0.device)
        return torch.tensor(loss, dtype=torch.float64, device=kappa.device)

    @staticmethod
    def backward(ctx, grad_out):
        dk, dh, df = ctx.saved_tensors
        g = grad_out.detach().double().cpu()
        ks, hs, fs = ctx.shapes
        kd, hd, fd = ctx.devices
        out = [(g * dk).reshape(ks).to(kd), (g * dh).reshape(hs).to(hd)]
        out += [(g * df[c]).reshape(fs).to(fd) for c in range(3)]
        return (*out, None, None)


def c3_misfit(kappa, h, rho0, phi0, psi0, target, *, lattice=9, nx, ny, nz=1, alpha=1.0, tau_f=1.0, M_phi=0.1,
              M_psi=0.1, solid=None, nsteps, checkpoint_every=100, precision="fp64"):
    """Differentiable C_3 misfit (see the module docstring); precision "fp64" or
    "fp32" (the adjoint then runs in FP32 with FP64 parameter sums)."""
    cfg = dict(lattice=lattice, nx=nx, ny=ny, nz=nz, alpha=alpha, tau_f=tau_f, M_phi=M_phi, M_psi=M_psi,
               solid=None if solid is None else np.asarray(solid).reshape(-1), nsteps=nsteps,
               checkpoint_every=checkpoint_every, precision=precision)
    return C3Misfit.apply(kappa, h, rho0, phi0, psi0, target, cfg)
