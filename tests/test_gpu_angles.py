"""Contact angles of sessile drops against Young's equation (Sec. Contact Angles).

Fluid-3 drops in fluid 1 on a flat wall, h from the library's inversion of the
target angle theta_31 (through the drop; theta_12 = 90 fixes the gauge's other
pair), all members advanced together as one batch under a CUDA graph.  Each
target is approached from a cap 5 degrees below and one 5 degrees above it;
the angle is read off the C_3 = 1/2 contour by a circle fit.

Bounds, from runs on GB300 (200x100 lattices, drop area of a half disc of
radius 30; alpha = 1, tau = 1, tau_psi = 2/3, kappa = 0.01 each, as in the
paper's Fig. 2 settings):
- both starts settle on the same angle (within 0.5 degrees);
- the settled angle is within 3 degrees of Young's prediction over
  60..135 degrees.  The measured cos(theta) exceeds the predicted one by a
  near-constant factor of about 1.05, so the deviation grows toward the ends of
  the range (about 5 degrees at 150, 11 at 160); the paper reports at most
  4 degrees over 14..166.
- FP32, FP16 and BF16 storage give angles within 0.5 degrees of FP64 (the
  FP64 engine itself matches the FP64 oracle to 1e-12).
"""
import numpy as np
import pytest

import paper_1511_02155_gb300 as tl
from paper_1511_02155_gb300 import workloads as W
from contact_angle import drop_angle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KAPPA = (0.01, 0.01, 0.01)
NX, NY, R_HALF = 200, 100, 30.0


def _drop(target, start, precision):
    h = tl.wetting_from_angles(KAPPA, 1.0, 90.0, 180.0 - target)
    th = np.radians(start)
    R = np.sqrt(np.pi * R_HALF ** 2 / 2 / (th - np.sin(th) * np.cos(th)))  # same area for every start
    C, solid = W.sessile_drop(NX, NY, R, m=2, n=0, theta0=start)
    rho, phi, psi = W.to_aux(*C)
    for a in (rho, phi, psi):
        a[solid != 0] = 0.0
    eng = tl.TernaryLB(9, NX, NY, 1, KAPPA, 1.0, 1.0, 0.5, 1.0 / 6.0, h, solid, precision)
    eng.init_fields(rho, phi, psi)
    return eng


def _angle(eng):
    return drop_angle(eng.fields()["C3"].reshape(NY, NX), 0.5)[0]


def test_sessile_drop_angles_follow_young():
    targets = (60.0, 90.0, 120.0, 135.0)
    engines = [_drop(t, t + d, "fp32") for t in targets for d in (-5.0, 5.0)]
    with tl.TernaryBatch(engines) as b:
        b.set_graph(True)
        b.step(300000)
    got = [_angle(e) for e in engines]
    for k, t in enumerate(targets):
        lo, hi = got[2 * k], got[2 * k + 1]
        young = tl.contact_angles(KAPPA, 1.0, tl.wetting_from_angles(KAPPA, 1.0, 90.0, 180.0 - t))[2]
        assert young == pytest.approx(t, abs=1e-6)
        print(f"target {t:.0f}: from below {lo:.2f}, from above {hi:.2f}")
        assert abs(lo - hi) <= 0.5
        assert abs(0.5 * (lo + hi) - t) <= 3.0
    for e in engines:
        e.close()


def test_storage_precisions_give_the_same_angles():
    out = {}
    for prec in ("fp32", "fp64", "fp16", "bf16"):
        engines = [_drop(t, t, prec) for t in (60.0, 120.0)]
        with tl.TernaryBatch(engines) as b:
            b.set_graph(True)
            b.step(40000)
        out[prec] = [_angle(e) for e in engines]
    print(out)
    for prec in ("fp32", "fp16", "bf16"):
        assert np.max(np.abs(np.subtract(out[prec], out["fp64"]))) <= 0.5, prec
