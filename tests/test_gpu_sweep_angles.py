"""Contact-angle sweep (Sec. Contact Angles, Fig. 2 settings): square-well
members of the 96-lattice sweep, batched (one launch per step under a CUDA
graph), against the analytic contact angle of the model's wetting theory
(Young's equation with gamma_sm = I_m + sum J_n, Eq. solidST, and
gamma_mn = alpha (kappa_m + kappa_n) / 6, Eq. SurfTens).

Each member (workloads.sweep_wells) has its well's lower half filled with
fluid 3 under fluid 1, and h from the library's inversion of its target pair
(theta_12, theta_13) in [30, 150) degrees.  The angle measured is theta_31,
where the fluid-3/fluid-1 meniscus meets the well's side walls
(tests/well_angle.py: circle fit to the C_3 = 1/2 crossings; the meniscus must
be free -- contact line and apex away from the well's corners and floor).

The representative subset is every fourth member (24 lattices from 128x64 to
768x384).  After 150000 steps every free member's angle is within the paper's
4 degree band of the prediction; at the configured 20000 steps narrow wells
have settled but wide ones (width ~100) are still moving.  Measured on GB300
over all 96 members: see the design notes.

Run as a script (python tests/test_gpu_sweep_angles.py) to print every
member's angle at 20000, 60000 and 150000 steps.
"""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
for _p in (HERE, os.path.dirname(HERE)):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import paper_1511_02155_gb300 as tl  # noqa: E402
from paper_1511_02155_gb300 import workloads as W  # noqa: E402
from well_angle import meniscus_angle  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

BAND = 4.0  # degrees (the paper's accuracy over 14..166 degrees)


def build(members):
    engines = []
    for m in members:
        for a in m["angles"]:
            try:
                m["h"] = tl.wetting_from_angles(m["kappa"], m["alpha"], *a)
                break
            except tl.TLBMError:
                continue
        rho, phi, psi = W.to_aux(*m["C"])
        m["C"] = None
        for a in (rho, phi, psi):
            a[m["solid"] != 0] = 0.0
        e = tl.TernaryLB(9, m["nx"], m["ny"], 1, m["kappa"], m["alpha"], m["tau_f"], m["M_phi"], m["M_psi"],
                         m["h"], m["solid"], "fp32")
        e.init_fields(rho, phi, psi)
        m["young31"] = tl.contact_angles(m["kappa"], m["alpha"], m["h"])[2]
        engines.append(e)
    return engines


def measure(members, engines):
    out = []
    for m, e in zip(members, engines):
        C3 = e.fields()["C3"].reshape(m["ny"], m["nx"])
        theta, _, free = meniscus_angle(C3, m["well"])
        out.append((theta, free))
    return out


def run(members, checkpoints):
    engines = build(members)
    results = {}
    with tl.TernaryBatch(engines) as b:
        b.set_graph(True)
        done = 0
        for T in checkpoints:
            b.step(T - done)
            done = T
            results[T] = measure(members, engines)
    for e in engines:
        e.close()
    return results


def test_sweep_subset_angles_within_the_paper_band():
    members = W.sweep_wells(96)[::4]
    res = run(members, (20000, 150000))
    free = 0
    for k, m in enumerate(members):
        theta, ok = res[150000][k]
        print(f"member {4 * k}: {m['nx']}x{m['ny']} well {m['well']['x1'] - m['well']['x0']}x"
              f"{m['well']['y1'] - m['well']['y0']}  Young {m['young31']:.2f}  20k {res[20000][k][0]:.2f}  "
              f"150k {theta:.2f} free {ok}")
        if ok:
            free += 1
            assert abs(theta - m["young31"]) <= BAND, (4 * k, theta, m["young31"])
    assert free >= 2 * len(members) // 3


if __name__ == "__main__":
    torch.cuda.set_device(0)
    members = W.sweep_wells(96)
    res = run(members, (20000, 60000, 150000))
    for T, r in res.items():
        err = [t - m["young31"] for (t, ok), m in zip(r, members) if ok]
        print(json.dumps({"steps": T, "free": len(err), "mean": float(np.mean(err)),
                          "rms": float(np.sqrt(np.mean(np.square(err)))), "max_abs": float(np.max(np.abs(err))),
                          "within_4deg": int(np.sum(np.abs(err) <= BAND))}))
    for k, m in enumerate(members):
        print(json.dumps({"member": k, "nx": m["nx"], "well": m["well"], "young31": round(m["young31"], 3),
                          **{f"theta_{T}": (round(float(res[T][k][0]), 3), bool(res[T][k][1])) for T in res}}))
