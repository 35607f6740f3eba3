"""Writes the FP64 oracle's fields after 30000 steps of the two D2Q9 benchmark
geometries of the paper's Sec. Liquid Lense and Double Emulsion (Fig. 1), for
the GPU test that compares the FP32 and FP16-storage engines against them:

  config2_lens.npz      512x256 periodic liquid lens (fluid-3 lens of radius 60
                        on a flat 1/2 interface), kappa from seed 2
  config2_emulsion.npz  512x512 periodic double emulsion (fluid-1 core radius
                        60, fluid-3 shell to radius 100, in fluid 2), kappa
                        from seed 3

Both: alpha = 1, tau_f = 1, M_phi = M_psi = 0.1 (Gamma = 1).  The inputs are
the seeded recipes of paper_1511_02155_gb300.workloads (no step arithmetic);
every number written comes from oracle/ alone.

Storage: each field C_m is quantised to integers q = round(C_m 2^30)
(resolution 9.3e-10, far below the 1e-4 comparison), stored as differences
along x (small integers that compress well); decode() undoes both.
Run: python tests/golden/make_config2.py   (about 30 min on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STEPS = 30000
SCALE = float(2 ** 30)


def encode(C: np.ndarray) -> np.ndarray:
    q = np.round(C * SCALE).astype(np.int64)
    d = np.diff(q, axis=-1, prepend=0)
    assert np.abs(d).max() < 2 ** 31
    return d.astype(np.int32)


def decode(d: np.ndarray) -> np.ndarray:
    return np.cumsum(d.astype(np.int64), axis=-1).astype(np.float64) / SCALE


def cases():
    from paper_1511_02155_gb300 import workloads as W
    return {"lens": W.lens_512x256(), "emulsion": W.emulsion_512()}


def run(name: str, cfg: dict) -> str:
    import oracle
    nx, ny = cfg["nx"], cfg["ny"]
    p = oracle.make_params(9, nx, ny, 1, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"], cfg["M_psi"])
    f, g, k = oracle.init_equilibrium(p, *W_to_aux(cfg["C"]))
    m0 = oracle.mass(p, f, g, k)
    t0 = time.time()
    oracle.step(p, f, g, k, STEPS)
    C1, C2, C3, rho, u = oracle.fields(p, f, g, k)
    m1 = oracle.mass(p, f, g, k)
    out = os.path.join(HERE, f"config2_{name}.npz")
    np.savez_compressed(out, C1=encode(C1.reshape(ny, nx)), C2=encode(C2.reshape(ny, nx)),
                        C3=encode(C3.reshape(ny, nx)), kappa=np.asarray(cfg["kappa"]), steps=STEPS,
                        mass0=np.asarray(m0), mass1=np.asarray(m1),
                        umax=float(np.abs(u).max()))
    print(f"{name}: {STEPS} steps in {time.time() - t0:.0f} s, |u|max {np.abs(u).max():.3e}, "
          f"mass drift {np.abs(np.asarray(m1) - np.asarray(m0)).max():.3e} -> {out}", flush=True)
    return out


def W_to_aux(C):
    from paper_1511_02155_gb300 import workloads as W
    return W.to_aux(*C)


if __name__ == "__main__":
    which = sys.argv[1:] or ["lens", "emulsion"]
    cs = cases()
    for name in which:
        run(name, cs[name])
