"""FP64 CPU oracle of the ternary free-energy lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the GPU
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does.  It shares no code
with the CUDA path: the arithmetic lives in ``tlbm_oracle.c`` (plain C, compiled
with ``-ffp-contract=off``), this module only marshals numpy arrays.

Paper: Semprebon, Krueger, Kusumaatmaja, arXiv:1511.02155.  Each exported
function cites the section or equation it follows; see ``tlbm_oracle.c``.

Array layout everywhere: node index ``x + nx*(y + ny*z)`` (x fastest);
populations are ``[Q][N]`` float64 arrays in conventional (post-streaming)
form, i.e. ``f_i(r, t)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlbm_oracle.c")
_LIB = os.path.join(_HERE, "libtlbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C, OpenMP, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in tlbm_oracle.c."""

    _fields_ = [
        ("Q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("kappa", ctypes.c_double * 3), ("alpha", ctypes.c_double),
        ("tau", ctypes.c_double * 3), ("gamma", ctypes.c_double * 2),
        ("h", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            pp = ctypes.POINTER(Params)
            lib.orc_step.argtypes = [pp, u8p, dp, dp, dp, ctypes.c_long]
            lib.orc_step.restype = ctypes.c_int
            lib.orc_init_equilibrium.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_init_equilibrium.restype = ctypes.c_int
            lib.orc_moments.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_moments.restype = None
            lib.orc_ghosts.argtypes = [pp, u8p, dp, dp, dp]
            lib.orc_ghosts.restype = None
            lib.orc_derivatives.argtypes = [pp, dp, dp, dp]
            lib.orc_derivatives.restype = None
            lib.orc_stream.argtypes = [pp, u8p, dp, dp]
            lib.orc_stream.restype = None
            lib.orc_mass.argtypes = [pp, u8p, dp, dp, dp, dp]
            lib.orc_mass.restype = None
            lib.orc_thermo_node.argtypes = [pp, dp, dp, dp, dp, dp]
            lib.orc_thermo_node.restype = None
            lib.orc_equilibrium_node.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_equilibrium_node.restype = None
            lib.orc_wetting_gradients.argtypes = [pp, dp]
            lib.orc_wetting_gradients.restype = None
            lib.orc_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp,
                                        ctypes.POINTER(ctypes.c_int)]
            lib.orc_lattice.restype = ctypes.c_int
            lib.orc_step_guo.argtypes = [pp, dp, dp, dp, ctypes.c_long]
            lib.orc_step_guo.restype = ctypes.c_int
            lib.orc_init_equilibrium_guo.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            lib.orc_init_equilibrium_guo.restype = ctypes.c_int
            lib.orc_force.argtypes = [pp, dp, dp, dp, dp]
            lib.orc_force.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def make_params(Q, nx, ny, nz=1, kappa=(0.01, 0.02, 0.03), alpha=1.0, tau_f=1.0,
                M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), gamma_phi=1.0, gamma_psi=1.0):
    """Parameters of one run.  tau_X = 1/2 + M_X / Gamma_X (Eqs. Mobility1/2)."""
    p = Params()
    p.Q, p.nx, p.ny, p.nz = int(Q), int(nx), int(ny), int(nz)
    for m in range(3):
        p.kappa[m] = float(kappa[m])
        p.h[m] = float(h[m])
    p.alpha = float(alpha)
    p.tau[0] = float(tau_f)
    p.tau[1] = 0.5 + float(M_phi) / float(gamma_phi)
    p.tau[2] = 0.5 + float(M_psi) / float(gamma_psi)
    p.gamma[0] = float(gamma_phi)
    p.gamma[1] = float(gamma_psi)
    return p


def lattice(Q: int):
    """Velocity set, weights, gradient tensors (xx yy zz xy yz zx) and opposites."""
    lib = _load()
    e = (ctypes.c_int * (3 * Q))()
    w = np.zeros(Q)
    t = np.zeros((Q, 6))
    opp = (ctypes.c_int * Q)()
    if lib.orc_lattice(Q, e, _dp(w), _dp(t), opp) != 0:
        raise ValueError(f"unknown lattice Q={Q}")
    return np.array(list(e), dtype=np.int64).reshape(Q, 3), w, t, np.array(list(opp))


def _nodes(p):
    return p.nx * p.ny * p.nz


def init_equilibrium(p, rho, phi, psi, u=None, solid=None):
    """Populations at equilibrium with fields rho, phi, psi (and velocity u[3])."""
    lib = _load()
    N = _nodes(p)
    f = np.zeros((p.Q, N)); g = np.zeros((p.Q, N)); k = np.zeros((p.Q, N))
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(N)
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(N)
    ux = uy = uz = None
    if u is not None:
        ux, uy, uz = (np.ascontiguousarray(u[a], dtype=np.float64).reshape(N) for a in range(3))
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
    rc = lib.orc_init_equilibrium(ctypes.byref(p), _u8(sol), _dp(rho), _dp(phi), _dp(psi),
                                  _dp(ux), _dp(uy), _dp(uz), _dp(f), _dp(g), _dp(k))
    if rc != 0:
        raise RuntimeError(f"orc_init_equilibrium failed ({rc})")
    return f, g, k


def step(p, f, g, k, nsteps=1, solid=None):
    """Advance populations in place by nsteps (O1-O7 of tlbm_oracle.c)."""
    lib = _load()
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    rc = lib.orc_step(ctypes.byref(p), _u8(sol), _dp(f), _dp(g), _dp(k), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"orc_step failed ({rc})")
    return f, g, k


def moments(p, f, g, k, solid=None):
    """rho, j[3], phi, psi of conventional populations (Eq. lbconstraint)."""
    lib = _load()
    N = _nodes(p)
    out = [np.zeros(N) for _ in range(6)]
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    lib.orc_moments(ctypes.byref(p), _u8(sol), _dp(f), _dp(g), _dp(k), *[_dp(a) for a in out])
    rho, jx, jy, jz, phi, psi = out
    return rho, np.stack([jx, jy, jz]), phi, psi


def fields(p, f, g, k, solid=None):
    """C_1, C_2, C_3, rho and velocity u[3] (zeros on solid nodes)."""
    rho, j, phi, psi = moments(p, f, g, k, solid)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(rho != 0, j / np.where(rho != 0, rho, 1.0), 0.0)
    C1 = (rho + phi - psi) / 2.0
    C2 = (rho - phi - psi) / 2.0
    C3 = psi.copy()
    return C1, C2, C3, rho, u


def ghosts(p, rho, phi, psi, solid):
    """Fill rho, phi, psi in place on solid nodes (wetting ghost rule)."""
    lib = _load()
    sol = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    lib.orc_ghosts(ctypes.byref(p), _u8(sol), _dp(rho), _dp(phi), _dp(psi))


def derivatives(p, X):
    """Isotropic gradient [3][N] and Laplacian [N] of field X (periodic)."""
    lib = _load()
    N = _nodes(p)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(N)
    grad = np.zeros((3, N)); lap = np.zeros(N)
    lib.orc_derivatives(ctypes.byref(p), _dp(X), _dp(grad), _dp(lap))
    return grad, lap


def stream(p, xs, solid=None):
    """Pull streaming with halfway bounce-back of one population set [Q][N]."""
    lib = _load()
    x = np.zeros_like(xs)
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    lib.orc_stream(ctypes.byref(p), _u8(sol), _dp(np.ascontiguousarray(xs)), _dp(x))
    return x


def mass(p, f, g, k, solid=None):
    """Kahan-summed (sum rho, sum phi, sum psi) over fluid nodes."""
    lib = _load()
    out = np.zeros(3)
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    lib.orc_mass(ctypes.byref(p), _u8(sol), _dp(f), _dp(g), _dp(k), _dp(out))
    return out


def thermo_node(p, X, lap):
    """(C[3], mu[3] = (mu_rho, mu_phi, mu_psi), p_b) at one node."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    lap = np.ascontiguousarray(lap, dtype=np.float64)
    C = np.zeros(3); mu = np.zeros(3); pb = np.zeros(1)
    lib.orc_thermo_node(ctypes.byref(p), _dp(X), _dp(lap), _dp(C), _dp(mu), _dp(pb))
    return C, mu, float(pb[0])


def equilibrium_node(p, X, j, grad, lap):
    """f_eq, g_eq, k_eq (each [Q]) at one node from local values."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    j = np.ascontiguousarray(j, dtype=np.float64)
    grad = np.ascontiguousarray(grad, dtype=np.float64).reshape(3, 3)
    lap = np.ascontiguousarray(lap, dtype=np.float64)
    feq = np.zeros(p.Q); geq = np.zeros(p.Q); keq = np.zeros(p.Q)
    lib.orc_equilibrium_node(ctypes.byref(p), _dp(X), _dp(j), _dp(grad), _dp(lap),
                             _dp(feq), _dp(geq), _dp(keq))
    return feq, geq, keq


def wetting_gradients(p):
    """(G_rho, G_phi, G_psi): wall-normal gradients set by h_m (Sec. Auxiliary variables)."""
    lib = _load()
    G = np.zeros(3)
    lib.orc_wetting_gradients(ctypes.byref(p), _dp(G))
    return G


# ----------------------------------------------------- forcing coupling (Guo)

def step_guo(p, f, g, k, nsteps=1):
    """Advance populations in place by nsteps steps of the forcing coupling
    (periodic lattice; see the header of tlbm_oracle.c)."""
    lib = _load()
    rc = lib.orc_step_guo(ctypes.byref(p), _dp(f), _dp(g), _dp(k), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"orc_step_guo failed ({rc})")
    return f, g, k


def init_equilibrium_guo(p, rho, phi, psi):
    """Populations at the forcing coupling's equilibrium with the fields at rest."""
    lib = _load()
    N = _nodes(p)
    f = np.zeros((p.Q, N)); g = np.zeros((p.Q, N)); k = np.zeros((p.Q, N))
    a = [np.ascontiguousarray(x, dtype=np.float64).reshape(N) for x in (rho, phi, psi)]
    rc = lib.orc_init_equilibrium_guo(ctypes.byref(p), *[_dp(x) for x in a], _dp(f), _dp(g), _dp(k))
    if rc != 0:
        raise RuntimeError(f"orc_init_equilibrium_guo failed ({rc})")
    return f, g, k


def force(p, rho, phi, psi):
    """Body force [3][N] = -(rho grad mu_rho + phi grad mu_phi + psi grad mu_psi)."""
    lib = _load()
    N = _nodes(p)
    a = [np.ascontiguousarray(x, dtype=np.float64).reshape(N) for x in (rho, phi, psi)]
    F = np.zeros((3, N))
    rc = lib.orc_force(ctypes.byref(p), *[_dp(x) for x in a], _dp(F))
    if rc != 0:
        raise RuntimeError(f"orc_force failed ({rc})")
    return F
