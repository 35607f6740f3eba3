"""GB300-native engine for the ternary free-energy lattice Boltzmann method.

Semprebon, Krueger, Kusumaatmaja, "Ternary free energy lattice Boltzmann model
with tunable surface tensions and contact angles" (arXiv:1511.02155).

This module is a thin ctypes binding of the C ABI in ``include/tlbm.h``
(``libtlbm.so``, built in-tree by ``_build.py``): it marshals arguments and
nothing else.  Every step of the method runs in the library's CUDA kernels;
there is no CPU fallback, and constructing an engine without the library or
without a GPU raises.

PyTorch is optional plumbing: when it is importable and CUDA is available the
engine queues its work on ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["TernaryLB", "TernaryBatch", "TLBMError", "contact_angles", "wetting_from_angles", "load_library", "lib_path", "D2Q9", "D3Q19",
           "FP64", "FP32", "FP16_OFFSET", "BF16_OFFSET", "KERNEL_AUTO", "KERNEL_FUSED",
           "KERNEL_SPLIT", "COUPLING_PRESSURE_TENSOR", "COUPLING_FORCING"]

D2Q9, D3Q19 = 9, 19
FP64, FP32, FP16_OFFSET, BF16_OFFSET = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_FUSED, KERNEL_SPLIT = 0, 1, 2
COUPLING_PRESSURE_TENSOR, COUPLING_FORCING = 0, 1
_COUPLING = {"pressure_tensor": COUPLING_PRESSURE_TENSOR, "forcing": COUPLING_FORCING,
             "guo": COUPLING_FORCING, COUPLING_PRESSURE_TENSOR: COUPLING_PRESSURE_TENSOR,
             COUPLING_FORCING: COUPLING_FORCING}
_PREC = {"fp64": FP64, "fp32": FP32, "fp16": FP16_OFFSET, "bf16": BF16_OFFSET,
         FP64: FP64, FP32: FP32, FP16_OFFSET: FP16_OFFSET, BF16_OFFSET: BF16_OFFSET}
_KIND = {"auto": KERNEL_AUTO, "fused": KERNEL_FUSED, "split": KERNEL_SPLIT,
         KERNEL_AUTO: KERNEL_AUTO, KERNEL_FUSED: KERNEL_FUSED, KERNEL_SPLIT: KERNEL_SPLIT}
STATUS = ["TLBM_OK", "TLBM_ERR_ARG", "TLBM_ERR_PARAM", "TLBM_ERR_CUDA", "TLBM_ERR_OOM",
          "TLBM_ERR_NONFINITE", "TLBM_ERR_TIMEOUT", "TLBM_ERR_UNSUPPORTED"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return os.path.join(_HERE, "libtlbm.so")


class TLBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_H = ctypes.c_void_p  # opaque tlbm*


def _declare(lib):
    i, i64, sz, d = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
    sig = {
        "tlbm_create": (i, [ctypes.POINTER(_H), i, i, i, i, _dp, d, d, d, d, _dp,
                            ctypes.POINTER(ctypes.c_uint8), i, _vp]),
        "tlbm_destroy": (None, [_H]),
        "tlbm_set_gamma": (i, [_H, d, d]),
        "tlbm_set_kernel": (i, [_H, i]),
        "tlbm_get_kernel": (i, [_H]),
        "tlbm_set_tile": (i, [_H, i, i]),
        "tlbm_set_coupling": (i, [_H, i]),
        "tlbm_get_coupling": (i, [_H]),
        "tlbm_set_bounds_check": (i, [_H, i]),
        "tlbm_bounds_check_word": (i, [_H, ctypes.POINTER(ctypes.c_uint64)]),
        "tlbm_init_fields": (i, [_H, _dp, _dp, _dp, _dp, _dp, _dp]),
        "tlbm_step": (i, [_H, i64]),
        "tlbm_steps_done": (i64, [_H]),
        "tlbm_set_timing": (i, [_H, i]),
        "tlbm_kernel_time": (i, [_H, _dp, ctypes.POINTER(ctypes.c_int64)]),
        "tlbm_fields": (i, [_H, _dp, _dp, _dp, _dp, _dp]),
        "tlbm_mass": (i, [_H, _dp]),
        "tlbm_step_mass": (i, [_H, _dp]),
        "tlbm_get_populations_box": (i, [_H, i, i, i, i, i, i, _dp]),
        "tlbm_get_populations": (i, [_H, _dp]),
        "tlbm_set_populations": (i, [_H, _dp]),
        "tlbm_state_bytes": (sz, [_H]),
        "tlbm_get_state": (i, [_H, _vp, sz]),
        "tlbm_set_state": (i, [_H, _vp, sz]),
        "tlbm_launches_per_step": (i, [_H]),
        "tlbm_last_error": (ctypes.c_char_p, [_H]),
        "tlbm_status_string": (ctypes.c_char_p, [i]),
        "tlbm_batch_create": (i, [ctypes.POINTER(_H), ctypes.POINTER(_H), i]),
        "tlbm_batch_step": (i, [_H, i64]),
        "tlbm_batch_set_tile": (i, [_H, i, i]),
        "tlbm_batch_autotune": (i, [_H, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "tlbm_batch_set_graph": (i, [_H, i]),
        "tlbm_batch_blocks": (i64, [_H]),
        "tlbm_batch_set_timing": (i, [_H, i]),
        "tlbm_batch_kernel_time": (i, [_H, _dp, ctypes.POINTER(ctypes.c_int64)]),
        "tlbm_batch_last_error": (ctypes.c_char_p, [_H]),
        "tlbm_batch_destroy": (None, [_H]),
        "tlbm_contact_angles": (i, [_dp, d, _dp, _dp]),
        "tlbm_adjoint_c3_misfit": (i, [_H, i64, i, _dp, _dp, _dp, _dp, _dp]),
        "tlbm_wetting_from_angles": (i, [_dp, d, d, d, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load_library(build_if_missing: bool = True):
    """Load libtlbm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if build_if_missing:
                from . import _build
                _build.build()
            if not os.path.exists(path):
                raise TLBMError(7, f"{path} is missing: build it with paper_1511_02155_gb300._build")
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def _arr(a, n=None):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a, a.ctypes.data_as(_dp)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # torch missing or unusable: the default stream is used
        pass
    return None


class TernaryLB:
    """One ternary LB simulation on the current CUDA device.

    Arguments mirror ``tlbm_create``: lattice 9 (D2Q9, nz = 1) or 19 (D3Q19),
    sizes, kappa_1..3, alpha, tau_f, mobilities M_phi and M_psi, wetting
    parameters h_1..3, an optional solid mask (any array of nx*ny*nz values,
    nonzero = solid, indexed x fastest) and the storage precision
    ('fp64', 'fp32', 'fp16', 'bf16').
    """

    def __init__(self, lattice, nx, ny, nz=1, kappa=(0.01, 0.02, 0.03), alpha=1.0, tau_f=1.0,
                 M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), solid=None, precision="fp32",
                 stream="current"):
        self._lib = load_library()
        self.Q = int(lattice)
        self.shape = (int(nx), int(ny), int(nz))
        self.N = int(nx) * int(ny) * int(nz)
        self._h = _H()
        k = (ctypes.c_double * 3)(*[float(v) for v in kappa])
        hh = (ctypes.c_double * 3)(*[float(v) for v in (h if h is not None else (0, 0, 0))])
        self.solid = None
        sp = None
        if solid is not None:
            self.solid = np.ascontiguousarray(np.asarray(solid).reshape(-1) != 0, dtype=np.uint8)
            if self.solid.size != self.N:
                raise ValueError("solid mask must have nx*ny*nz entries")
            sp = self.solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        st = _default_stream() if stream == "current" else stream
        rc = self._lib.tlbm_create(ctypes.byref(self._h), self.Q, *self.shape, k, float(alpha),
                                   float(tau_f), float(M_phi), float(M_psi), hh, sp,
                                   _PREC[precision], st)
        if rc != 0:
            raise TLBMError(rc, self._lib.tlbm_last_error(None).decode())
        self.precision = _PREC[precision]

    # -------------------------------------------------------------- helpers
    def _check(self, rc):
        if rc != 0:
            raise TLBMError(rc, self._lib.tlbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.tlbm_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- settings
    def set_gamma(self, gamma_phi, gamma_psi):
        self._check(self._lib.tlbm_set_gamma(self._h, float(gamma_phi), float(gamma_psi)))

    def set_kernel(self, kind):
        self._check(self._lib.tlbm_set_kernel(self._h, _KIND[kind]))

    @property
    def kernel(self):
        return {KERNEL_FUSED: "fused", KERNEL_SPLIT: "split"}[self._lib.tlbm_get_kernel(self._h)]

    def set_tile(self, variant=0, chunk=0):
        self._check(self._lib.tlbm_set_tile(self._h, int(variant), int(chunk)))

    @property
    def launches_per_step(self):
        return int(self._lib.tlbm_launches_per_step(self._h))

    def set_coupling(self, coupling):
        """'pressure_tensor' (the default) or 'forcing' (Guo body force; periodic
        lattices, three kernels per step).  Call init_fields afterwards."""
        self._check(self._lib.tlbm_set_coupling(self._h, _COUPLING[coupling]))

    @property
    def coupling(self):
        return {COUPLING_PRESSURE_TENSOR: "pressure_tensor",
                COUPLING_FORCING: "forcing"}[self._lib.tlbm_get_coupling(self._h)]

    def set_bounds_check(self, on=True):
        """Run the bounds-checked variants of the fused step (FP32 storage)."""
        self._check(self._lib.tlbm_set_bounds_check(self._h, 1 if on else 0))

    def bounds_check_word(self):
        """First bounds violation since the last call (code << 56 | offset), 0 if none."""
        w = ctypes.c_uint64(0)
        self._check(self._lib.tlbm_bounds_check_word(self._h, ctypes.byref(w)))
        return int(w.value)

    def set_timing(self, on=True):
        """Time the main kernel(s) of each step with CUDA events (synchronous steps)."""
        self._check(self._lib.tlbm_set_timing(self._h, 1 if on else 0))

    def kernel_time(self):
        """(total main-kernel milliseconds, steps timed) since timing was set."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.tlbm_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    @property
    def steps_done(self):
        return int(self._lib.tlbm_steps_done(self._h))

    # ---------------------------------------------------------------- state
    def init_fields(self, rho, phi, psi, u=None):
        """Populations at equilibrium with fields rho, phi, psi (and velocity u)."""
        a = [_arr(x, self.N)[0] for x in (rho, phi, psi)]
        us = [None, None, None]
        if u is not None:
            for k in range(len(u)):
                us[k] = _arr(u[k], self.N)[0]
        ptr = lambda x: None if x is None else x.ctypes.data_as(_dp)  # noqa: E731
        self._check(self._lib.tlbm_init_fields(self._h, *[ptr(x) for x in a], *[ptr(x) for x in us]))

    def init_from_host_ptrs(self, rho_ptr, phi_ptr, psi_ptr):
        """init_fields from raw host pointers (e.g. pinned torch tensors)."""
        self._check(self._lib.tlbm_init_fields(self._h, ctypes.cast(rho_ptr, _dp),
                                               ctypes.cast(phi_ptr, _dp),
                                               ctypes.cast(psi_ptr, _dp), None, None, None))

    def step(self, n=1):
        self._check(self._lib.tlbm_step(self._h, int(n)))

    def fields(self):
        """dict of C1, C2, C3, rho (N,) and u (3, N) as float64 numpy arrays."""
        out = {k: np.zeros(self.N) for k in ("C1", "C2", "C3", "rho")}
        out["u"] = np.zeros((3, self.N))
        self._check(self._lib.tlbm_fields(self._h, *[out[k].ctypes.data_as(_dp)
                                                     for k in ("C1", "C2", "C3", "rho", "u")]))
        return out

    def fields_into(self, C1_ptr, C2_ptr, C3_ptr):
        """tlbm_fields into raw host pointers (e.g. pinned torch tensors); rho, u skipped."""
        self._check(self._lib.tlbm_fields(self._h, ctypes.cast(C1_ptr, _dp), ctypes.cast(C2_ptr, _dp),
                                          ctypes.cast(C3_ptr, _dp), None, None))

    def mass(self):
        out = np.zeros(3)
        self._check(self._lib.tlbm_mass(self._h, out.ctypes.data_as(_dp)))
        return out

    def step_mass(self):
        out = np.zeros(3)
        self._check(self._lib.tlbm_step_mass(self._h, out.ctypes.data_as(_dp)))
        return out

    def get_populations(self):
        out = np.zeros((3, self.Q, self.N))
        self._check(self._lib.tlbm_get_populations(self._h, out.ctypes.data_as(_dp)))
        return out

    def get_populations_box(self, x0, y0, z0, bx, by, bz):
        out = np.zeros((3, self.Q, bz, by, bx))
        self._check(self._lib.tlbm_get_populations_box(self._h, int(x0), int(y0), int(z0), int(bx),
                                                       int(by), int(bz), out.ctypes.data_as(_dp)))
        return out

    def set_populations(self, pops):
        a = np.ascontiguousarray(pops, dtype=np.float64).reshape(-1)
        if a.size != 3 * self.Q * self.N:
            raise ValueError("populations must have 3*Q*N values")
        self._check(self._lib.tlbm_set_populations(self._h, a.ctypes.data_as(_dp)))

    @property
    def state_bytes(self):
        return int(self._lib.tlbm_state_bytes(self._h))

    def get_state(self):
        buf = np.zeros(self.state_bytes, dtype=np.uint8)
        self._check(self._lib.tlbm_get_state(self._h, buf.ctypes.data_as(_vp), buf.size))
        return buf

    def adjoint_c3_misfit(self, nsteps, checkpoint_every, target, want_fields=True):
        """Loss sum_fluid (C_3(T) - target)^2 after nsteps from the initial equilibrium
        and its gradient: (loss, dL/dkappa[3], dL/dh[3], dL/d(rho, phi, psi)[3][N] or
        None).  Runs forward nsteps (the engine ends there) and the adjoint back."""
        tg, tp = _arr(target, self.N)
        loss = ctypes.c_double()
        dk = np.zeros(3)
        dh = np.zeros(3)
        df = np.zeros(3 * self.N) if want_fields else None
        self._check(self._lib.tlbm_adjoint_c3_misfit(
            self._h, int(nsteps), int(checkpoint_every), tp, ctypes.byref(loss), dk.ctypes.data_as(_dp),
            dh.ctypes.data_as(_dp), df.ctypes.data_as(_dp) if df is not None else None))
        return loss.value, dk, dh, (df.reshape(3, self.N) if df is not None else None)

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self._lib.tlbm_set_state(self._h, buf.ctypes.data_as(_vp), buf.size))


def contact_angles(kappa, alpha, h):
    """(theta_12, theta_23, theta_31) in degrees for wetting parameters h (host code)."""
    lib = load_library()
    k, kp = _arr(kappa, 3)
    hh, hp = _arr(h, 3)
    out = np.zeros(3)
    rc = lib.tlbm_contact_angles(kp, float(alpha), hp, out.ctypes.data_as(_dp))
    if rc != 0:
        raise TLBMError(rc, "no contact angles for these parameters")
    return tuple(float(v) for v in out)


def wetting_from_angles(kappa, alpha, theta12, theta13):
    """Wetting parameters (h_1, h_2, h_3) giving theta_12 and theta_13 (through fluid 1,
    degrees) with the gauge sum h_m/kappa_m = 0 (host code)."""
    lib = load_library()
    k, kp = _arr(kappa, 3)
    out = np.zeros(3)
    rc = lib.tlbm_wetting_from_angles(kp, float(alpha), float(theta12), float(theta13), out.ctypes.data_as(_dp))
    if rc != 0:
        raise TLBMError(rc, f"no admissible wetting parameters for theta_12={theta12}, theta_13={theta13}")
    return tuple(float(v) for v in out)


class TernaryBatch:
    """Many TernaryLB engines advanced together: one kernel launch per step.

    Members must share lattice, precision, device and stream, and all have (or
    all lack) solid nodes.  They stay usable on their own (fields, mass, ...);
    stepping one alone breaks the batch's common parity until it has taken an
    even number of lone steps.  The engines must outlive the batch.
    """

    def __init__(self, members):
        self._lib = load_library()
        self.members = list(members)
        hs = (_H * len(self.members))(*[m._h.value for m in self.members])
        self._h = _H()
        rc = self._lib.tlbm_batch_create(ctypes.byref(self._h), hs, len(self.members))
        if rc != 0:
            raise TLBMError(rc, self._lib.tlbm_batch_last_error(None).decode())

    def _check(self, rc):
        if rc != 0:
            raise TLBMError(rc, self._lib.tlbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.tlbm_batch_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n=1):
        self._check(self._lib.tlbm_batch_step(self._h, int(n)))

    def set_tile(self, variant=0, chunk=0):
        self._check(self._lib.tlbm_batch_set_tile(self._h, int(variant), int(chunk)))

    def set_graph(self, on=True):
        self._check(self._lib.tlbm_batch_set_graph(self._h, 1 if on else 0))

    def autotune(self, trial_steps=10):
        """Pick the fastest tile; every member advances by the trial steps."""
        v, c = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.tlbm_batch_autotune(self._h, int(trial_steps), ctypes.byref(v), ctypes.byref(c)))
        return v.value, c.value

    @property
    def blocks(self):
        return int(self._lib.tlbm_batch_blocks(self._h))

    def set_timing(self, on=True):
        self._check(self._lib.tlbm_batch_set_timing(self._h, 1 if on else 0))

    def kernel_time(self):
        """(total main-kernel ms, timed steps) since timing was turned on."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.tlbm_batch_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value
