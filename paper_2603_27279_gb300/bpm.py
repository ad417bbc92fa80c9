"""Python binding of the C ABI in include/bpm.h (argument marshalling only).

Every number is computed by the CUDA library libbpm_gb300.so; there is no
CPU fallback: importing the binding without the built library raises.

Functions keep the C names (``bpm_create``, ``bpm_forces``, ``bpm_step``,
``bpm_energy``, ...).  ``Simulation`` wraps a handle for a
``workloads.RodSystem``; array arguments may be numpy arrays (host) or
contiguous float64 CUDA tensors (device pointers are passed straight through).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbpm_gb300.so")

BPM_OK = 0
BPM_ERR_ARG = -1
BPM_ERR_CUDA = -2
BPM_ERR_NONFINITE = -3
BPM_ERR_TIMEOUT = -4
BPM_ERR_SINGULAR = -5
BPM_ERR_CAPACITY = -6
BPM_FP64 = 0
BPM_MIXED = 1
BPM_FF = 2
BPM_DIPOLE_OFF = 0
BPM_DIPOLE_GLOBAL = 1
BPM_DIPOLE_PER_ROD = 2
BPM_PLAN_AUTO = 0
BPM_PLAN_ORDERED = 1
BPM_PLAN_SYMMETRIC = 2

EXPORTED = ["bpm_create", "bpm_destroy", "bpm_forces", "bpm_step", "bpm_energy", "bpm_get_state",
            "bpm_set_state", "bpm_set_field", "bpm_set_dipoles", "bpm_set_timing", "bpm_get_timing",
            "bpm_last_error", "bpm_version", "bpm_dipole_forces_noalloc", "bpm_set_dipole_plan",
            "bpm_get_dipole_plan", "bpm_set_overlap", "bpm_get_overlap", "bpm_adjoint_begin",
            "bpm_adjoint_end", "bpm_lbm_fields", "bpm_create_device", "bpm_set_forces", "bpm_get_forces",
            "bpm_measure_pipes"]

_dp = C.POINTER(C.c_double)


class bpm_contact(C.Structure):
    _fields_ = [
        ("E", C.c_double), ("nu", C.c_double), ("mu", C.c_double), ("gamma_n", C.c_double),
        ("gamma_t", C.c_double), ("exclude", C.c_int32), ("max_contacts", C.c_int32),
    ]


class bpm_lbm(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_sub", C.c_int32), ("tau", C.c_double),
        ("body_force", C.c_double * 3), ("rho0", _dp), ("u0", _dp), ("coupled", C.POINTER(C.c_uint8)),
    ]


class bpm_device_state(C.Structure):
    _fields_ = [("x", _dp), ("q", _dp), ("v", _dp), ("omega", _dp), ("f", _dp), ("tau", _dp)]


class bpm_desc(C.Structure):
    _fields_ = [
        ("n_particles", C.c_int64), ("n_rods", C.c_int64), ("rod_offset", C.POINTER(C.c_int64)),
        ("x", _dp), ("q", _dp), ("v", _dp), ("omega", _dp), ("mass", _dp), ("radius", _dp),
        ("m_body", _dp), ("clamped", C.POINTER(C.c_uint8)), ("x_rest", _dp), ("q_rest", _dp),
        ("E", _dp), ("nu", _dp), ("d", _dp),
        ("B", C.c_double * 3), ("B_rod", _dp), ("Brot_amp", C.c_double), ("Brot_omega", C.c_double),
        ("Brot_e1", C.c_double * 3), ("Brot_e2", C.c_double * 3), ("gradB", C.c_double * 9),
        ("gradB_x0", C.c_double * 3), ("mu0_over_4pi", C.c_double), ("dipole_mode", C.c_int32),
        ("precision", C.c_int32), ("damping", C.c_double), ("dt", C.c_double), ("t0", C.c_double),
        ("stream", C.c_void_p), ("bond_damping", _dp), ("contact", C.POINTER(bpm_contact)),
        ("lbm", C.POINTER(bpm_lbm)),
    ]


class BpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bpm error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Loads libbpm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "bpm_create": ([C.POINTER(bpm_desc), C.POINTER(vp)], C.c_int),
        "bpm_destroy": ([vp], None),
        "bpm_forces": ([vp, vp, vp], C.c_int),
        "bpm_step": ([vp, C.c_int32], C.c_int),
        "bpm_energy": ([vp, _dp], C.c_int),
        "bpm_get_state": ([vp, vp, vp, vp, vp, _dp], C.c_int),
        "bpm_set_state": ([vp, vp, vp, vp, vp, C.c_double], C.c_int),
        "bpm_set_field": ([vp, vp, vp], C.c_int),
        "bpm_set_dipoles": ([vp, vp], C.c_int),
        "bpm_set_timing": ([vp, C.c_int32], C.c_int),
        "bpm_get_timing": ([vp, _dp], C.c_int),
        "bpm_last_error": ([vp], C.c_char_p),
        "bpm_version": ([], C.c_char_p),
        "bpm_dipole_forces_noalloc": ([C.c_int64, vp, vp, C.c_double, vp, vp, vp], C.c_int),
        "bpm_set_dipole_plan": ([vp, C.c_int32, C.c_int32], C.c_int),
        "bpm_get_dipole_plan": ([vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
        "bpm_set_overlap": ([vp, C.c_int32], C.c_int),
        "bpm_get_overlap": ([vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
        "bpm_adjoint_begin": ([vp, C.c_int32, C.c_int32], C.c_int),
        "bpm_adjoint_end": ([vp, vp, vp, _dp], C.c_int),
        "bpm_lbm_fields": ([vp, vp, vp], C.c_int),
        "bpm_create_device": ([C.POINTER(bpm_desc), C.POINTER(bpm_device_state), C.POINTER(vp)], C.c_int),
        "bpm_set_forces": ([vp, vp, vp], C.c_int),
        "bpm_get_forces": ([vp, vp, vp], C.c_int),
        "bpm_measure_pipes": ([_dp], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


# ----------------------------------------------------------------------------
# thin wrappers with the C names
# ----------------------------------------------------------------------------

def _check(rc: int, handle=None):
    if rc != BPM_OK:
        msg = load().bpm_last_error(handle)
        raise BpmError(rc, msg.decode() if msg else "")


def bpm_create(desc: bpm_desc):
    h = C.c_void_p()
    _check(load().bpm_create(C.byref(desc), C.byref(h)), None)
    return h


def bpm_create_device(desc: bpm_desc, state: bpm_device_state):
    h = C.c_void_p()
    _check(load().bpm_create_device(C.byref(desc), C.byref(state), C.byref(h)), None)
    return h


def bpm_set_forces(h, f, tau):
    _check(load().bpm_set_forces(h, _ptr(f), _ptr(tau)), h)


def bpm_get_forces(h, f=None, tau=None):
    _check(load().bpm_get_forces(h, _ptr(f, True), _ptr(tau, True)), h)


def bpm_measure_pipes() -> dict:
    """Lane operations per SM per clock, per second, the SM clock (MHz) and the
    kernel time (ms) of the FP64 fma, FP32 fma, packed FP32 fma, FP32 rsqrt
    and FP64 add probes on the current device."""
    out = np.zeros(20)
    _check(load().bpm_measure_pipes(out.ctypes.data_as(_dp)), None)
    names = ("fp64_fma", "fp32_fma", "fp32x2_fma", "mufu_rsqrt", "fp64_add")
    return {nm: {"per_sm_per_clk": float(out[4 * k]), "per_s": float(out[4 * k + 1]),
                 "sm_mhz": float(out[4 * k + 2]), "ms": float(out[4 * k + 3])} for k, nm in enumerate(names)}


def bpm_destroy(h):
    load().bpm_destroy(h)


def bpm_forces(h, f, tau):
    _check(load().bpm_forces(h, _ptr(f, True), _ptr(tau, True)), h)


def bpm_step(h, n: int):
    _check(load().bpm_step(h, int(n)), h)


def bpm_energy(h) -> np.ndarray:
    out = np.zeros(5)
    _check(load().bpm_energy(h, out.ctypes.data_as(_dp)), h)
    return out


def bpm_get_state(h, x=None, q=None, v=None, omega=None) -> float:
    t = C.c_double()
    _check(load().bpm_get_state(h, _ptr(x, True), _ptr(q, True), _ptr(v, True), _ptr(omega, True),
                                C.byref(t)), h)
    return t.value


def bpm_set_state(h, x=None, q=None, v=None, omega=None, t: float = 0.0):
    _check(load().bpm_set_state(h, _ptr(x), _ptr(q), _ptr(v), _ptr(omega), float(t)), h)


def bpm_set_field(h, B=None, B_rod=None):
    _check(load().bpm_set_field(h, _ptr(B), _ptr(B_rod)), h)


def bpm_set_dipoles(h, m_body):
    _check(load().bpm_set_dipoles(h, _ptr(m_body)), h)


def bpm_set_dipole_plan(h, kind: int, param: int = 0):
    _check(load().bpm_set_dipole_plan(h, int(kind), int(param)), h)


def bpm_get_dipole_plan(h):
    k, p = C.c_int32(), C.c_int32()
    _check(load().bpm_get_dipole_plan(h, C.byref(k), C.byref(p)), h)
    return k.value, p.value


def bpm_set_overlap(h, mode: int):
    _check(load().bpm_set_overlap(h, int(mode)), h)


def bpm_get_overlap(h):
    """(on, dipole_blocks, bond_blocks) of the form in use."""
    on, db, bb = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().bpm_get_overlap(h, C.byref(on), C.byref(db), C.byref(bb)), h)
    return on.value, db.value, bb.value


def bpm_lbm_fields(h, nodes: int):
    """(rho [nodes], u [nodes, 3]) of the fluid's current state."""
    rho = np.zeros(nodes)
    u = np.zeros((nodes, 3))
    _check(load().bpm_lbm_fields(h, rho.ctypes.data_as(_dp), u.ctypes.data_as(_dp)), h)
    return rho, u


def bpm_adjoint_begin(h, n_steps: int, checkpoint_every: int):
    _check(load().bpm_adjoint_begin(h, int(n_steps), int(checkpoint_every)), h)


def bpm_adjoint_end(h, dL_dx, grad_m_body=None):
    gB = np.zeros(3)
    _check(load().bpm_adjoint_end(h, _ptr(dL_dx), _ptr(grad_m_body, True), gB.ctypes.data_as(_dp)), h)
    return gB


def bpm_set_timing(h, enable: bool):
    _check(load().bpm_set_timing(h, 1 if enable else 0), h)


def bpm_get_timing(h) -> np.ndarray:
    out = np.zeros(15)
    _check(load().bpm_get_timing(h, out.ctypes.data_as(_dp)), h)
    return out


def bpm_dipole_forces_noalloc(n: int, x, m, mu0_over_4pi: float, f, tau, stream=None):
    """Allocation-free all-pairs dipole forces: x, m in, f, tau out, each a
    contiguous float64 CUDA tensor of the current device with at least 3n
    elements (AoS [n,3])."""
    n = int(n)
    for name, a in (("x", x), ("m", m), ("f", f), ("tau", tau)):
        if not hasattr(a, "data_ptr") or not getattr(a, "is_cuda", False):
            raise TypeError(f"{name}: bpm_dipole_forces_noalloc takes CUDA tensors")
        import torch
        if a.device.index != torch.cuda.current_device():
            raise TypeError(f"{name}: tensor on cuda:{a.device.index}, current device is "
                            f"cuda:{torch.cuda.current_device()}")
        if a.numel() < 3 * n:
            raise ValueError(f"{name}: {a.numel()} elements, {3 * n} needed")
    _check(load().bpm_dipole_forces_noalloc(n, _ptr(x), _ptr(m), float(mu0_over_4pi), _ptr(f, True),
                                            _ptr(tau, True), stream), None)


def bpm_version() -> str:
    return load().bpm_version().decode()


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------

def _ptr(a, writable: bool = False):
    """Host numpy array or CUDA tensor -> raw pointer (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous():
            raise TypeError("tensors crossing the ABI must be contiguous float64")
        return C.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("arrays crossing the ABI must be C-contiguous float64 numpy arrays")
    if writable and not a.flags.writeable:
        raise TypeError("output array is read-only")
    return C.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_desc(sysm: W.RodSystem, stream: Optional[int] = None, precision: Optional[int] = None):
    """bpm_desc for a RodSystem; returns (desc, keep-alive list)."""
    keep = []

    def p(a, dtype=np.float64, ctype=C.c_double):
        if a is None:
            return None
        arr = np.ascontiguousarray(a, dtype=dtype)
        keep.append(arr)
        return arr.ctypes.data_as(C.POINTER(ctype))

    d = bpm_desc()
    d.n_particles = sysm.n
    d.n_rods = sysm.n_rods
    d.rod_offset = p(sysm.rod_offset, np.int64, C.c_int64)
    d.x = p(sysm.x)
    d.q = p(sysm.q)
    d.v = p(sysm.v)
    d.omega = p(sysm.omega)
    d.mass = p(sysm.mass)
    d.radius = p(sysm.radius)
    d.m_body = p(sysm.m_body)
    d.clamped = p(sysm.clamped, np.uint8, C.c_uint8)
    d.x_rest = p(sysm.x_rest)
    d.q_rest = p(sysm.q_rest)
    d.E = p(sysm.E)
    d.nu = p(sysm.nu)
    d.d = p(sysm.d)
    d.B[:] = [float(v) for v in sysm.B]
    d.B_rod = p(sysm.B_rod) if sysm.B_rod is not None else None
    d.Brot_amp = float(sysm.Brot_amp)
    d.Brot_omega = float(sysm.Brot_omega)
    d.Brot_e1[:] = [float(v) for v in sysm.Brot_e1]
    d.Brot_e2[:] = [float(v) for v in sysm.Brot_e2]
    d.gradB[:] = [float(v) for v in np.asarray(sysm.gradB).ravel()]
    d.gradB_x0[:] = [float(v) for v in sysm.gradB_x0]
    d.mu0_over_4pi = float(sysm.mu0_over_4pi)
    d.dipole_mode = int(sysm.dipole_mode)
    d.precision = int(sysm.precision if precision is None else precision)
    d.damping = float(sysm.damping)
    d.dt = float(sysm.dt)
    d.t0 = float(sysm.t0)
    d.stream = stream
    d.bond_damping = p(sysm.bond_damping) if sysm.bond_damping is not None else None
    if sysm.contact is not None:
        cp = sysm.contact
        cs = bpm_contact(E=float(cp.E), nu=float(cp.nu), mu=float(cp.mu), gamma_n=float(cp.gamma_n),
                         gamma_t=float(cp.gamma_t), exclude=int(cp.exclude), max_contacts=int(cp.cap))
        keep.append(cs)
        d.contact = C.pointer(cs)
    if sysm.lbm is not None:
        lp = sysm.lbm
        ls = bpm_lbm(nx=int(lp.nx), ny=int(lp.ny), nz=int(lp.nz), n_sub=int(lp.n_sub), tau=float(lp.tau))
        ls.body_force[:] = [float(v) for v in lp.body_force]
        ls.rho0 = p(lp.rho0) if lp.rho0 is not None else None
        ls.u0 = p(lp.u0) if lp.u0 is not None else None
        ls.coupled = p(lp.coupled, np.uint8, C.c_uint8) if lp.coupled is not None else None
        keep.append(ls)
        d.lbm = C.pointer(ls)
    return d, keep


class Simulation:
    """One bpm handle for a RodSystem (host numpy in and out by default).

    With ``device_state`` (a dict of contiguous float64 CUDA tensors "x",
    "q", "v", "omega", "f", "tau" of shapes (3, N), (4, N), (3, N), (3, N),
    (3, N), (3, N), holding the initial state), the handle is made by
    bpm_create_device and works on those tensors in place; the system's own
    x, q, v, omega are then not used and its rest orientations must be the
    identity."""

    def __init__(self, sysm: W.RodSystem, stream: Optional[int] = None, precision: Optional[int] = None,
                 device_state: Optional[dict] = None):
        load()
        self.n = sysm.n
        self.nodes = sysm.lbm.nodes if sysm.lbm is not None else 0
        desc, keep = make_desc(sysm, stream, precision)
        if device_state is None:
            self.h = bpm_create(desc)
        else:
            shapes = {"x": 3, "q": 4, "v": 3, "omega": 3, "f": 3, "tau": 3}
            st = bpm_device_state()
            for k, c in shapes.items():
                t = device_state[k]
                if not getattr(t, "is_cuda", False) or tuple(t.shape) != (c, sysm.n):
                    raise TypeError(f"device_state[{k!r}] must be a CUDA tensor of shape ({c}, {sysm.n})")
                setattr(st, k, C.cast(_ptr(t), _dp))
            desc.x = desc.q = desc.v = desc.omega = None
            if sysm.q_rest is not None and not np.allclose(sysm.q_rest, [1.0, 0.0, 0.0, 0.0], rtol=0, atol=0):
                raise ValueError("a device-state handle has identity rest orientations")
            desc.q_rest = None
            self.device_state = device_state  # kept alive with the handle
            self.h = bpm_create_device(desc, st)
        del keep

    def close(self):
        if getattr(self, "h", None):
            bpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def forces(self, f=None, tau=None):
        if f is None and tau is None:
            f = np.zeros((self.n, 3))
            tau = np.zeros((self.n, 3))
        bpm_forces(self.h, f, tau)
        return f, tau

    def step(self, n: int):
        bpm_step(self.h, n)

    def energy(self) -> np.ndarray:
        return bpm_energy(self.h)

    def get_state(self):
        x = np.zeros((self.n, 3))
        q = np.zeros((self.n, 4))
        v = np.zeros((self.n, 3))
        w = np.zeros((self.n, 3))
        t = bpm_get_state(self.h, x, q, v, w)
        return x, q, v, w, t

    def set_state(self, x=None, q=None, v=None, omega=None, t: float = 0.0):
        bpm_set_state(self.h, *(None if a is None else (a if hasattr(a, "data_ptr") else _f64(a))
                                for a in (x, q, v, omega)), t=t)

    def set_forces(self, f, tau):
        """Declares f, tau ([N,3], host or device) the forces of the current
        state (bpm_set_forces)."""
        bpm_set_forces(self.h, f if hasattr(f, "data_ptr") else _f64(f), tau if hasattr(tau, "data_ptr") else _f64(tau))

    def get_forces(self, f=None, tau=None):
        """The stored forces of the current state, without evaluating them."""
        if f is None and tau is None:
            f = np.zeros((self.n, 3))
            tau = np.zeros((self.n, 3))
        bpm_get_forces(self.h, f, tau)
        return f, tau

    def set_field(self, B=None, B_rod=None):
        bpm_set_field(self.h, None if B is None else _f64(B), None if B_rod is None else _f64(B_rod))

    def set_dipoles(self, m_body):
        bpm_set_dipoles(self.h, m_body if hasattr(m_body, "data_ptr") else _f64(m_body))

    def set_dipole_plan(self, kind: int, param: int = 0):
        bpm_set_dipole_plan(self.h, kind, param)

    def set_overlap(self, mode: int):
        """-1: timed by the autotuner (default), 0: sequential, 1: bond and
        dipole kernels at the same time."""
        bpm_set_overlap(self.h, mode)

    def overlap(self):
        """(on, dipole_blocks, bond_blocks) after the first force evaluation."""
        return bpm_get_overlap(self.h)

    def adjoint_begin(self, n_steps: int, checkpoint_every: int):
        bpm_adjoint_begin(self.h, n_steps, checkpoint_every)

    def adjoint_end(self, dL_dx):
        """(dL/dm~ [N,3], dL/dB [3]) for the trajectory of adjoint_begin."""
        g = np.zeros((self.n, 3))
        gB = bpm_adjoint_end(self.h, dL_dx if hasattr(dL_dx, "data_ptr") else _f64(dL_dx), g)
        return g, gB

    def dipole_plan(self):
        return bpm_get_dipole_plan(self.h)

    def set_timing(self, enable: bool):
        bpm_set_timing(self.h, enable)

    def timing(self) -> dict:
        t = bpm_get_timing(self.h)
        names = ("bond", "dipole", "integrate", "contact", "lbm")
        return {names[k]: {"launches": t[3 * k], "ms": t[3 * k + 1], "units": t[3 * k + 2]}
                for k in range(5) if k < 3 or t[3 * k] > 0}

    def lbm_fields(self):
        """(rho [nodes], u [nodes, 3]) of the fluid's current state."""
        return bpm_lbm_fields(self.h, self.nodes)
