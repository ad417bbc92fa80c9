"""ctypes front end of the C oracle (bpm_oracle.c).

TEST INFRASTRUCTURE ONLY.  Marshals a ``RodSystem`` into the oracle's
``orc_system`` struct; every number is computed in bpm_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # a prebuilt oracle may be substituted (used to check that the pins
        # catch deliberately planted mistakes)
        path = os.environ.get("BPM_ORACLE_LIB") or _build.build()
        _lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        _lib.orc_bond.argtypes = [dp, dp, dp, dp, dp, dp, C.c_int, dp, dp, dp, dp, dp, dp]
        _lib.orc_bond.restype = None
        _lib.orc_bond_damped.argtypes = [dp, dp, dp, dp, dp, dp, dp, dp, dp, C.c_void_p, C.c_double,
                                         dp, dp, dp, dp, dp, dp]
        _lib.orc_bond_damped.restype = None
        _lib.orc_contact_pair.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, C.c_double, C.c_double,
                                          C.c_void_p, C.c_double, dp, dp, dp, dp]
        _lib.orc_contact_pair.restype = C.c_int
        _lib.orc_contact_sample.argtypes = [C.c_void_p, dp, dp, dp, C.POINTER(C.c_int64), C.c_int64, dp, dp]
        _lib.orc_contact_sample.restype = C.c_int
        _lib.orc_lbm_lattice.argtypes = [C.POINTER(C.c_int), dp]
        _lib.orc_ibm_phi.argtypes = [C.c_double]
        _lib.orc_ibm_phi.restype = C.c_double
        _lib.orc_lbm_init.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_lbm_macro.argtypes = [C.c_void_p, C.c_void_p, dp]
        _lib.orc_lbm_step.argtypes = [C.c_void_p]
        _lib.orc_lbm_step.restype = C.c_int
        _lib.orc_lbm_interp.argtypes = [C.c_void_p, dp, C.c_int64, dp]
        _lib.orc_init_bonds.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib.orc_init_bonds.restype = C.c_int
        _lib.orc_forces.argtypes = [C.c_void_p, dp, dp, dp, dp, C.c_double, dp, dp, C.c_void_p, C.c_void_p]
        _lib.orc_forces.restype = C.c_int
        _lib.orc_dipole_sample.argtypes = [C.c_void_p, dp, dp, C.POINTER(C.c_int64), C.c_int64, dp, dp, C.c_void_p]
        _lib.orc_dipole_sample.restype = C.c_int
        _lib.orc_term_scales.argtypes = [C.c_void_p, dp, dp, dp, dp, C.c_double, C.POINTER(C.c_int64),
                                         C.c_int64, dp, dp]
        _lib.orc_term_scales.restype = C.c_int
        _lib.orc_run.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, C.c_int, dp, dp, C.c_int]
        _lib.orc_run.restype = C.c_int
        _lib.orc_quat_mul.argtypes = [dp, dp, dp]
        _lib.orc_rotate.argtypes = [dp, dp, dp]
        _lib.orc_richardson.argtypes = [dp, dp, C.c_double, dp]
        _lib.orc_align_z.argtypes = [dp, C.c_int, dp]
    return _lib


class _OrcContact(C.Structure):
    _fields_ = [
        ("E", C.c_double), ("nu", C.c_double), ("mu", C.c_double), ("gamma_n", C.c_double),
        ("gamma_t", C.c_double), ("exclude", C.c_int), ("cap", C.c_int), ("level", C.c_int),
        ("valid", C.c_int * 2), ("count", C.POINTER(C.c_int)), ("partner", C.POINTER(C.c_int64)),
        ("xi", C.POINTER(C.c_double)), ("overflow", C.c_int),
    ]


class _OrcLbm(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_sub", C.c_int), ("tau", C.c_double),
        ("body_force", C.c_double * 3), ("f", C.POINTER(C.c_double)), ("f_tmp", C.POINTER(C.c_double)),
        ("F", C.POINTER(C.c_double)), ("U", C.POINTER(C.c_double)), ("coupled", C.POINTER(C.c_uint8)),
        ("phase", C.c_int), ("steps", C.c_int64),
    ]


class _OrcSystem(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("n_rods", C.c_int64), ("rod_offset", C.POINTER(C.c_int64)),
        ("n_bonds", C.c_int64), ("bond_p1", C.POINTER(C.c_int64)), ("bond_p2", C.POINTER(C.c_int64)),
        ("bond_ri", C.POINTER(C.c_double)), ("bond_K", C.POINTER(C.c_double)),
        ("q_rest", C.POINTER(C.c_double)), ("mass", C.POINTER(C.c_double)),
        ("radius", C.POINTER(C.c_double)), ("m_body", C.POINTER(C.c_double)),
        ("clamped", C.POINTER(C.c_uint8)),
        ("B", C.c_double * 3), ("B_rod", C.POINTER(C.c_double)),
        ("Brot_amp", C.c_double), ("Brot_omega", C.c_double),
        ("Brot_e1", C.c_double * 3), ("Brot_e2", C.c_double * 3),
        ("gradB", C.c_double * 9), ("gradB_x0", C.c_double * 3),
        ("c", C.c_double), ("dipole_mode", C.c_int), ("n_threads", C.c_int),
        ("damping", C.c_double), ("dt", C.c_double),
        ("bond_g", C.POINTER(C.c_double)), ("bond_hist", C.POINTER(C.c_double)),
        ("contact", C.POINTER(_OrcContact)), ("lbm", C.POINTER(_OrcLbm)),
    ]


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Oracle bound to one RodSystem (copies every array it keeps)."""

    def __init__(self, sysm, n_threads: int = 0):
        L = lib()
        self.sys = sysm
        self.n = sysm.n
        self._keep = {}
        k = self._keep
        k["rod_offset"] = np.ascontiguousarray(sysm.rod_offset, dtype=np.int64)
        nb = self.n - sysm.n_rods
        k["p1"] = np.zeros(max(nb, 1), dtype=np.int64)
        k["p2"] = np.zeros(max(nb, 1), dtype=np.int64)
        k["ri"] = np.zeros(3 * max(nb, 1))
        k["K"] = np.zeros(4 * max(nb, 1))
        k["q_rest"] = _c64(sysm.q_rest).ravel()
        k["mass"] = _c64(sysm.mass)
        k["radius"] = _c64(sysm.radius)
        k["m_body"] = _c64(sysm.m_body).ravel()
        k["clamped"] = np.ascontiguousarray(sysm.clamped, dtype=np.uint8)
        s = _OrcSystem()
        s.n = self.n
        s.n_rods = sysm.n_rods
        s.rod_offset = k["rod_offset"].ctypes.data_as(C.POINTER(C.c_int64))
        s.bond_p1 = k["p1"].ctypes.data_as(C.POINTER(C.c_int64))
        s.bond_p2 = k["p2"].ctypes.data_as(C.POINTER(C.c_int64))
        s.bond_ri = _dp(k["ri"])
        s.bond_K = _dp(k["K"])
        s.q_rest = _dp(k["q_rest"])
        s.mass = _dp(k["mass"])
        s.radius = _dp(k["radius"])
        s.m_body = _dp(k["m_body"])
        s.clamped = k["clamped"].ctypes.data_as(C.POINTER(C.c_uint8))
        s.B[:] = list(map(float, sysm.B))
        if sysm.B_rod is not None:
            k["B_rod"] = _c64(sysm.B_rod).ravel()
            s.B_rod = _dp(k["B_rod"])
        s.Brot_amp = float(sysm.Brot_amp)
        s.Brot_omega = float(sysm.Brot_omega)
        s.Brot_e1[:] = list(map(float, sysm.Brot_e1))
        s.Brot_e2[:] = list(map(float, sysm.Brot_e2))
        s.gradB[:] = list(map(float, np.asarray(sysm.gradB).ravel()))
        s.gradB_x0[:] = list(map(float, sysm.gradB_x0))
        s.c = float(sysm.mu0_over_4pi)
        s.dipole_mode = int(sysm.dipole_mode)
        s.n_threads = int(n_threads)
        s.damping = float(sysm.damping)
        s.dt = float(sysm.dt)
        self._s = s
        xr = _c64(sysm.x_rest).ravel()
        rc = L.orc_init_bonds(C.byref(s), _dp(xr), _dp(_c64(sysm.E)), _dp(_c64(sysm.nu)), _dp(_c64(sysm.d)))
        if rc != 0:
            raise ValueError("oracle: bad rest configuration (zero-length bond)")
        if sysm.bond_damping is not None:
            # per-rod coefficients repeated on each bond of the rod
            g_rod = _c64(sysm.bond_damping).reshape(sysm.n_rods, 4)
            lens = np.maximum(np.diff(np.asarray(sysm.rod_offset, dtype=np.int64)) - 1, 0)
            k["bond_g"] = np.ascontiguousarray(np.repeat(g_rod, lens, axis=0).ravel())
            if k["bond_g"].size == 0:
                k["bond_g"] = np.zeros(4)
            k["bond_hist"] = np.full(6 * max(nb, 1), np.nan)
            s.bond_g = _dp(k["bond_g"])
            s.bond_hist = _dp(k["bond_hist"])
        if sysm.contact is not None:
            cp = sysm.contact
            cs = _OrcContact()
            cs.E, cs.nu, cs.mu = float(cp.E), float(cp.nu), float(cp.mu)
            cs.gamma_n, cs.gamma_t = float(cp.gamma_n), float(cp.gamma_t)
            cs.exclude, cs.cap = int(cp.exclude), int(cp.cap)
            cs.level = 0
            cs.valid[0] = cs.valid[1] = 0
            k["c_count"] = np.zeros(2 * max(self.n, 1), dtype=np.int32)
            k["c_partner"] = np.zeros(2 * max(self.n, 1) * cp.cap, dtype=np.int64)
            k["c_xi"] = np.zeros(2 * max(self.n, 1) * cp.cap * 3)
            cs.count = k["c_count"].ctypes.data_as(C.POINTER(C.c_int))
            cs.partner = k["c_partner"].ctypes.data_as(C.POINTER(C.c_int64))
            cs.xi = _dp(k["c_xi"])
            k["contact"] = cs
            s.contact = C.pointer(cs)
        # state
        self.x = _c64(sysm.x).ravel().copy()
        if sysm.lbm is not None:
            lp = sysm.lbm
            ls = _OrcLbm()
            ls.nx, ls.ny, ls.nz, ls.n_sub = int(lp.nx), int(lp.ny), int(lp.nz), int(lp.n_sub)
            ls.tau = float(lp.tau)
            ls.body_force[:] = [float(b) for b in lp.body_force]
            nn = lp.nodes
            k["l_f"] = np.zeros(19 * nn)
            k["l_ft"] = np.zeros(19 * nn)
            k["l_F"] = np.zeros(3 * nn)
            k["l_U"] = np.zeros(3 * max(self.n, 1))
            ls.f, ls.f_tmp, ls.F, ls.U = _dp(k["l_f"]), _dp(k["l_ft"]), _dp(k["l_F"]), _dp(k["l_U"])
            if lp.coupled is not None:
                k["l_c"] = np.ascontiguousarray(lp.coupled, dtype=np.uint8)
                ls.coupled = k["l_c"].ctypes.data_as(C.POINTER(C.c_uint8))
            k["lbm"] = ls
            s.lbm = C.pointer(ls)
            r0 = None if lp.rho0 is None else _c64(lp.rho0).ravel()
            u0 = None if lp.u0 is None else _c64(lp.u0).ravel()
            L.orc_lbm_init(C.byref(ls), None if r0 is None else r0.ctypes.data,
                           None if u0 is None else u0.ctypes.data)
            L.orc_lbm_interp(C.byref(ls), _dp(self.x), self.n, _dp(k["l_U"]))
        self.q = _c64(sysm.q).ravel().copy()
        self.v = _c64(sysm.v).ravel().copy()
        self.w = _c64(sysm.omega).ravel().copy()
        self.t = C.c_double(float(sysm.t0))
        self.f = np.zeros(3 * self.n)
        self.tau = np.zeros(3 * self.n)
        self.forces_valid = False

    @property
    def bond_K(self):
        return self._keep["K"].reshape(-1, 4)[: self.n - self.sys.n_rods]

    @property
    def bond_ri(self):
        return self._keep["ri"].reshape(-1, 3)[: self.n - self.sys.n_rods]

    @property
    def bond_history(self):
        """[n_bonds, 2, 3]: (gamma, psi, theta) of the previous and current level."""
        h = self._keep.get("bond_hist")
        return None if h is None else h.reshape(-1, 2, 3)[: self.n - self.sys.n_rods].copy()

    def reset_history(self):
        """Forget the recorded bond measures and contact displacements (as a
        new state does)."""
        if "bond_hist" in self._keep:
            self._keep["bond_hist"][:] = np.nan
        if "contact" in self._keep:
            cs = self._keep["contact"]
            cs.valid[0] = cs.valid[1] = 0
            cs.level = 0

    def contacts(self, level="current"):
        """{(i, j): xi} of the given level ("current" or "previous"), or None
        when that level holds no record."""
        cs = self._keep.get("contact")
        if cs is None:
            return None
        L = cs.level if level == "current" else 1 - cs.level
        if not cs.valid[L]:
            return None
        n, cap = self.n, cs.cap
        cnt = self._keep["c_count"].reshape(2, n)[L]
        par = self._keep["c_partner"].reshape(2, n, cap)[L]
        xi = self._keep["c_xi"].reshape(2, n, cap, 3)[L]
        return {(i, int(par[i, k])): xi[i, k].copy() for i in range(n) for k in range(cnt[i])}

    # ---- fluid (R12)
    @property
    def lbm(self):
        return self._keep.get("lbm")

    def lbm_macro(self):
        """(rho [nodes], u [nodes, 3]) of the current fluid state."""
        ls = self._keep["lbm"]
        nn = ls.nx * ls.ny * ls.nz
        rho = np.zeros(nn)
        u = np.zeros(3 * nn)
        lib().orc_lbm_macro(C.byref(ls), rho.ctypes.data, _dp(u))
        return rho, u.reshape(-1, 3)

    def lbm_step(self, n: int = 1):
        for _ in range(n):
            lib().orc_lbm_step(C.byref(self._keep["lbm"]))

    def lbm_force_field(self):
        """[3, nodes] reaction force accumulated for the next LBM step."""
        return self._keep["l_F"].reshape(3, -1).copy()

    def lbm_interp(self, x):
        x = _c64(x).ravel()
        U = np.zeros_like(x)
        lib().orc_lbm_interp(C.byref(self._keep["lbm"]), _dp(x), len(x) // 3, _dp(U))
        return U.reshape(-1, 3)

    @property
    def lbm_U(self):
        return self._keep["l_U"][: 3 * self.n].reshape(-1, 3).copy()

    @property
    def contact_overflow(self):
        cs = self._keep.get("contact")
        return bool(cs.overflow) if cs is not None else False

    def set_threads(self, n_threads: int):
        self._s.n_threads = int(n_threads)

    def forces(self, x=None, q=None, v=None, w=None, t=None, want_energy=False, want_m=False):
        """Forces/torques [N,3] of the given (or current) state."""
        x = self.x if x is None else _c64(x).ravel()
        q = self.q if q is None else _c64(q).ravel()
        v = self.v if v is None else _c64(v).ravel()
        w = self.w if w is None else _c64(w).ravel()
        t = self.t.value if t is None else float(t)
        f = np.zeros(3 * self.n)
        tau = np.zeros(3 * self.n)
        m = np.zeros(3 * self.n) if want_m else None
        e = np.zeros(5) if want_energy else None
        rc = lib().orc_forces(C.byref(self._s), _dp(x), _dp(q), _dp(v), _dp(w), t, _dp(f), _dp(tau),
                              m.ctypes.data if m is not None else None,
                              e.ctypes.data if e is not None else None)
        if rc != 0:
            raise RuntimeError("oracle forces failed")
        out = [f.reshape(-1, 3), tau.reshape(-1, 3)]
        if want_m:
            out.append(m.reshape(-1, 3))
        if want_energy:
            out.append(e)
        return tuple(out)

    def energy(self):
        return self.forces(want_energy=True)[2]

    def dipole_sample(self, idx, x=None, m=None):
        """Dipole force/torque/field on particles idx (all partners)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        x = self.x if x is None else _c64(x).ravel()
        if m is None:
            m = self.forces(want_m=True)[2].ravel()
        m = _c64(m).ravel()
        F = np.zeros(3 * len(idx))
        T = np.zeros(3 * len(idx))
        H = np.zeros(3 * len(idx))
        rc = lib().orc_dipole_sample(C.byref(self._s), _dp(x), _dp(m),
                                     idx.ctypes.data_as(C.POINTER(C.c_int64)), len(idx),
                                     _dp(F), _dp(T), H.ctypes.data)
        if rc != 0:
            raise RuntimeError("oracle dipole_sample failed")
        return F.reshape(-1, 3), T.reshape(-1, 3), H.reshape(-1, 3)

    def term_scales(self, idx=None):
        """Per-particle condition scales (sum of the magnitudes of every
        bond, Zeeman, dipole-pair and damping term) of the force and torque
        of the current state, for particles idx (default: all)."""
        idx = np.arange(self.n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
        sf = np.zeros(len(idx))
        st = np.zeros(len(idx))
        rc = lib().orc_term_scales(C.byref(self._s), _dp(self.x), _dp(self.q), _dp(self.v), _dp(self.w),
                                   self.t.value, idx.ctypes.data_as(C.POINTER(C.c_int64)), len(idx),
                                   _dp(sf), _dp(st))
        if rc != 0:
            raise RuntimeError("oracle term_scales failed")
        return sf, st

    def contact_sample(self, idx):
        """Contact forces/torques on particles idx from all others, fresh state."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        F = np.zeros(3 * len(idx))
        T = np.zeros(3 * len(idx))
        rc = lib().orc_contact_sample(C.byref(self._s), _dp(self.x), _dp(self.v), _dp(self.w),
                                      idx.ctypes.data_as(C.POINTER(C.c_int64)), len(idx), _dp(F), _dp(T))
        if rc != 0:
            raise RuntimeError("oracle contact_sample failed")
        return F.reshape(-1, 3), T.reshape(-1, 3)

    def run(self, n_steps: int):
        rc = lib().orc_run(C.byref(self._s), _dp(self.x), _dp(self.q), _dp(self.v), _dp(self.w),
                           C.byref(self.t), int(n_steps), _dp(self.f), _dp(self.tau),
                           1 if self.forces_valid else 0)
        if rc != 0:
            raise RuntimeError("oracle run failed")
        self.forces_valid = True

    def state(self):
        return (self.x.reshape(-1, 3).copy(), self.q.reshape(-1, 4).copy(),
                self.v.reshape(-1, 3).copy(), self.w.reshape(-1, 3).copy(), self.t.value)


def bond(x1, x2, q1, q2, ri, K, m_branch=-1):
    """Single-bond evaluation: returns f1, tau1, f2, tau2, U, diag."""
    L = lib()
    a = [_c64(v).copy() for v in (x1, x2, q1, q2, ri, K)]
    outs = [np.zeros(3) for _ in range(4)]
    U = np.zeros(1)
    diag = np.zeros(8)
    L.orc_bond(*[_dp(v) for v in a], int(m_branch), *[_dp(o) for o in outs], _dp(U), _dp(diag))
    return outs[0], outs[1], outs[2], outs[3], float(U[0]), diag


def bond_damped(x1, x2, q1, q2, ri, K, g, v1, v2, prev, dt):
    """Single damped bond: prev = (gamma, psi, theta) or None.
    Returns f1, tau1, f2, tau2, U, (gamma, psi, theta)."""
    L = lib()
    a = [_c64(v).copy() for v in (x1, x2, q1, q2, ri, K, g, v1, v2)]
    pv = None if prev is None else _c64(prev).copy()
    outs = [np.zeros(3) for _ in range(4)]
    U = np.zeros(1)
    meas = np.zeros(3)
    L.orc_bond_damped(*[_dp(v) for v in a], None if pv is None else pv.ctypes.data, float(dt),
                      *[_dp(o) for o in outs], _dp(U), _dp(meas))
    return outs[0], outs[1], outs[2], outs[3], float(U[0]), meas


def contact_pair(params, xi, xj, vi, vj, wi, wj, Ri, Rj, xi_old, dt):
    """One Hertz-Mindlin pair: None when apart, else (f_i, tau_i, tau_j, xi_new)."""
    cs = _OrcContact()
    cs.E, cs.nu, cs.mu = float(params.E), float(params.nu), float(params.mu)
    cs.gamma_n, cs.gamma_t = float(params.gamma_n), float(params.gamma_t)
    a = [_c64(v).copy() for v in (xi, xj, vi, vj, wi, wj)]
    xo = None if xi_old is None else _c64(xi_old).copy()
    outs = [np.zeros(3) for _ in range(4)]
    hit = lib().orc_contact_pair(C.byref(cs), *[_dp(v) for v in a], float(Ri), float(Rj),
                                 None if xo is None else xo.ctypes.data, float(dt), *[_dp(o) for o in outs])
    return tuple(outs) if hit else None


def lbm_lattice():
    e = (C.c_int * 57)()
    w = np.zeros(19)
    lib().orc_lbm_lattice(e, _dp(w))
    return np.array(list(e), dtype=np.int64).reshape(19, 3), w


def ibm_phi(r):
    return float(lib().orc_ibm_phi(float(r)))


def richardson(q, w, dt):
    out = np.zeros(4)
    lib().orc_richardson(_dp(_c64(q).copy()), _dp(_c64(w).copy()), float(dt), _dp(out))
    return out


def quat_mul(a, b):
    out = np.zeros(4)
    lib().orc_quat_mul(_dp(_c64(a).copy()), _dp(_c64(b).copy()), _dp(out))
    return out


def align_z(r, branch=-1):
    out = np.zeros(4)
    lib().orc_align_z(_dp(_c64(r).copy()), int(branch), _dp(out))
    return out


def rotate(q, v):
    out = np.zeros(3)
    lib().orc_rotate(_dp(_c64(q).copy()), _dp(_c64(v).copy()), _dp(out))
    return out


__all__ = ["Oracle", "bond", "bond_damped", "contact_pair", "lbm_lattice", "ibm_phi", "richardson", "quat_mul", "rotate", "align_z", "lib"]
