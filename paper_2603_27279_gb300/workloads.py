"""Seeded synthetic rod systems shaped like the paper's examples.

This module only *describes* systems (positions, orientations, material,
field, topology).  It holds none of the method's arithmetic: no bond
kinematics, no forces, no integration.  Both the CUDA library (through
``paper_2603_27279_gb300.bpm``) and the CPU FP64 oracle (``oracle/``) read the
same ``RodSystem`` arrays, so the random numbers never have to match across
languages.

Conventions shared by every consumer:

* particle arrays are AoS per particle: ``x[N,3]``, ``q[N,4]`` (w, x, y, z;
  Hamilton product; a body vector maps to space as ``q v q*``), ``v[N,3]``,
  ``omega[N,3]`` (space frame);
* rods are CSR: rod ``r`` holds particles ``rod_offset[r] .. rod_offset[r+1]-1``
  and bonds join consecutive particles of a rod (the paper's rods, Fig. 1);
* material is per rod: Young's modulus ``E``, Poisson ratio ``nu``
  (G = E / (2 (1 + nu))) and bond diameter ``d`` (the cylinder of the
  spring-constant derivation, SI "Deriving the spring constants").

Workloads (sizes and recipes are those of the benchmark configurations):

* ``straight_rod``   64 particles along x, small seeded perturbation;
* ``helix``          one 16384-particle helix (radius 20, pitch 5) with a 4*pi
                     twist spread along the rod (stand-in for the writhing rods
                     of the plectoneme examples);
* ``batched_rods``   2048 independent straight rods, lengths U{16..1024},
                     a random field per rod;
* ``adjoint_rod``    2048-particle clamped rod with Gaussian magnetisation;
* ``cilia``          512 vertical rods x 256 particles on a 16 x 32 lattice
                     (stand-in for the magnetic cilia array example) with a
                     rotating field.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 20261203

PRECISION_FP64 = 0
PRECISION_MIXED = 1
PRECISION_FF = 2

DIPOLE_OFF = 0
DIPOLE_GLOBAL = 1
DIPOLE_PER_ROD = 2


@dataclasses.dataclass
class ContactParams:
    """Hertz-Mindlin contact between non-bonded particles (Methods, "Contact")."""

    E: float = 1e4          # particle Young's modulus
    nu: float = 0.3         # particle Poisson ratio
    mu: float = 0.5         # Coulomb friction coefficient
    gamma_n: float = 0.0    # viscous damping of the normal contact velocity
    gamma_t: float = 0.0    # viscous damping of the tangential contact velocity
    exclude: int = 3        # same-rod pairs within this many bonds have no contact
    cap: int = 16           # most contacts per particle


@dataclasses.dataclass
class LbmParams:
    """Periodic D3Q19 lattice-Boltzmann fluid coupled to the particles by a
    penalty immersed boundary (Methods, "Lattice Boltzmann method",
    "Immersed boundary coupling").  Lattice units: spacing 1, one LBM step =
    n_sub DEM steps = 1 time unit (so the system's dt must be 1 / n_sub),
    reference density 1."""

    nx: int = 32
    ny: int = 32
    nz: int = 32
    n_sub: int = 10
    tau: float = 0.8
    body_force: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    rho0: Optional[np.ndarray] = None     # [nodes] initial density (None: 1)
    u0: Optional[np.ndarray] = None       # [nodes, 3] initial velocity (None: 0)
    coupled: Optional[np.ndarray] = None  # uint8 [N] particles coupled to the fluid (None: all)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass
class RodSystem:
    """Raw description of a bonded-particle rod system (all float64 / numpy)."""

    name: str
    rod_offset: np.ndarray          # int64 [R+1]
    x: np.ndarray                   # [N,3]
    q: np.ndarray                   # [N,4]
    v: np.ndarray                   # [N,3]
    omega: np.ndarray               # [N,3]
    mass: np.ndarray                # [N]
    radius: np.ndarray              # [N]
    m_body: np.ndarray              # [N,3] body-frame dipole moment
    clamped: np.ndarray             # uint8 [N]
    x_rest: np.ndarray              # [N,3] configuration in which bonds are created
    q_rest: np.ndarray              # [N,4]
    E: np.ndarray                   # [R]
    nu: np.ndarray                  # [R]
    d: np.ndarray                   # [R] bond diameter
    B: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    B_rod: Optional[np.ndarray] = None     # [R,3] per-rod uniform field
    Brot_amp: float = 0.0                  # rotating component amplitude
    Brot_omega: float = 0.0                # its angular frequency
    Brot_e1: np.ndarray = dataclasses.field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    Brot_e2: np.ndarray = dataclasses.field(default_factory=lambda: np.array([0.0, 1.0, 0.0]))
    gradB: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((3, 3)))
    gradB_x0: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    mu0_over_4pi: float = 1.0
    dipole_mode: int = DIPOLE_GLOBAL
    damping: float = 0.0
    bond_damping: Optional[np.ndarray] = None  # [R,4] g_r, g_s, g_t, g_b per rod
    contact: Optional[ContactParams] = None
    lbm: Optional[LbmParams] = None
    dt: float = 1e-3
    t0: float = 0.0
    n_steps: int = 1
    precision: int = PRECISION_FP64

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_rods(self) -> int:
        return int(self.rod_offset.shape[0] - 1)

    @property
    def n_bonds(self) -> int:
        return self.n - self.n_rods

    def rod_lengths(self) -> np.ndarray:
        return np.diff(self.rod_offset)

    def ordered_pairs(self) -> int:
        """Ordered dipole pairs i != j evaluated per force call."""
        if self.dipole_mode == DIPOLE_OFF:
            return 0
        if self.dipole_mode == DIPOLE_GLOBAL:
            return self.n * (self.n - 1)
        L = self.rod_lengths().astype(np.int64)
        return int(np.sum(L * (L - 1)))

    def copy(self) -> "RodSystem":
        out = dataclasses.replace(self)
        for f in dataclasses.fields(self):
            val = getattr(self, f.name)
            if isinstance(val, np.ndarray):
                setattr(out, f.name, val.copy())
            elif isinstance(val, (ContactParams, LbmParams)):
                setattr(out, f.name, dataclasses.replace(val))
        return out


# --------------------------------------------------------------------------
# helpers (input construction only)
# --------------------------------------------------------------------------

def _axis_angle_quat(axis: np.ndarray, angle: np.ndarray) -> np.ndarray:
    """Unit quaternion (cos a/2, sin a/2 n) for unit axes n[...,3], angles a[...]."""
    half = 0.5 * np.asarray(angle, dtype=np.float64)
    out = np.empty(axis.shape[:-1] + (4,))
    out[..., 0] = np.cos(half)
    out[..., 1:] = np.sin(half)[..., None] * axis
    return out


def _unit_sphere(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def random_unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    g[g[:, 0] < 0] *= -1.0
    return g


def _identity_q(n: int) -> np.ndarray:
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return q


def _material(R: int, E=1e4, nu=0.3, d=1.0):
    return np.full(R, E), np.full(R, nu), np.full(R, d)


def _straight_rods_along(axis: np.ndarray, lengths: np.ndarray, origins: np.ndarray, spacing=1.0):
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    N = int(offs[-1])
    x = np.empty((N, 3))
    for r, L in enumerate(lengths):
        k = np.arange(L, dtype=np.float64)[:, None]
        x[offs[r]:offs[r + 1]] = origins[r][None, :] + spacing * k * axis[None, :]
    return offs, x


def _perturb(rng, x, q, pos_sigma, rot_max):
    """Positions += N(0, sigma^2); orientations pre-multiplied by a random
    rotation of angle U[0, rot_max) about a uniform axis (q is identity here)."""
    N = x.shape[0]
    x = x + pos_sigma * rng.standard_normal((N, 3))
    axis = _unit_sphere(rng, N)
    ang = rng.uniform(0.0, rot_max, N)
    assert np.allclose(q, _identity_q(N))
    q = _axis_angle_quat(axis, ang)
    return x, q


# --------------------------------------------------------------------------
# benchmark-shaped workloads
# --------------------------------------------------------------------------

def straight_rod(n: int = 64, seed: int = SEED_BASE + 0, dipole_mode: int = DIPOLE_GLOBAL,
                 pos_sigma: float = 1e-3, rot_max: float = 1e-3) -> RodSystem:
    """One rod of n particles (diameter 1, spacing 1, mass 1) along x.

    Bonds are created on the unperturbed straight rod (q = 1); then positions
    get N(0, 1e-3^2) noise per component and orientations a random rotation
    below 1e-3 rad.  |m| = 1 along the rod axis, B = 0.5 (cos 30, sin 30, 0),
    mu0/4pi = 1, particle 0 clamped, damping 0.1, dt = 1e-3, 1000 steps.
    """
    rng = np.random.default_rng(seed)
    offs, x0 = _straight_rods_along(np.array([1.0, 0.0, 0.0]), np.array([n]), np.zeros((1, 3)))
    q0 = _identity_q(n)
    x, q = _perturb(rng, x0, q0, pos_sigma, rot_max)
    E, nu, d = _material(1)
    clamped = np.zeros(n, dtype=np.uint8)
    clamped[0] = 1
    deg = math.pi / 180.0
    return RodSystem(
        name=f"straight_rod_{n}", rod_offset=offs, x=x, q=q, v=np.zeros((n, 3)), omega=np.zeros((n, 3)),
        mass=np.ones(n), radius=np.full(n, 0.5), m_body=np.tile([1.0, 0.0, 0.0], (n, 1)), clamped=clamped,
        x_rest=x0, q_rest=q0, E=E, nu=nu, d=d,
        B=0.5 * np.array([math.cos(30 * deg), math.sin(30 * deg), 0.0]),
        mu0_over_4pi=1.0, dipole_mode=dipole_mode, damping=0.1, dt=1e-3, n_steps=1000,
        precision=PRECISION_FP64)


def helix(n: int = 16384, seed: int = SEED_BASE + 1, radius: float = 20.0, pitch: float = 5.0,
          total_twist: float = 4.0 * math.pi, precision: int = PRECISION_FP64) -> RodSystem:
    """One helical rod: x_k = (R cos t_k, R sin t_k, p t_k / 2pi), arc spacing 1.

    Rest state is this helix with q = 1 (bonds created in the coiled state);
    the current state carries a twist of total_twist spread linearly along the
    rod, q_k = exp(1/2 * total_twist * k/(n-1) * T_k) about the local tangent.
    m_body = T_k, B = 0.2 z, particle 0 clamped, no damping, dt = 5e-4.
    The seed is unused (the configuration is deterministic) but kept for a
    uniform signature.
    """
    del seed
    c = pitch / (2.0 * math.pi)
    s_per_t = math.sqrt(radius * radius + c * c)
    t = np.arange(n, dtype=np.float64) / s_per_t
    x = np.stack([radius * np.cos(t), radius * np.sin(t), c * t], axis=1)
    T = np.stack([-radius * np.sin(t), radius * np.cos(t), np.full(n, c)], axis=1) / s_per_t
    psi = total_twist * np.arange(n) / max(n - 1, 1)
    q = _axis_angle_quat(T, psi)
    E, nu, d = _material(1)
    clamped = np.zeros(n, dtype=np.uint8)
    clamped[0] = 1
    return RodSystem(
        name=f"helix_{n}", rod_offset=np.array([0, n], dtype=np.int64), x=x, q=q,
        v=np.zeros((n, 3)), omega=np.zeros((n, 3)), mass=np.ones(n), radius=np.full(n, 0.5),
        m_body=T.copy(), clamped=clamped, x_rest=x.copy(), q_rest=_identity_q(n), E=E, nu=nu, d=d,
        B=np.array([0.0, 0.0, 0.2]), mu0_over_4pi=1.0, dipole_mode=DIPOLE_GLOBAL, damping=0.0,
        dt=5e-4, n_steps=100, precision=precision)


def batched_rods(n_rods: int = 2048, lmin: int = 16, lmax: int = 1024, seed: int = SEED_BASE + 2,
                 precision: int = PRECISION_MIXED, pos_sigma: float = 1e-3,
                 rot_max: float = 1e-3) -> RodSystem:
    """Independent straight rods along x, lengths U{lmin..lmax} (seeded).

    Each rod has its own uniform field: direction uniform on S^2, magnitude
    U[0.1, 1].  Axial |m| = 1, particle 0 of each rod clamped, damping 0.1,
    dt = 1e-3, per-rod all-pairs dipole, 200 steps.  Rods sit 4 apart in y.
    """
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lmin, lmax + 1, size=n_rods)
    origins = np.zeros((n_rods, 3))
    origins[:, 1] = 4.0 * np.arange(n_rods)
    offs, x0 = _straight_rods_along(np.array([1.0, 0.0, 0.0]), lengths, origins)
    N = x0.shape[0]
    q0 = _identity_q(N)
    x, q = _perturb(rng, x0, q0, pos_sigma, rot_max)
    dirs = _unit_sphere(rng, n_rods)
    mags = rng.uniform(0.1, 1.0, n_rods)
    clamped = np.zeros(N, dtype=np.uint8)
    clamped[offs[:-1]] = 1
    E, nu, d = _material(n_rods)
    return RodSystem(
        name=f"batched_rods_{n_rods}", rod_offset=offs, x=x, q=q, v=np.zeros((N, 3)),
        omega=np.zeros((N, 3)), mass=np.ones(N), radius=np.full(N, 0.5),
        m_body=np.tile([1.0, 0.0, 0.0], (N, 1)), clamped=clamped, x_rest=x0, q_rest=q0,
        E=E, nu=nu, d=d, B=np.zeros(3), B_rod=dirs * mags[:, None], mu0_over_4pi=1.0,
        dipole_mode=DIPOLE_PER_ROD, damping=0.1, dt=1e-3, n_steps=200, precision=precision)


def subset_rods(sysm: RodSystem, rods) -> RodSystem:
    """The rods `rods` (indices, in order) of a system as a system of their
    own: particle arrays, per-rod material and fields cut out, the global
    field, dipole mode and time stepping kept.  For systems whose rods do not
    interact (per-rod or no dipoles, no contact, no fluid) each rod then
    evolves exactly as it does inside the whole system."""
    rods = np.asarray(rods, dtype=np.int64)
    offs = np.asarray(sysm.rod_offset, dtype=np.int64)
    parts = [np.arange(offs[r], offs[r + 1]) for r in rods]
    idx = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
    new_offs = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    out = sysm.copy()
    out.name = f"{sysm.name}_rods{len(rods)}"
    out.rod_offset = new_offs
    for k in ("x", "q", "v", "omega", "mass", "radius", "m_body", "clamped", "x_rest", "q_rest"):
        setattr(out, k, np.ascontiguousarray(getattr(sysm, k)[idx]))
    for k in ("E", "nu", "d"):
        setattr(out, k, np.ascontiguousarray(getattr(sysm, k)[rods]))
    if sysm.B_rod is not None:
        out.B_rod = np.ascontiguousarray(np.asarray(sysm.B_rod)[rods])
    if sysm.bond_damping is not None:
        out.bond_damping = np.ascontiguousarray(np.asarray(sysm.bond_damping)[rods])
    return out


def adjoint_rod(n: int = 2048, seed: int = SEED_BASE + 3) -> RodSystem:
    """Clamped rod along x with per-particle magnetisation m_i ~ N(0, 1)^3.

    B = (0, 0.3, 0), damping 0.1, dt = 1e-3, 500 steps, all-pairs dipole.
    """
    rng = np.random.default_rng(seed)
    offs, x0 = _straight_rods_along(np.array([1.0, 0.0, 0.0]), np.array([n]), np.zeros((1, 3)))
    q0 = _identity_q(n)
    m = rng.standard_normal((n, 3))
    E, nu, d = _material(1)
    clamped = np.zeros(n, dtype=np.uint8)
    clamped[0] = 1
    return RodSystem(
        name=f"adjoint_rod_{n}", rod_offset=offs, x=x0.copy(), q=q0.copy(), v=np.zeros((n, 3)),
        omega=np.zeros((n, 3)), mass=np.ones(n), radius=np.full(n, 0.5), m_body=m, clamped=clamped,
        x_rest=x0, q_rest=q0, E=E, nu=nu, d=d, B=np.array([0.0, 0.3, 0.0]), mu0_over_4pi=1.0,
        dipole_mode=DIPOLE_GLOBAL, damping=0.1, dt=1e-3, n_steps=500, precision=PRECISION_FP64)


def cilia(nx: int = 16, ny: int = 32, length: int = 256, spacing: float = 4.0,
          tilt_deg: float = 20.0, seed: int = SEED_BASE + 4,
          precision: int = PRECISION_MIXED) -> RodSystem:
    """Vertical rods (along z) on an nx x ny square lattice, bases clamped.

    m_body = (sin tilt, 0, cos tilt), B(t) = 0.5 (cos w t, sin w t, 0) with
    w = 2 pi / 2000, damping 0.1, dt = 1e-3, global all-pairs dipole, 50 steps.
    """
    del seed
    R = nx * ny
    gx, gy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    origins = np.zeros((R, 3))
    origins[:, 0] = spacing * gx.ravel()
    origins[:, 1] = spacing * gy.ravel()
    lengths = np.full(R, length)
    offs, x = _straight_rods_along(np.array([0.0, 0.0, 1.0]), lengths, origins)
    N = x.shape[0]
    clamped = np.zeros(N, dtype=np.uint8)
    clamped[offs[:-1]] = 1
    tilt = math.radians(tilt_deg)
    E, nu, d = _material(R)
    return RodSystem(
        name=f"cilia_{nx}x{ny}x{length}", rod_offset=offs, x=x, q=_identity_q(N), v=np.zeros((N, 3)),
        omega=np.zeros((N, 3)), mass=np.ones(N), radius=np.full(N, 0.5),
        m_body=np.tile([math.sin(tilt), 0.0, math.cos(tilt)], (N, 1)), clamped=clamped,
        x_rest=x.copy(), q_rest=_identity_q(N), E=E, nu=nu, d=d, B=np.zeros(3),
        Brot_amp=0.5, Brot_omega=2.0 * math.pi / 2000.0, mu0_over_4pi=1.0,
        dipole_mode=DIPOLE_GLOBAL, damping=0.1, dt=1e-3, n_steps=50, precision=precision)


# --------------------------------------------------------------------------
# small randomised systems for parity tests
# --------------------------------------------------------------------------

def random_rods(lengths, seed: int = SEED_BASE + 100, pos_sigma: float = 0.05,
                rot_max: float = 0.3, random_rest_q: bool = True, vel_sigma: float = 0.1,
                dipole_mode: int = DIPOLE_GLOBAL, with_gradient: bool = True,
                with_rotating: bool = True, per_rod_field: bool = False,
                damping: float = 0.1, dt: float = 1e-3,
                precision: int = PRECISION_FP64) -> RodSystem:
    """Rods along random directions with large deformations and random rest
    orientations: exercises every term of the bond and field models."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    R = len(lengths)
    offs = np.zeros(R + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    N = int(offs[-1])
    x_rest = np.empty((N, 3))
    for r in range(R):
        axis = _unit_sphere(rng, 1)[0]
        origin = rng.uniform(-3.0 * R, 3.0 * R, 3)
        # gently curved rest line so rest bond vectors differ
        k = np.arange(lengths[r], dtype=np.float64)
        bend = _unit_sphere(rng, 1)[0]
        bend -= axis * (bend @ axis)
        bend /= np.linalg.norm(bend)
        x_rest[offs[r]:offs[r + 1]] = origin + np.outer(k, axis) + 0.02 * np.outer(k * k, bend)
    q_rest = random_unit_quaternions(rng, N) if random_rest_q else _identity_q(N)
    x = x_rest + pos_sigma * rng.standard_normal((N, 3))
    # current orientation: the rest quaternion plus Gaussian noise of size
    # rot_max / 2 per component, renormalised (a rotation of order rot_max)
    q = q_rest + 0.5 * rot_max * rng.standard_normal((N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    v = vel_sigma * rng.standard_normal((N, 3))
    omega = vel_sigma * rng.standard_normal((N, 3))
    clamped = np.zeros(N, dtype=np.uint8)
    clamped[offs[:-1]] = 1
    v[clamped == 1] = 0.0
    omega[clamped == 1] = 0.0
    m_body = rng.standard_normal((N, 3))
    E = rng.uniform(5e3, 2e4, R)
    nu = rng.uniform(0.2, 0.45, R)
    d = rng.uniform(0.6, 1.2, R)
    sysm = RodSystem(
        name=f"random_rods_{R}x{int(lengths.mean())}", rod_offset=offs, x=x, q=q, v=v, omega=omega,
        mass=rng.uniform(0.5, 2.0, N), radius=rng.uniform(0.3, 0.7, N), m_body=m_body, clamped=clamped,
        x_rest=x_rest, q_rest=q_rest, E=E, nu=nu, d=d, B=rng.standard_normal(3) * 0.5,
        mu0_over_4pi=1.0, dipole_mode=dipole_mode, damping=damping, dt=dt, n_steps=10,
        precision=precision)
    if per_rod_field:
        sysm.B_rod = rng.standard_normal((R, 3)) * 0.5
    if with_rotating:
        sysm.Brot_amp = 0.3
        sysm.Brot_omega = 2.0 * math.pi / 50.0
        e1 = _unit_sphere(rng, 1)[0]
        e2 = _unit_sphere(rng, 1)[0]
        e2 -= e1 * (e1 @ e2)
        sysm.Brot_e1, sysm.Brot_e2 = e1, e2 / np.linalg.norm(e2)
        sysm.t0 = 0.37
    if with_gradient:
        G = 0.01 * rng.standard_normal((3, 3))
        G = 0.5 * (G + G.T)
        G -= np.eye(3) * np.trace(G) / 3.0
        sysm.gradB = G
        sysm.gradB_x0 = rng.standard_normal(3)
    return sysm


CONFIGS = {
    "straight_rod_64": straight_rod,
    "helix_16384": helix,
    "batched_rods_2048": batched_rods,
    "adjoint_rod_2048": adjoint_rod,
    "cilia_512x256": cilia,
}


def granular(nx: int = 16, ny: int = 16, nz: int = 16, spacing: float = 0.95, seed: int = SEED_BASE + 5,
             jitter: float = 0.04, rmin: float = 0.45, rmax: float = 0.55, vel_sigma: float = 0.05,
             contact: Optional[ContactParams] = None, dt: float = 1e-3) -> RodSystem:
    """Unbonded spheres on a jittered cubic lattice whose spacing is a little
    below their diameter, so that each touches most of its six lattice
    neighbours: the contact-only workload (every particle a rod of one)."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), axis=-1)
    x = g.reshape(-1, 3).astype(np.float64) * spacing
    N = x.shape[0]
    x += rng.uniform(-jitter, jitter, (N, 3))
    offs = np.arange(N + 1, dtype=np.int64)
    return RodSystem(
        name=f"granular_{nx}x{ny}x{nz}", rod_offset=offs, x=x, q=random_unit_quaternions(rng, N),
        v=vel_sigma * rng.standard_normal((N, 3)), omega=vel_sigma * rng.standard_normal((N, 3)),
        mass=rng.uniform(0.8, 1.2, N), radius=rng.uniform(rmin, rmax, N), m_body=np.zeros((N, 3)),
        clamped=np.zeros(N, dtype=np.uint8), x_rest=x.copy(), q_rest=_identity_q(N), E=np.full(N, 1e4),
        nu=np.full(N, 0.3), d=np.full(N, 0.5), dipole_mode=DIPOLE_OFF, damping=0.0,
        contact=contact or ContactParams(E=1e4, nu=0.3, mu=0.5, gamma_n=0.1, gamma_t=0.05), dt=dt)


def crossing_rods(seed: int = SEED_BASE + 6, spacing: float = 0.8, radius: float = 0.5, gap: float = 0.9,
                  dipole_mode: int = DIPOLE_PER_ROD, contact: Optional[ContactParams] = None,
                  dt: float = 1e-3) -> RodSystem:
    """Rods whose particles overlap their bonded neighbours (spacing < 2R, as
    in the paper's contact examples): two straight rods crossing at a centre
    distance `gap` < 2R and a hairpin whose arms lie `gap` apart, so contacts
    occur between rods and between far-apart particles of one rod."""
    rng = np.random.default_rng(seed)
    k = np.arange(30, dtype=np.float64)
    a = np.stack([(k - 15) * spacing, np.zeros(30), np.zeros(30)], axis=1)
    b = np.stack([np.zeros(30) + 0.3 * spacing, (k - 15) * spacing, np.full(30, gap)], axis=1)
    arm = np.arange(20, dtype=np.float64) * spacing
    bend = [[arm[-1] + gap / 2 * math.sin(t), 5.0 + gap / 2 - gap / 2 * math.cos(t), -3.0]
            for t in np.linspace(math.pi / 4, 3 * math.pi / 4, 3)]
    c = np.concatenate([np.stack([arm, np.full(20, 5.0), np.full(20, -3.0)], axis=1), np.array(bend),
                        np.stack([arm[::-1], np.full(20, 5.0 + gap), np.full(20, -3.0)], axis=1)])
    x_rest = np.concatenate([a, b, c])
    N = x_rest.shape[0]
    offs = np.array([0, 30, 60, N], dtype=np.int64)
    q_rest = _identity_q(N)
    x, q = _perturb(rng, x_rest, q_rest, 0.02, 0.05)
    E, nu, d = _material(3)
    return RodSystem(
        name="crossing_rods", rod_offset=offs, x=x, q=q, v=0.05 * rng.standard_normal((N, 3)),
        omega=0.05 * rng.standard_normal((N, 3)), mass=np.ones(N), radius=np.full(N, radius),
        m_body=0.3 * rng.standard_normal((N, 3)), clamped=np.zeros(N, dtype=np.uint8), x_rest=x_rest,
        q_rest=q_rest, E=E, nu=nu, d=d, B=np.array([0.1, 0.0, 0.2]), dipole_mode=dipole_mode, damping=0.05,
        contact=contact or ContactParams(E=1e4, nu=0.3, mu=0.5, gamma_n=0.1, gamma_t=0.05, exclude=3), dt=dt)


def _smooth_field(rng, n, modes=4, amp=0.02):
    """A smooth periodic field on an (nx, ny, nz) lattice: a few random
    Fourier modes per component.  Returns [nodes, 3] (node = i + nx (j + ny k))."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((nx * ny * nz, 3))
    for c in range(3):
        acc = np.zeros_like(i, dtype=np.float64)
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 3, 3)
            ph = rng.uniform(0, 2 * math.pi)
            acc += rng.standard_normal() * np.cos(2 * math.pi * (kx * i / nx + ky * j / ny + kz * k / nz) + ph)
        out[:, c] = amp * acc.ravel() / modes
    return out


def fluid_rods(n=(24, 20, 28), rods=(12, 20), n_sub: int = 10, tau: float = 0.8, seed: int = SEED_BASE + 7,
               body=(2e-5, 0.0, -1e-5), dipole_mode: int = DIPOLE_PER_ROD,
               precision: int = PRECISION_FP64) -> RodSystem:
    """Rods immersed in a periodic D3Q19 fluid with a smooth random initial
    flow and a uniform body force; every particle coupled (lattice units:
    dt = 1 / n_sub, particles inside the box, soft rods (E ~ 1) so that the
    DEM step resolves their fastest mode)."""
    rng = np.random.default_rng(seed)
    s = random_rods(list(rods), seed=seed, dipole_mode=dipole_mode, vel_sigma=0.01, damping=0.02,
                    dt=1.0 / n_sub, precision=precision, with_rotating=False, pos_sigma=0.02, rot_max=0.1)
    s.E = rng.uniform(0.5, 1.0, s.n_rods)
    s.m_body = 0.01 * s.m_body
    s.B = 0.05 * s.B
    s.gradB = 0.05 * s.gradB
    # place the rods inside the box
    lo, hi = s.x_rest.min(axis=0), s.x_rest.max(axis=0)
    box = np.array(n, dtype=np.float64)
    scale = min(1.0, float(np.min((box - 4.0) / np.maximum(hi - lo, 1e-9))))
    shift = (box - (hi - lo) * scale) / 2 - lo * scale
    s.x = s.x * scale + shift
    s.x_rest = s.x_rest * scale + shift
    s.gradB_x0 = s.gradB_x0 * scale + shift
    nodes = n[0] * n[1] * n[2]
    s.lbm = LbmParams(nx=n[0], ny=n[1], nz=n[2], n_sub=n_sub, tau=tau, body_force=np.asarray(body, float),
                      rho0=1.0 + 0.01 * rng.standard_normal(nodes), u0=_smooth_field(rng, n))
    s.name = f"fluid_rods_{n[0]}x{n[1]}x{n[2]}"
    return s


def fluid_cilia(nx: int = 16, ny: int = 16, length: int = 64, lattice=(256, 256, 128), spacing: float = 16.0,
                n_sub: int = 10, tau: float = 0.8, seed: int = SEED_BASE + 8,
                precision: int = PRECISION_FP64) -> RodSystem:
    """A magnetic cilia array in a periodic D3Q19 fluid (lattice units):
    nx x ny vertical rods of `length` particles (spacing 1, radius 0.5, soft
    material E = 2) on a square lattice of `spacing`, bases clamped at
    z = 8, body dipoles tilted 20 degrees toward +x, a rotating field in the
    x-y plane, dipoles within each rod, and a uniform body force driving the
    fluid along +x.  dt = 1 / n_sub."""
    rng = np.random.default_rng(seed)
    R = nx * ny
    lengths = np.full(R, length, dtype=np.int64)
    origins = np.array([[spacing * (i + 0.5), spacing * (j + 0.5), 8.0] for i in range(nx) for j in range(ny)])
    offs, x = _straight_rods_along(np.array([0.0, 0.0, 1.0]), lengths, origins)
    N = x.shape[0]
    x_rest = x.copy()
    x, q = _perturb(rng, x, _identity_q(N), 0.01, 0.01)
    clamped = np.zeros(N, dtype=np.uint8)
    clamped[offs[:-1]] = 1
    tilt = math.radians(20.0)
    m_body = np.tile([0.02 * math.sin(tilt), 0.0, 0.02 * math.cos(tilt)], (N, 1))
    E, nu, d = _material(R, E=2.0)
    s = RodSystem(
        name=f"fluid_cilia_{nx}x{ny}x{length}", rod_offset=offs, x=x, q=q, v=np.zeros((N, 3)),
        omega=np.zeros((N, 3)), mass=np.ones(N), radius=np.full(N, 0.5), m_body=m_body, clamped=clamped,
        x_rest=x_rest, q_rest=_identity_q(N), E=E, nu=nu, d=d, B=np.zeros(3), dipole_mode=DIPOLE_PER_ROD,
        damping=0.0, dt=1.0 / n_sub, precision=precision)
    s.Brot_amp = 0.05
    s.Brot_omega = 2.0 * math.pi / 200.0
    s.Brot_e1 = np.array([1.0, 0.0, 0.0])
    s.Brot_e2 = np.array([0.0, 1.0, 0.0])
    s.lbm = LbmParams(nx=lattice[0], ny=lattice[1], nz=lattice[2], n_sub=n_sub, tau=tau,
                      body_force=np.array([1e-6, 0.0, 0.0]))
    return s
