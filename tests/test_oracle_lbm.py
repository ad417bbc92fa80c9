"""Pins of the oracle's lattice-Boltzmann fluid and immersed-boundary
coupling (Methods, "Lattice Boltzmann method", "Immersed boundary
coupling"; reading R12 of the oracle's header).

* D3Q19 lattice: weights sum to 1, odd moments vanish, the second moment
  is c_s^2 I and the fourth moment is isotropic, c_s^4 (dd + dd + dd).
* BGK with Guo forcing recovers Navier-Stokes with nu = c_s^2 (tau - 1/2):
  a decaying shear wave decays at nu k^2, and the forced Kolmogorov flow
  reaches u = F0 / (rho nu k^2), both with second-order errors in k.  A
  uniform force adds exactly F per node per step to sum f e + F/2.
* Peskin's four-point delta: partition of unity, zero first moment, sum of
  squares 3/8, support of four nodes.
* Penalty coupling: a particle in fluid at rest relaxes at rate
  kappa / m = 1 / dt_LBM within its first cycle, and the reaction spread on
  the lattice sums to -F_p / n_sub for each force evaluation.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, ibm_phi, lbm_lattice
from paper_2603_27279_gb300 import workloads as W


def fluid(n=(16, 4, 16), tau=0.8, n_sub=1, body=(0.0, 0.0, 0.0), rho0=None, u0=None, particles=None,
          masses=None, velocities=None, coupled=None):
    """A fluid box; by default with one particle that does not couple."""
    x = np.array([[0.5, 0.5, 0.5]]) if particles is None else np.asarray(particles, float)
    N = len(x)
    lp = W.LbmParams(nx=n[0], ny=n[1], nz=n[2], n_sub=n_sub, tau=tau, body_force=np.asarray(body, float),
                     rho0=rho0, u0=u0,
                     coupled=np.zeros(N, np.uint8) if (particles is None and coupled is None) else coupled)
    return W.RodSystem(name="fluid", rod_offset=np.arange(N + 1, dtype=np.int64), x=x,
                       q=np.tile([1.0, 0, 0, 0], (N, 1)),
                       v=np.zeros((N, 3)) if velocities is None else np.asarray(velocities, float),
                       omega=np.zeros((N, 3)), mass=np.ones(N) if masses is None else np.asarray(masses, float),
                       radius=np.full(N, 0.5), m_body=np.zeros((N, 3)), clamped=np.zeros(N, np.uint8),
                       x_rest=x.copy(), q_rest=np.tile([1.0, 0, 0, 0], (N, 1)), E=np.ones(N),
                       nu=np.full(N, 0.3), d=np.ones(N), dipole_mode=0, damping=0.0, dt=1.0 / n_sub,
                       lbm=lp)


def test_d3q19_moments():
    e, w = lbm_lattice()
    assert e.shape == (19, 3) and len({tuple(v) for v in e}) == 19
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(w @ e).max() < 1e-16
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(m2, np.eye(3) / 3, atol=1e-16)
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(m3).max() < 1e-16
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)


def test_equilibrium_moments_and_conservation():
    """A random smooth initial state: mass is conserved exactly and momentum
    without forces; a uniform force adds exactly F per node per step."""
    n = (8, 6, 10)
    nodes = n[0] * n[1] * n[2]
    rng = np.random.default_rng(3)
    rho0 = 1.0 + 0.05 * rng.standard_normal(nodes)
    u0 = 0.02 * rng.standard_normal((nodes, 3))
    o = Oracle(fluid(n, rho0=rho0, u0=u0))
    rho, u = o.lbm_macro()
    M0, P0 = rho.sum(), (rho[:, None] * u).sum(axis=0)
    o.lbm_step(25)
    rho, u = o.lbm_macro()
    assert rho.sum() == pytest.approx(M0, rel=1e-14)
    assert np.abs((rho[:, None] * u).sum(axis=0) - P0).max() < 1e-13 * nodes
    F = np.array([1e-4, -2e-4, 3e-4])
    o = Oracle(fluid(n, body=F, rho0=rho0, u0=u0))
    rho, u = o.lbm_macro()
    P0 = (rho[:, None] * u).sum(axis=0)
    o.lbm_step(10)
    rho, u = o.lbm_macro()
    assert np.abs((rho[:, None] * u).sum(axis=0) - P0 - 10 * F * nodes).max() < 1e-12 * nodes


def _shear_decay_rate(L, tau):
    n = (L, 2, 2)
    nodes = L * 4
    xs = np.arange(nodes) % L
    u0 = np.zeros((nodes, 3))
    u0[:, 1] = 1e-4 * np.sin(2 * math.pi * xs / L)       # u_y(x)
    o = Oracle(fluid(n, tau=tau, u0=u0))
    amps, ts = [], []
    for t in range(0, 400, 20):
        rho, u = o.lbm_macro()
        amps.append(2 * np.mean(u[:, 1] * np.sin(2 * math.pi * xs / L)))
        ts.append(t)
        o.lbm_step(20)
    return -np.polyfit(ts, np.log(amps), 1)[0]


def test_shear_wave_decays_at_the_bgk_viscosity():
    tau = 0.8
    nu = (tau - 0.5) / 3
    errs = []
    for L in (16, 32):
        k = 2 * math.pi / L
        errs.append(abs(_shear_decay_rate(L, tau) / (nu * k * k) - 1))
    assert errs[1] < 2e-3, errs
    assert 3.0 < errs[0] / errs[1] < 5.0, errs                 # second order in k


def _kolmogorov(L, tau, F0=1e-6, steps=6000):
    n = (2, 2, L)
    nodes = 4 * L
    zs = np.arange(nodes) // 4
    s = fluid(n, tau=tau)
    o = Oracle(s)
    # a sinusoidal body force needs a per-node force: use the reaction field
    o.lbm.body_force[:] = [0.0, 0.0, 0.0]
    Fx = F0 * np.sin(2 * math.pi * zs / L)
    ff = o._keep["l_F"].reshape(3, -1)
    for _ in range(steps):
        ff[0, :] = Fx
        o.lbm_step(1)
    ff[0, :] = Fx          # the half-step velocity of the next step's force
    rho, u = o.lbm_macro()
    ux = u[:, 0] + 0.5 * Fx / rho
    return 2 * np.mean(ux * np.sin(2 * math.pi * zs / L))


def test_kolmogorov_flow_with_guo_forcing():
    tau, F0 = 0.7, 1e-6
    nu = (tau - 0.5) / 3
    errs = []
    for L in (16, 32):
        k = 2 * math.pi / L
        errs.append(abs(_kolmogorov(L, tau, F0, steps=int(12 / (nu * k * k))) / (F0 / (nu * k * k)) - 1))
    # second order in k: about 0.14 k^2 at tau = 0.7
    assert errs[1] < 1e-2, errs
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_peskin_four_point_delta():
    for r in np.random.default_rng(1).uniform(0, 1, 20):
        j = np.arange(-3, 4)
        ph = np.array([ibm_phi(r - jj) for jj in j])
        assert ph.sum() == pytest.approx(1.0, abs=1e-15)
        assert ((r - j) * ph).sum() == pytest.approx(0.0, abs=1e-15)
        assert (ph * ph).sum() == pytest.approx(3 / 8, abs=1e-15)
        assert np.count_nonzero(ph > 0) <= 4
    assert ibm_phi(2.0) == 0.0 and ibm_phi(0.0) == 0.5
    assert ibm_phi(1.0 - 1e-12) == pytest.approx(ibm_phi(1.0 + 1e-12), abs=1e-11)


def test_penalty_relaxation_within_a_cycle():
    """A particle moving at v0 through fluid at rest: within the first cycle
    the interpolated fluid velocity stays 0, so m dv/dt = -kappa v with
    kappa = m / dt_LBM: v(1) = v0 e^-1, to first order in the DEM step."""
    errs = []
    for n_sub in (20, 40):
        s = fluid((16, 16, 16), n_sub=n_sub, particles=[[8.3, 7.6, 8.1]], velocities=[[1e-3, -2e-3, 0.5e-3]],
                  masses=[2.0], coupled=np.ones(1, np.uint8))
        o = Oracle(s)
        o.run(n_sub)          # one cycle (the LBM step at its end does not touch v)
        v = o.state()[2][0]
        errs.append(np.abs(v - np.array([1e-3, -2e-3, 0.5e-3]) * math.exp(-1)).max() / 2e-3)
    assert errs[0] < 0.03, errs
    assert 1.6 < errs[0] / errs[1] < 2.6, errs


def test_spread_reaction_sums_to_the_penalty_force():
    """Each step's force evaluation spreads -F_p / n_sub: after each step the
    lattice force field grows by exactly minus the evaluation's penalty
    forces over n_sub (partition of unity), and the LBM step at the end of
    the cycle adds the whole field to the fluid momentum."""
    n_sub = 4
    rng = np.random.default_rng(7)
    xs = rng.uniform(2, 10, (5, 3))
    s = fluid((12, 12, 12), n_sub=n_sub, particles=xs, velocities=rng.standard_normal((5, 3)) * 1e-3,
              masses=rng.uniform(0.5, 2, 5), coupled=np.ones(5, np.uint8))
    o = Oracle(s)
    expect = np.zeros(3)
    for _ in range(n_sub - 1):
        o.run(1)
        expect -= o.f.reshape(-1, 3).sum(axis=0) / n_sub   # only penalty forces act
        assert o.lbm_force_field().sum(axis=1) == pytest.approx(expect, rel=1e-12, abs=1e-20)
    rho, u = o.lbm_macro()
    P_before = (rho[:, None] * u).sum(axis=0)
    o.run(1)                                   # last evaluation of the cycle + LBM step
    expect -= o.f.reshape(-1, 3).sum(axis=0) / n_sub
    rho, u = o.lbm_macro()
    P_after = (rho[:, None] * u).sum(axis=0)
    assert np.abs(o.lbm_force_field()).max() == 0.0   # consumed by the LBM step
    assert P_after - P_before == pytest.approx(expect, rel=1e-10, abs=1e-20)


def test_momentum_balance_over_cycles():
    """Particles coupled to a fluid at rest, no other forces: the particles'
    half-step momentum plus the fluid momentum stays constant over whole
    cycles to rounding (the particles gain sum_k F_p^k dt, the fluid
    receives sum_k -F_p^k / n_sub at each LBM step)."""
    n_sub = 5
    rng = np.random.default_rng(11)
    xs = rng.uniform(3, 13, (6, 3))
    m = rng.uniform(0.5, 2, 6)
    v0 = rng.standard_normal((6, 3)) * 1e-3
    s = fluid((16, 16, 16), n_sub=n_sub, particles=xs, velocities=v0, masses=m, coupled=np.ones(6, np.uint8))
    o = Oracle(s)
    o.forces_valid = False

    def total(o):
        rho, u = o.lbm_macro()
        # half-step particle momentum: v^{n+1/2} = v^n + dt/2 F^n / m
        vh = o.state()[2] + 0.5 * s.dt * o.f.reshape(-1, 3) / m[:, None]
        return (m[:, None] * vh).sum(axis=0) + (rho[:, None] * u).sum(axis=0)

    o.run(n_sub)
    P1 = total(o)
    o.run(3 * n_sub)
    P2 = total(o)
    assert np.abs(P2 - P1).max() < 1e-12 * max(np.abs(m[:, None] * v0).sum(), 1e-30) * 10, (P1, P2)


def test_guo_forcing_is_galilean_invariant():
    """The forced Kolmogorov flow on a uniform background flow U_b along the
    force is the same flow shifted by U_b: its amplitude error equals the one
    without background to 1e-6 (relative) and the mean velocity stays U_b.
    This needs the second-order terms of Guo's source, which carry u.F."""
    L, tau, F0 = 32, 0.7, 1e-5
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / L
    steps = int(12 / (nu * k * k))
    res = []
    for Ub in (0.0, 0.1):
        n = (2, 2, L)
        nodes = 4 * L
        zs = np.arange(nodes) // 4
        u0 = np.zeros((nodes, 3))
        u0[:, 0] = Ub
        o = Oracle(fluid(n, tau=tau, u0=u0))
        Fx = F0 * np.sin(2 * math.pi * zs / L)
        ff = o._keep["l_F"].reshape(3, -1)
        for _ in range(steps):
            ff[0, :] = Fx
            o.lbm_step(1)
        ff[0, :] = Fx
        rho, u = o.lbm_macro()
        ux = u[:, 0] + 0.5 * Fx / rho
        res.append((2 * np.mean(ux * np.sin(2 * math.pi * zs / L)), np.mean(u[:, 0])))
    assert res[1][0] == pytest.approx(res[0][0], rel=1e-6), res
    assert res[1][1] == pytest.approx(0.1, rel=1e-12), res


def test_macroscopic_velocity_includes_half_the_force():
    """From rest under a uniform force, sum f e = n F after n steps, and the
    macroscopic momentum is rho u = sum f e + F/2 = (n + 1/2) F per node."""
    F = np.array([2e-4, -1e-4, 3e-4])
    o = Oracle(fluid((4, 4, 4), body=F))
    o.lbm_step(7)
    rho, u = o.lbm_macro()
    assert (rho[:, None] * u) == pytest.approx(np.tile(7.5 * F, (64, 1)), rel=1e-12)


def test_fluid_velocity_is_interpolated_once_per_cycle():
    """A particle crossing a linear shear flow u_x = g z during one cycle
    feels the fluid velocity interpolated at the cycle's first force
    evaluation (the four-point delta reproduces linear fields exactly):
    v_x(1) = U0 + (v_x0 - U0) e^-1 with U0 = g z(first evaluation), to
    first order in the DEM step."""
    g, L = 1e-3, 16
    nodes = L ** 3
    zs = np.arange(nodes) // (L * L)
    u0 = np.zeros((nodes, 3))
    u0[:, 0] = g * zs
    errs = []
    for n_sub in (20, 40):
        x0 = np.array([7.3, 8.6, 6.2])
        v0 = np.array([0.0, 0.0, 0.8])          # crosses 0.8 lattice units in z
        s = fluid((L, L, L), n_sub=n_sub, u0=u0, particles=[x0], velocities=[v0], masses=[1.5],
                  coupled=np.ones(1, np.uint8))
        o = Oracle(s)
        o.run(n_sub)
        vx = o.state()[2][0][0]
        z1 = x0[2] + v0[2] / n_sub              # position of the first force evaluation
        U0 = g * z1
        errs.append(abs(vx - (U0 + (0.0 - U0) * math.exp(-1))) / U0)
    assert errs[0] < 0.02, errs
    assert 1.6 < errs[0] / errs[1] < 2.6, errs
