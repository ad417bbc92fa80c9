"""Pins of the oracle's magnetic terms (Methods, "Magnetic interactions";
main text "Magnetized beams": the dipole rotates with the particle)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _util import qexp, qmul, qrot_matrix, random_quat


def loose_particles(x, m_space, c=1.0, B=(0, 0, 0), gradB=None, dipole_mode=1, q=None,
                    rods=None):
    """Unbonded particles (one per rod unless rods is given) carrying dipoles."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if q is None:
        q = np.tile([1.0, 0, 0, 0], (n, 1))
    # body dipole so that q m_body q* = m_space
    m_body = np.array([qrot_matrix(qi).T @ mi for qi, mi in zip(q, np.asarray(m_space, float))])
    offs = np.arange(n + 1, dtype=np.int64) if rods is None else np.asarray(rods, dtype=np.int64)
    R = len(offs) - 1
    s = W.RodSystem(name="loose", rod_offset=offs, x=x.copy(), q=np.array(q, float), v=np.zeros((n, 3)),
                    omega=np.zeros((n, 3)), mass=np.ones(n), radius=np.full(n, 0.5), m_body=m_body,
                    clamped=np.zeros(n, np.uint8), x_rest=x.copy(), q_rest=np.array(q, float),
                    E=np.ones(R), nu=np.full(R, 0.3), d=np.ones(R), B=np.array(B, float),
                    mu0_over_4pi=c, dipole_mode=dipole_mode, damping=0.0)
    if gradB is not None:
        s.gradB = np.asarray(gradB, float)
    return s


@pytest.mark.parametrize("r,mu,c", [(1.0, 1.0, 1.0), (2.5, 0.7, 3.0)])
def test_coaxial_head_to_tail_attraction(r, mu, c):
    """Coaxial dipoles attract with 6 c m^2 / r^4; no torque."""
    s = loose_particles([[0, 0, 0], [0, 0, r]], [[0, 0, mu], [0, 0, mu]], c=c)
    f, t = Oracle(s).forces()
    assert f[1, 2] == pytest.approx(-6 * c * mu * mu / r ** 4, rel=1e-14)
    assert f[0, 2] == pytest.approx(6 * c * mu * mu / r ** 4, rel=1e-14)
    assert np.abs(f[:, :2]).max() == 0.0 and np.abs(t).max() == 0.0


@pytest.mark.parametrize("r,mu", [(1.0, 1.0), (1.7, 2.0)])
def test_side_by_side_repulsion(r, mu):
    """Parallel dipoles side by side repel with 3 c m^2 / r^4; no torque."""
    s = loose_particles([[0, 0, 0], [r, 0, 0]], [[0, 0, mu], [0, 0, mu]])
    f, t = Oracle(s).forces()
    assert f[1, 0] == pytest.approx(3 * mu * mu / r ** 4, rel=1e-14)
    assert np.abs(t).max() == 0.0


def test_perpendicular_pair_torque_closed_form():
    """m_i = x at the origin, m_j = z at r x: B_j(x_i) = -c m_j / r^3, so
    tau_i = m_i x B_j = c/r^3 y."""
    r = 1.3
    s = loose_particles([[0, 0, 0], [r, 0, 0]], [[1, 0, 0], [0, 0, 1]])
    f, t = Oracle(s).forces()
    assert np.allclose(t[0], [0, 1 / r ** 3, 0], rtol=1e-14)


def _random_cloud(rng, n=6):
    x = rng.uniform(-2, 2, (n, 3))
    x += 3 * np.arange(n)[:, None] * np.array([1.0, 0.3, 0.1])
    m = rng.standard_normal((n, 3))
    q = np.array([random_quat(rng) for _ in range(n)])
    return x, m, q


def test_dipole_force_and_torque_are_energy_gradients():
    """F_i = -dU/dx_i and tau_i = -dU/dphi_i for U = sum_{i<j} U_ij: the
    dipole-dipole and Zeeman terms are exact gradients (unlike the bonds)."""
    rng = np.random.default_rng(11)
    x, m, q = _random_cloud(rng)
    G = 0.05 * rng.standard_normal((3, 3))
    s = loose_particles(x, m, c=1.7, B=rng.standard_normal(3), gradB=G, q=q)
    o = Oracle(s)
    f, t, e = o.forces(want_energy=True)
    n = len(x)
    h = 1e-6

    def U(xx, qq):
        e = o.forces(x=xx, q=qq, want_energy=True)[2]
        return e[1] + e[2]

    for i in range(n):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (U(xp, q) - U(xm, q)) / (2 * h)
            assert -g == pytest.approx(f[i, a], rel=1e-6, abs=1e-8)
            inc = np.zeros(3)
            inc[a] = h
            qp, qm = q.copy(), q.copy()
            qp[i] = qmul(qexp(inc), q[i])
            qm[i] = qmul(qexp(-inc), q[i])
            g = (U(x, qp) - U(x, qm)) / (2 * h)
            assert -g == pytest.approx(t[i, a], rel=1e-6, abs=1e-8)


def test_dipole_momentum_conservation():
    """Isolated dipoles: sum F = 0 and sum (x x F + tau) = 0."""
    rng = np.random.default_rng(12)
    x, m, q = _random_cloud(rng, n=9)
    o = Oracle(loose_particles(x, m, q=q))
    f, t = o.forces()
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-13 * scale * len(x)
    L = np.cross(x, f).sum(0) + t.sum(0)
    assert np.abs(L).max() < 1e-12 * scale * np.abs(x).max() * len(x)


def test_dipole_energy_pair_sum():
    """E_dipole counts each pair once: U_12 for two dipoles (closed form)."""
    r = 1.4
    s = loose_particles([[0, 0, 0], [0, 0, r]], [[0, 0, 1.0], [0, 0, 1.0]])
    e = Oracle(s).energy()
    assert e[2] == pytest.approx((1 - 3) / r ** 3, rel=1e-14)


def test_per_rod_mode_excludes_other_rods():
    """dipole mode 2 = all pairs within each rod only: equal to the rods
    evaluated one at a time."""
    rng = np.random.default_rng(13)
    x, m, q = _random_cloud(rng, n=7)
    rods = [0, 3, 7]
    both = Oracle(loose_particles(x, m, q=q, rods=rods, dipole_mode=2)).forces()
    a = Oracle(loose_particles(x[:3], m[:3], q=q[:3], rods=[0, 3], dipole_mode=1)).forces()
    b = Oracle(loose_particles(x[3:], m[3:], q=q[3:], rods=[0, 4], dipole_mode=1)).forces()
    assert np.allclose(both[0], np.vstack([a[0], b[0]]), rtol=1e-14, atol=0)
    assert np.allclose(both[1], np.vstack([a[1], b[1]]), rtol=1e-14, atol=0)


def test_zeeman_uniform_torque():
    """tau = m x B; for the straight-rod workload (m = x, B = 0.5 (cos 30,
    sin 30, 0)) each unperturbed particle feels tau_z = 0.5 sin 30 = 0.25."""
    s = W.straight_rod(pos_sigma=0.0, rot_max=0.0, dipole_mode=W.DIPOLE_OFF)
    f, t = Oracle(s).forces()
    assert np.allclose(t[:, 2], 0.25, rtol=1e-14)
    assert np.abs(t[:, :2]).max() < 1e-15 and np.abs(f).max() < 1e-9


def test_zeeman_constant_gradient_gives_uniform_force():
    """B = G x: every dipole m feels the same force G^T m, independent of x."""
    rng = np.random.default_rng(14)
    G = rng.standard_normal((3, 3))
    m = np.tile(rng.standard_normal(3), (5, 1))
    x = rng.uniform(-5, 5, (5, 3)) + 10 * np.arange(5)[:, None]
    f, t = Oracle(loose_particles(x, m, gradB=G, dipole_mode=0)).forces()
    assert np.allclose(f, np.tile(G.T @ m[0], (5, 1)), rtol=1e-14)


def test_rotating_field():
    """B(t) = amp (cos wt e1 + sin wt e2): torque on m = z at a known phase."""
    s = loose_particles([[0, 0, 0]], [[0, 0, 1.0]], dipole_mode=0)
    s.Brot_amp, s.Brot_omega = 0.5, 2 * math.pi / 2000.0
    o = Oracle(s)
    t_now = 250.0  # quarter period / 2 -> phase pi/4
    f, tau = o.forces(t=t_now)
    B = 0.5 * np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0])
    assert np.allclose(tau[0], np.cross([0, 0, 1.0], B), rtol=1e-14)


def test_dipole_rotates_with_particle():
    """m = R m~: rotating a particle by q rotates its dipole (and field
    torque) by q."""
    rng = np.random.default_rng(15)
    q = random_quat(rng)
    mb = rng.standard_normal(3)
    s = loose_particles([[0, 0, 0]], [qrot_matrix(q) @ mb], q=[q], dipole_mode=0, B=[0.0, 0.0, 0.0])
    o = Oracle(s)
    _, _, m = o.forces(want_m=True)
    assert np.allclose(m[0], qrot_matrix(q) @ mb, rtol=1e-14)
