"""Pins of the oracle's time integration (SI "Equations of motion": velocity
Verlet for x, v, omega; Richardson extrapolation for q with renormalisation
after every substep) and of global damping (Methods, "Damping")."""
import math

import numpy as np
import pytest

from oracle import Oracle, richardson
from paper_2603_27279_gb300 import workloads as W

from _util import qexp, qmul


def _free_particle(v0=(0, 0, 0), w0=(0, 0, 0), q0=(1, 0, 0, 0), damping=0.0, dt=1e-2, mass=1.0):
    x = np.zeros((1, 3))
    q = np.array([q0], dtype=float)
    return W.RodSystem(name="free", rod_offset=np.array([0, 1], dtype=np.int64), x=x, q=q,
                       v=np.array([v0], float), omega=np.array([w0], float), mass=np.array([mass]),
                       radius=np.array([0.5]), m_body=np.zeros((1, 3)), clamped=np.zeros(1, np.uint8),
                       x_rest=x.copy(), q_rest=q.copy(), E=np.ones(1), nu=np.full(1, 0.3),
                       d=np.ones(1), dipole_mode=0, damping=damping, dt=dt)


def _two_particles(K, stretch=0.0, twist=0.0, dt=1e-3):
    x = np.array([[0.0, 0, 0], [1.0 + stretch, 0, 0]])
    x_rest = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    q = np.array([[1.0, 0, 0, 0], qexp([twist, 0, 0])])
    s = W.RodSystem(name="dimer", rod_offset=np.array([0, 2], dtype=np.int64), x=x, q=q,
                    v=np.zeros((2, 3)), omega=np.zeros((2, 3)), mass=np.ones(2), radius=np.full(2, 0.5),
                    m_body=np.zeros((2, 3)), clamped=np.zeros(2, np.uint8), x_rest=x_rest,
                    q_rest=np.tile([1.0, 0, 0, 0], (2, 1)), E=np.ones(1), nu=np.full(1, 0.3), d=np.ones(1),
                    dipole_mode=0, damping=0.0, dt=dt)
    o = Oracle(s)
    o.bond_K[:] = K
    return o


def test_richardson_rotor_is_second_order():
    """Free rotor with constant omega: q(T) -> exp(omega T / 2) q0 with an
    error quadratic in dt (the SI's claim for the extrapolated update)."""
    w = np.array([0.3, -1.2, 2.0])
    q0 = qexp([0.2, 0.1, -0.4])
    exact = qmul(qexp(w * 1.0), q0)
    errs = []
    for dt in (1e-2, 5e-3, 2.5e-3):
        o = Oracle(_free_particle(w0=w, q0=q0, dt=dt))
        o.run(int(round(1.0 / dt)))
        errs.append(np.linalg.norm(o.q - exact))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)
    assert errs[2] < 2e-6


def test_richardson_rotor_error_constant():
    """For a fixed axis the extrapolated update turns by w dt + (w dt)^3/24
    per step (single Euler step: -(w dt)^3/12, two half steps: -(w dt)^3/48),
    so after time T the phase leads by w^3 T dt^2 / 24."""
    w = 2.0
    dt = 1e-2
    T = 1.0
    o = Oracle(_free_particle(w0=(0.0, 0.0, w), dt=dt))
    o.run(int(round(T / dt)))
    ang = 2 * math.atan2(o.q[3], o.q[0])
    lead = ang - w * T
    assert lead == pytest.approx(w ** 3 * T * dt ** 2 / 24, rel=0.02)


def test_richardson_substeps_are_normalised():
    q = richardson(qexp([0.1, 0.2, 0.3]), [5.0, -3.0, 2.0], 0.05)
    assert np.linalg.norm(q) == pytest.approx(1.0, abs=1e-15)


def test_free_translation_exact():
    o = Oracle(_free_particle(v0=(1.0, -2.0, 0.5), dt=0.01))
    o.run(100)
    assert np.allclose(o.x, [1.0, -2.0, 0.5], rtol=1e-13)


@pytest.mark.parametrize("mode", ["stretch", "twist"])
def test_velocity_verlet_energy_error_is_second_order(mode):
    """A harmonic dimer (pure radial or pure twist spring, where the force is
    an exact gradient): the energy error of velocity Verlet scales as dt^2."""
    K = np.array([100.0, 0.0, 0.0, 0.0]) if mode == "stretch" else np.array([0.0, 0.0, 3.0, 0.0])
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        o = _two_particles(K, stretch=0.05 if mode == "stretch" else 0.0,
                           twist=0.3 if mode == "twist" else 0.0, dt=dt)
        e0 = o.energy()
        H0 = e0[0] + e0[3] + e0[4]
        worst = 0.0
        for _ in range(int(round(0.5 / dt))):
            o.run(1)
            e = o.energy()
            # energy at integer steps: velocities are full-step after run()
            worst = max(worst, abs(e[0] + e[3] + e[4] - H0))
        errs.append(worst / H0)
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.25)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.25)


def test_global_damping_uses_half_step_velocity():
    """Free particle with viscous damping g: v(T) -> v0 exp(-g T / m).  With
    the damping force evaluated from the half-step velocity (reading R8) the
    scheme is first order: halving dt halves the error."""
    g, m, v0 = 0.8, 2.0, np.array([1.0, 0.5, -0.25])
    exact = v0 * math.exp(-g * 1.0 / m)
    errs = []
    for dt in (1e-2, 5e-3, 2.5e-3):
        o = Oracle(_free_particle(v0=v0, damping=g, dt=dt, mass=m))
        o.run(int(round(1.0 / dt)))
        errs.append(np.linalg.norm(o.v - exact))
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.1)


def test_clamped_particles_do_not_move():
    s = W.random_rods([7, 5], seed=3)
    o = Oracle(s)
    x0, q0 = o.x.copy(), o.q.copy()
    o.run(25)
    cl = np.where(s.clamped == 1)[0]
    assert np.array_equal(o.x.reshape(-1, 3)[cl], x0.reshape(-1, 3)[cl])
    assert np.array_equal(o.q.reshape(-1, 4)[cl], q0.reshape(-1, 4)[cl])
    free = np.where(s.clamped == 0)[0]
    assert np.abs(o.x.reshape(-1, 3)[free] - x0.reshape(-1, 3)[free]).max() > 0
