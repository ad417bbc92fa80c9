"""The CUDA bond kernel against closed-form bond states, without the oracle.

Two-particle rods whose relative rotation combines a finite bend with a
finite twist (SI "Symmetric rotational decomposition", bend before twist;
main text Eqs. bpm-tb and bpm-tt).  The expected torques come from the
paper's definitions composed with scipy's rotations, as in the oracle's own
pin (tests/test_oracle_bond.py), so the kernel's composition order is checked
directly and not only through parity with the oracle.
"""
import math

import numpy as np
import pytest

from paper_2603_27279_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


CASES = [(a, b, p, o) for (a, b, p) in ((0.9, 0.7, 0.3), (-0.6, 1.0, 2.2), (0.35, 0.25, -1.1), (1.0, 0.5, 4.0),
                                        (-0.8, 0.9, 0.0), (1e-3, 2e-3, 0.7), (0.4, 1e-4, 1.3))
         for o in ("bend_first", "twist_first")]


def _expected(alpha, beta, phi, order, Rot):
    z = np.array([0.0, 0.0, 1.0])
    tw = Rot.from_rotvec(alpha * z)
    bd = Rot.from_rotvec(beta * np.array([math.cos(phi), math.sin(phi), 0.0]))
    u = tw * bd if order == "bend_first" else bd * tw
    t2 = tw
    b2 = t2.inv() * u
    b1 = t2 * b2.inv() * t2.inv()
    return u, 2.0 * alpha, (b2 * b1.inv()).as_rotvec()


def test_combined_bend_and_twist_on_the_gpu(bpm):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    n_rods = len(CASES)
    Lr, E, nu, d = 1.1, 1e4, 0.3, 1.0
    x = np.zeros((2 * n_rods, 3))
    q = np.zeros((2 * n_rods, 4))
    x_rest = np.zeros((2 * n_rods, 3))
    expect_t = np.zeros((2 * n_rods, 3))
    G = E / (2 * (1 + nu))
    Kt = G * math.pi * d ** 4 / 32 / Lr
    Kb = E * math.pi * d ** 4 / 64 / Lr
    z = np.array([0.0, 0.0, 1.0])
    for r, (alpha, beta, phi, order) in enumerate(CASES):
        u, psi, theta_b = _expected(alpha, beta, phi, order, Rot)
        base = np.array([10.0 * r, 0.0, 0.0])
        x[2 * r] = base
        x[2 * r + 1] = base + Lr * u.apply(z)
        x_rest[2 * r] = base
        x_rest[2 * r + 1] = base + Lr * z
        q[2 * r] = [1.0, 0.0, 0.0, 0.0]
        xyzw = (u * u).as_quat()
        q[2 * r + 1] = [xyzw[3], xyzw[0], xyzw[1], xyzw[2]]
        tau = u.apply(Kb * theta_b + Kt * psi * z)
        expect_t[2 * r] = tau
        expect_t[2 * r + 1] = -tau
    q_rest = np.tile([1.0, 0.0, 0.0, 0.0], (2 * n_rods, 1))
    sysm = W.RodSystem(
        name="bend_twist_pins", rod_offset=np.arange(0, 2 * n_rods + 1, 2, dtype=np.int64), x=x, q=q,
        v=np.zeros_like(x), omega=np.zeros_like(x), mass=np.ones(2 * n_rods), radius=np.full(2 * n_rods, 0.5),
        m_body=np.zeros_like(x), clamped=np.zeros(2 * n_rods, np.uint8), x_rest=x_rest, q_rest=q_rest,
        E=np.full(n_rods, E), nu=np.full(n_rods, nu), d=np.full(n_rods, d), dipole_mode=W.DIPOLE_OFF)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        f, t = sim.forces()
    scale = max(Kt, Kb)
    assert np.abs(f).max() < 1e-11 * scale
    err = np.abs(t - expect_t).max(axis=1) / np.maximum(np.linalg.norm(expect_t, axis=1), 1e-300)
    assert err.max() < 1e-11, err
