"""System-level pins of the oracle: spring constants built from (E, nu, d)
and rest states with arbitrary orientations (main text: spring constants
after Eq. bpm-vector; the q^i = 1 convention of the bond definition)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _util import qexp, qmul, qrot_matrix, random_quat


def _dimer(E, nu, d, L, q_rest=None):
    x = np.array([[0.0, 0, 0], [L, 0, 0]])
    qr = np.tile([1.0, 0, 0, 0], (2, 1)) if q_rest is None else np.asarray(q_rest, float)
    return W.RodSystem(name="dimer", rod_offset=np.array([0, 2], dtype=np.int64), x=x.copy(), q=qr.copy(),
                       v=np.zeros((2, 3)), omega=np.zeros((2, 3)), mass=np.ones(2), radius=np.full(2, 0.5),
                       m_body=np.zeros((2, 3)), clamped=np.zeros(2, np.uint8), x_rest=x.copy(),
                       q_rest=qr.copy(), E=np.array([E]), nu=np.array([nu]), d=np.array([d]),
                       dipole_mode=0, damping=0.0)


@pytest.mark.parametrize("E,nu,d,L", [(1e4, 0.3, 1.0, 1.0), (3e3, 0.45, 0.7, 0.6)])
def test_dimer_stiffness_from_material(E, nu, d, L):
    """Stretch, twist and the two bending modes of a dimer built from
    (E, nu, d): the Euler-Bernoulli element values EA/L, GJ/L, 12EI/L^3 and
    4EI/L / 2EI/L for a cylinder (A = pi d^2/4, I = pi d^4/64, J = pi d^4/32)."""
    o = Oracle(_dimer(E, nu, d, L))
    G = E / (2 * (1 + nu))
    A, I, J = math.pi * d * d / 4, math.pi * d ** 4 / 64, math.pi * d ** 4 / 32
    h = 1e-6
    x0 = o.x.reshape(-1, 3).copy()
    q0 = o.q.reshape(-1, 4).copy()

    def F(dx2=np.zeros(3), dphi1=np.zeros(3)):
        x = x0.copy()
        x[1] += dx2
        q = q0.copy()
        q[0] = qmul(qexp(dphi1), q[0])
        return o.forces(x=x, q=q)

    # axial: d f1_x / d x2_x = EA/L
    kax = (F(dx2=np.array([h, 0, 0]))[0][0, 0] - F(dx2=np.array([-h, 0, 0]))[0][0, 0]) / (2 * h)
    assert kax == pytest.approx(E * A / L, rel=1e-7)
    # transverse: d f1_y / d x2_y = 12 EI / L^3
    ktr = (F(dx2=np.array([0, h, 0]))[0][0, 1] - F(dx2=np.array([0, -h, 0]))[0][0, 1]) / (2 * h)
    assert ktr == pytest.approx(12 * E * I / L ** 3, rel=1e-7)
    # torsion: d tau1_x / d phi1_x = -GJ/L
    ktw = (F(dphi1=np.array([h, 0, 0]))[1][0, 0] - F(dphi1=np.array([-h, 0, 0]))[1][0, 0]) / (2 * h)
    assert ktw == pytest.approx(-G * J / L, rel=1e-7)
    # bending: d tau1_z / d phi1_z = -4EI/L, d tau2_z / d phi1_z = -2EI/L
    fp, fm = F(dphi1=np.array([0, 0, h])), F(dphi1=np.array([0, 0, -h]))
    assert (fp[1][0, 2] - fm[1][0, 2]) / (2 * h) == pytest.approx(-4 * E * I / L, rel=1e-7)
    assert (fp[1][1, 2] - fm[1][1, 2]) / (2 * h) == pytest.approx(-2 * E * I / L, rel=1e-7)


def test_rest_orientations_are_a_gauge():
    """Arbitrary rest orientations: any rigid motion of the rest state is force
    free, and the forces equal those of the same deformation built on q^i = 1."""
    rng = np.random.default_rng(17)
    s = W.random_rods([6, 4], seed=5, with_gradient=False, with_rotating=False)
    s.dipole_mode = 0
    s.B = np.zeros(3)
    s.damping = 0.0
    o = Oracle(s)
    R = random_quat(rng)
    Rm = qrot_matrix(R)
    T = rng.standard_normal(3)
    x_rig = s.x_rest @ Rm.T + T
    q_rig = np.array([qmul(R, qr) for qr in s.q_rest])
    f, t = o.forces(x=x_rig, q=q_rig, v=np.zeros_like(x_rig), w=np.zeros_like(x_rig))
    assert np.abs(f).max() < 1e-9 and np.abs(t).max() < 1e-9
    # same deformation expressed relative to identity rest orientations
    f1, t1 = o.forces()
    s2 = s.copy()
    s2.q_rest = np.tile([1.0, 0, 0, 0], (s.n, 1))
    s2.q = np.array([qmul(q, np.array([qr[0], -qr[1], -qr[2], -qr[3]])) for q, qr in zip(s.q, s.q_rest)])
    f2, t2 = Oracle(s2).forces()
    assert np.allclose(f1, f2, rtol=0, atol=1e-9 * np.abs(f1).max())
    assert np.allclose(t1, t2, rtol=0, atol=1e-9 * np.abs(t1).max())


def test_subset_of_independent_rods_evolves_as_in_the_whole_batch():
    """Rods without mutual interaction (per-rod dipoles): a subset cut out of
    the batch follows the same trajectory as inside the batch, bit for bit,
    which lets the GPU's full batch be checked on a few rods."""
    s = W.batched_rods(9, 16, 60, precision=W.PRECISION_FP64)
    rods = [1, 4, 8]
    sub = W.subset_rods(s, rods)
    a = Oracle(s)
    a.run(20)
    b = Oracle(sub)
    b.run(20)
    xa = a.state()[0]
    offs = s.rod_offset
    idx = np.concatenate([np.arange(offs[r], offs[r + 1]) for r in rods])
    assert np.array_equal(xa[idx], b.state()[0])
