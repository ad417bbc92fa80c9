"""Pins of the oracle's bond model against what the paper and mechanics fix.

Paper passages: main text "Bonded-particle model for elastic rods" (Eqs.
bpm-fr .. bpm-vector, total-energy) and SI "Symmetric rotational
decomposition", "Deriving the spring constants" (Eq. beam-stiffness-matrix),
"Elastic energy".
"""
import math

import numpy as np
import pytest

from oracle import align_z, bond, quat_mul, rotate

from _util import default_K, qexp, qmul, qrot_matrix, random_quat, read_golden

K0 = default_K()


def _random_bond(rng, amp=0.2):
    ri = rng.standard_normal(3)
    ri *= rng.uniform(0.7, 1.3) / np.linalg.norm(ri)
    x1 = rng.standard_normal(3)
    x2 = x1 + ri + amp * rng.standard_normal(3)
    q1 = qexp(amp * rng.standard_normal(3))
    q2 = qexp(amp * rng.standard_normal(3))
    return x1, x2, q1, q2, ri


def test_quaternion_conventions():
    i = np.array([0.0, 1, 0, 0])
    j = np.array([0.0, 0, 1, 0])
    k = np.array([0.0, 0, 0, 1])
    assert np.allclose(quat_mul(i, j), k) and np.allclose(quat_mul(j, i), -k)
    # q v q* with q a +90 degree turn about z maps x onto y
    qz = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    assert np.allclose(rotate(qz, [1.0, 0, 0]), [0, 1, 0], atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(5):
        q = random_quat(rng)
        v = rng.standard_normal(3)
        assert np.allclose(rotate(q, v), qrot_matrix(q) @ v, atol=1e-14)


def test_rigid_motion_of_rest_state_is_force_free():
    """Zero force and torque in any rigidly translated and rotated rest state."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        ri = rng.standard_normal(3)
        R = random_quat(rng)
        T = rng.standard_normal(3) * 10
        x1 = T
        x2 = T + rotate(R, ri)
        f1, t1, f2, t2, U, _ = bond(x1, x2, R, R, ri, K0)
        scale = np.abs(K0).max() * np.linalg.norm(ri)
        for v in (f1, t1, f2, t2):
            assert np.abs(v).max() < 1e-12 * scale
        assert abs(U) < 1e-20 * scale


def test_covariance_under_global_rotation():
    rng = np.random.default_rng(2)
    for _ in range(20):
        x1, x2, q1, q2, ri = _random_bond(rng)
        R = random_quat(rng)
        Rm = qrot_matrix(R)
        a = bond(x1, x2, q1, q2, ri, K0)
        b = bond(Rm @ x1, Rm @ x2, qmul(R, q1), qmul(R, q2), ri, K0)
        for u, v in zip(a[:4], b[:4]):
            assert np.allclose(Rm @ u, v, rtol=0, atol=1e-10 * np.abs(K0).max())
        assert b[4] == pytest.approx(a[4], rel=1e-12)


def test_exchange_symmetry():
    """Swapping particles 1 and 2 gives the same forces (SI: the central frame
    makes the model symmetric under particle exchange)."""
    rng = np.random.default_rng(3)
    for _ in range(30):
        x1, x2, q1, q2, ri = _random_bond(rng, amp=0.3)
        f1, t1, f2, t2, U, _ = bond(x1, x2, q1, q2, ri, K0)
        g1, s1, g2, s2, V, _ = bond(x2, x1, q2, q1, -ri, K0)
        tol = 1e-11 * np.abs(K0).max()
        assert np.allclose(g1, f2, atol=tol) and np.allclose(g2, f1, atol=tol)
        assert np.allclose(s1, t2, atol=tol) and np.allclose(s2, t1, atol=tol)
        assert V == pytest.approx(U, rel=1e-10)


def test_momentum_balance_per_bond():
    """Net force zero exactly; net angular momentum flux zero to rounding."""
    rng = np.random.default_rng(4)
    for _ in range(30):
        x1, x2, q1, q2, ri = _random_bond(rng, amp=0.4)
        f1, t1, f2, t2, U, _ = bond(x1, x2, q1, q2, ri, K0)
        assert np.array_equal(f1 + f2, np.zeros(3))
        L = np.cross(x1, f1) + np.cross(x2, f2) + t1 + t2
        assert np.abs(L).max() < 1e-11 * np.abs(K0).max() * (1 + np.abs(x1).max())


def test_symmetric_rotation_gives_no_shear():
    """Ends rotated by -phi/2 and +phi/2 about any axis: the slerp midpoint is
    the identity, so an unstretched bond has no radial or shear force."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        phi = rng.standard_normal(3)
        phi *= rng.uniform(0.1, 2.5) / np.linalg.norm(phi)
        ri = rng.standard_normal(3)
        f1, t1, f2, t2, U, _ = bond([0, 0, 0], ri, qexp(-phi / 2), qexp(phi / 2), ri, K0)
        assert np.abs(f1).max() < 1e-11 * np.abs(K0).max()


@pytest.mark.parametrize("Phi", [1e-6, 1e-3, 0.4, 1.7, 3.0])
def test_pure_twist(Phi):
    """Twist by Phi about the bond axis: tau_t = K_t Phi (Eq. bpm-tt)."""
    rng = np.random.default_rng(6)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    L = 1.3
    f1, t1, f2, t2, U, d = bond([0, 0, 0], L * n, [1, 0, 0, 0], qexp(Phi * n), L * n, K0)
    assert np.allclose(t1, K0[2] * Phi * n, rtol=1e-12, atol=1e-13 * K0[2])
    assert np.allclose(t2, -K0[2] * Phi * n, rtol=1e-12, atol=1e-13 * K0[2])
    assert np.abs(f1).max() < 1e-12 * K0[0]
    assert U == pytest.approx(0.5 * K0[2] * Phi ** 2, rel=1e-10)
    assert d[1] == pytest.approx(Phi, rel=1e-12)


@pytest.mark.parametrize("alpha", [1e-6, 1e-3, 0.3, 1.2])
def test_pure_planar_bend(alpha):
    """Ends turned by -alpha/2 and +alpha/2 about an axis normal to the bond:
    tau_b = K_b alpha on particle 1, -K_b alpha on particle 2 (Eq. bpm-tb)."""
    rng = np.random.default_rng(7)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    a = rng.standard_normal(3)
    a -= n * (a @ n)
    a /= np.linalg.norm(a)
    f1, t1, f2, t2, U, d = bond([0, 0, 0], n, qexp(-alpha / 2 * a), qexp(alpha / 2 * a), n, K0)
    assert np.allclose(t1, K0[3] * alpha * a, rtol=1e-11, atol=1e-14 * K0[3])
    assert np.allclose(t2, -K0[3] * alpha * a, rtol=1e-11, atol=1e-14 * K0[3])
    assert U == pytest.approx(0.5 * K0[3] * alpha ** 2, rel=1e-10)


def _eb_matrix():
    g = read_golden("eb_beam_stiffness.txt")
    i = g.index("matrix")
    j = g.index("null")
    mat = [[(float(r.split()[2 * c]), int(r.split()[2 * c + 1])) for c in range(4)] for r in g[i + 1:j]]
    null = [[(float(r.split()[2 * c]), int(r.split()[2 * c + 1])) for c in range(4)] for r in g[j + 1:]]
    return mat, null


@pytest.mark.parametrize("E,nu,d,L", [(1e4, 0.3, 1.0, 1.0), (2.1e3, 0.45, 0.6, 0.8)])
def test_linear_stiffness_equals_eb_frame_element(E, nu, d, L):
    """At rest, the bond's linearised force map equals the 3D Euler-Bernoulli
    frame element: axial EA/L, torsion GJ/L, and in both bending planes the
    printed 4x4 matrix (SI Eq. beam-stiffness-matrix), with its null space."""
    K = default_K(E, nu, d, L)
    G = E / (2 * (1 + nu))
    A, I, J = math.pi * d * d / 4, math.pi * d ** 4 / 64, math.pi * d ** 4 / 32
    mat, null = _eb_matrix()
    Kp = np.array([[c * L ** p for (c, p) in row] for row in mat]) * E * I / L ** 3
    # assemble the 12x12 frame stiffness, DOFs (u1, phi1, u2, phi2), bond along x
    Kf = np.zeros((12, 12))
    Kf[np.ix_([0, 6], [0, 6])] = E * A / L * np.array([[1, -1], [-1, 1]])
    Kf[np.ix_([3, 9], [3, 9])] = G * J / L * np.array([[1, -1], [-1, 1]])
    iy = [1, 5, 7, 11]                       # (v1, phi_z1, v2, phi_z2)
    Kf[np.ix_(iy, iy)] = Kp
    iz = [2, 4, 8, 10]                       # (w1, phi_y1, w2, phi_y2), slope = -phi_y
    T = np.diag([1.0, -1.0, 1.0, -1.0])
    Kf[np.ix_(iz, iz)] = T @ Kp @ T
    # central finite differences of the oracle's bond map
    ri = np.array([L, 0.0, 0.0])

    def gen_forces(u):
        x1 = u[0:3]
        x2 = ri + u[6:9]
        f1, t1, f2, t2, _, _ = bond(x1, x2, qexp(u[3:6]), qexp(u[9:12]), ri, K)
        return np.concatenate([f1, t1, f2, t2])

    h = 1e-6
    Jac = np.zeros((12, 12))
    for j in range(12):
        e = np.zeros(12)
        e[j] = h
        Jac[:, j] = (gen_forces(e) - gen_forces(-e)) / (2 * h)
    assert np.allclose(Jac, -Kf, rtol=0, atol=1e-6 * np.abs(Kf).max())
    # the printed null-space vectors give no force in each bending plane
    for vec in null:
        nv = np.array([c * L ** p for (c, p) in vec])
        assert np.abs(Kp @ nv).max() < 1e-12 * np.abs(Kp).max()


def test_m_matches_printed_quaternion():
    """Reading R4 reproduces the printed m (SI Eq. S-quat-h) where the printed
    form is defined, and both branches take z onto r_f[C]."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        r = rng.standard_normal(3)
        x, y, z = r
        rn = np.linalg.norm(r)
        m = align_z(r, 0)
        s = math.sqrt(x * x + y * y)
        printed = np.array([math.sqrt(2) / 2 * math.sqrt(1 + z / rn),
                            -math.sqrt(2) / 2 * math.sqrt(1 - z / rn) * y / s,
                            math.sqrt(2) / 2 * math.sqrt(1 - z / rn) * x / s, 0.0])
        assert np.allclose(m, printed, atol=1e-12)
        for branch in (0, 1, -1):
            mb = align_z(r, branch)
            assert np.linalg.norm(mb) == pytest.approx(1.0, abs=1e-15)
            assert np.allclose(rotate(mb, [0, 0, 1.0]), r / rn, atol=1e-12)
    # the automatic choice is regular at r = -z
    assert np.allclose(rotate(align_z([0, 0, -2.0]), [0, 0, 1.0]), [0, 0, -1], atol=1e-15)


def test_m_gauge_does_not_change_forces():
    """Any m taking z onto r_f[C] gives the same forces (R4's justification)."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        x1, x2, q1, q2, ri = _random_bond(rng, amp=0.3)
        a = bond(x1, x2, q1, q2, ri, K0, m_branch=0)
        b = bond(x1, x2, q1, q2, ri, K0, m_branch=1)
        for u, v in zip(a[:4], b[:4]):
            assert np.allclose(u, v, rtol=0, atol=1e-11 * np.abs(K0).max())


def test_forces_are_gradients_only_to_leading_order():
    """The paper states the forces are not exact gradients of Eq.
    total-energy; the mismatch must vanish linearly with the deformation."""
    rng = np.random.default_rng(10)
    ddir = rng.standard_normal(12)
    ddir /= np.linalg.norm(ddir)
    ri = np.array([1.0, 0.0, 0.0])

    def state(u):
        return u[0:3], ri + u[6:9], qexp(u[3:6]), qexp(u[9:12])

    def energy(u):
        return bond(*state(u), ri, K0)[4]

    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        u0 = eps * ddir
        f1, t1, f2, t2, _, _ = bond(*state(u0), ri, K0)
        gen = np.concatenate([f1, t1, f2, t2])
        grad = np.zeros(12)
        h = 1e-6 * eps
        for j in range(12):
            e = np.zeros(12)
            e[j] = h
            up, um = u0 + e, u0 - e
            # rotation DOFs: compose the increment in space, q <- exp(dphi) q
            if j in (3, 4, 5, 9, 10, 11):
                def comp(s):
                    x1, x2, q1, q2 = state(u0)
                    inc = np.zeros(3)
                    inc[j % 3] = s
                    if j < 6:
                        q1 = qmul(qexp(inc), q1)
                    else:
                        q2 = qmul(qexp(inc), q2)
                    return bond(x1, x2, q1, q2, ri, K0)[4]
                grad[j] = (comp(h) - comp(-h)) / (2 * h)
            else:
                grad[j] = (energy(up) - energy(um)) / (2 * h)
        errs.append(np.linalg.norm(gen + grad) / np.linalg.norm(gen))
    assert errs[2] < 1e-3
    assert 5.0 < errs[0] / errs[1] < 20.0 and 5.0 < errs[1] / errs[2] < 20.0


def test_quaternion_sign_does_not_matter():
    """q and -q are the same rotation: flipping either end's sign (which puts
    q_1 . q_2 < 0) must not change anything (slerp on the shorter arc)."""
    rng = np.random.default_rng(16)
    for _ in range(20):
        x1, x2, q1, q2, ri = _random_bond(rng, amp=0.5)
        a = bond(x1, x2, q1, q2, ri, K0)
        for s1, s2 in ((1, -1), (-1, 1), (-1, -1)):
            b = bond(x1, x2, s1 * q1, s2 * q2, ri, K0)
            for u, v in zip(a[:4], b[:4]):
                assert np.allclose(u, v, rtol=0, atol=1e-11 * np.abs(K0).max())


def _twist_bend_cases():
    """(label, alpha, beta, phi, order): a half rotation u built from a twist
    by alpha about z and a bend by beta about n = (cos phi, sin phi, 0), in
    either composition order, with finite angles up to about 1 rad."""
    cases = []
    for alpha, beta, phi in ((0.9, 0.7, 0.3), (-0.6, 1.0, 2.2), (0.35, 0.25, -1.1), (1.0, 0.5, 4.0),
                             (-0.8, 0.9, 0.0)):
        for order in ("bend_first", "twist_first"):
            cases.append((f"{order}_{alpha}_{beta}_{phi}", alpha, beta, phi, order))
    return cases


@pytest.mark.parametrize("label,alpha,beta,phi,order", _twist_bend_cases())
def test_combined_bend_and_twist_follow_the_bend_before_twist_decomposition(label, alpha, beta, phi, order):
    """Finite bend and twist together (SI "Symmetric rotational
    decomposition": u = t_2 b_2 and u* = t_1 b_1, each a bend followed by a
    twist about z of C', b = b_2 b_1*, t = t_2 t_1*; main text Eqs. bpm-tb and
    bpm-tt).  Particle 1 sits at the identity and particle 2 at u u, so the
    central frame is u itself; particle 2 sits on the z axis of that frame at
    the rest length, so there is no stretch or shear and C' = C.

    The expected values come from the definitions alone, composed with
    scipy's rotations (an implementation independent of the oracle): u's
    bend-before-twist factors are t_2 = twist(alpha) and b_2 = t_2^-1 u (a
    rotation about an axis normal to z in both orders); then t_1 = t_2^-1 and
    b_1 = t_2 b_2^-1 t_2^-1, so psi = 2 alpha and theta b^ is the rotation
    vector of b_2 t_2 b_2 t_2^-1.  The torque on particle 1 is
    u (K_b theta b^ + K_t psi z) and particle 2 gets its negative.  Taking the
    factors in the other order (b_2 = u t_2^-1) keeps psi and |theta| but
    flips the z part of theta b^, which these checks see."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    z = np.array([0.0, 0.0, 1.0])
    n = np.array([math.cos(phi), math.sin(phi), 0.0])
    tw = Rot.from_rotvec(alpha * z)
    bd = Rot.from_rotvec(beta * n)
    u = tw * bd if order == "bend_first" else bd * tw   # scipy: (a * b) applies b first
    # u's own bend-before-twist factors: the twist is the z-rotation whose
    # inverse leaves a rotation about an axis normal to z
    t2 = tw
    b2 = t2.inv() * u
    assert abs(b2.as_rotvec()[2]) < 1e-15
    t1 = t2.inv()
    b1 = t2 * b2.inv() * t2.inv()
    assert abs(b1.as_rotvec()[2]) < 1e-15
    assert np.allclose((t1 * b1).as_quat(), u.inv().as_quat()) or np.allclose((t1 * b1).as_quat(),
                                                                                -u.inv().as_quat())
    psi = 2.0 * alpha
    theta_b = (b2 * b1.inv()).as_rotvec()
    # the state: particle 1 at the identity, particle 2 at u u (scalar-first)
    xyzw = (u * u).as_quat()
    q2 = np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]])
    if q2[0] < 0:
        q2 = -q2
    Lr = 1.1
    x2 = Lr * u.apply(z)
    f1, t1_, f2, t2_, U, d = bond([0, 0, 0], x2, [1, 0, 0, 0], q2, Lr * z, K0)
    assert d[1] == pytest.approx(psi, rel=1e-13, abs=1e-14)
    assert np.allclose(d[2:5], theta_b, rtol=0, atol=1e-13)
    tau = u.apply(K0[3] * theta_b + K0[2] * psi * z)
    assert np.allclose(t1_, tau, rtol=0, atol=1e-12 * np.abs(K0).max())
    assert np.allclose(t2_, -tau, rtol=0, atol=1e-12 * np.abs(K0).max())
    assert np.abs(f1).max() < 1e-12 * np.abs(K0).max()
    assert U == pytest.approx(0.5 * K0[2] * psi ** 2 + 0.5 * K0[3] * theta_b @ theta_b, rel=1e-12)
    # both angles are finite, so the order matters: the factors taken the
    # other way round (b_2 = u t_2^-1, b_1 = u* t_1^-1) give another vector
    b2m = u * t2.inv()
    b1m = u.inv() * t1.inv()
    theta_m = (b2m * b1m.inv()).as_rotvec()
    assert np.linalg.norm(theta_m - theta_b) > 1e-2 * np.linalg.norm(theta_b)
