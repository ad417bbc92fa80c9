"""Extended-precision (numpy longdouble: 80-bit on x86-64, 128-bit on
aarch64) evaluation of bond, Zeeman and dipole forces, used only to measure
the rounding error of FP64 evaluations (the oracle's and the GPU's).

It restates the same equations as the oracle and so pins nothing about their
correctness; it measures how far an FP64 evaluation can sit from the same
mathematics computed with more mantissa bits.
"""
import numpy as np

L = np.longdouble
EPS64 = np.finfo(np.float64).eps


def _qmul(a, b):
    w1, v1 = a[..., :1], a[..., 1:]
    w2, v2 = b[..., :1], b[..., 1:]
    return np.concatenate([w1 * w2 - np.sum(v1 * v2, -1, keepdims=True),
                           w1 * v2 + w2 * v1 + np.cross(v1, v2)], -1)


def _conj(a):
    return a * np.array([1, -1, -1, -1], dtype=L)


def _rot(q, v):
    p = np.concatenate([np.zeros(v.shape[:-1] + (1,), L), v], -1)
    return _qmul(_qmul(q, p), _conj(q))[..., 1:]


def _nrm(v):
    return np.sqrt(np.sum(v * v, -1, keepdims=True))


def forces_extended(s, with_dipole=True):
    """Bond + uniform-field Zeeman (+ all-pairs dipole) forces and torques of
    a RodSystem with zero velocities, in longdouble; returns float64 arrays."""
    x = s.x.astype(L)
    q = s.q.astype(L)
    qr = s.q_rest.astype(L)
    q = q / _nrm(q)
    qr = qr / _nrm(qr)
    qp = _qmul(q, _conj(qr))
    n = len(x)
    f = np.zeros((n, 3), L)
    t = np.zeros((n, 3), L)
    offs = s.rod_offset
    for r in range(s.n_rods):
        a, b = offs[r], offs[r + 1]
        if b - a < 2:
            continue
        i1 = np.arange(a, b - 1)
        i2 = i1 + 1
        ri = (s.x_rest[i2] - s.x_rest[i1]).astype(L)
        Ln = _nrm(ri)
        rih = ri / Ln
        d, E = L(s.d[r]), L(s.E[r])
        G = E / (2 * (1 + L(s.nu[r])))
        pi = L(np.pi)
        A, I, J = pi * d * d / 4, pi * d ** 4 / 64, pi * d ** 4 / 32
        Kr, Ks, Kt, Kb = E * A / Ln, 12 * E * I / Ln ** 3, G * J / Ln, E * I / Ln
        q1 = qp[i1]
        q2 = qp[i2].copy()
        sg = np.sign(np.sum(q1 * q2, -1, keepdims=True))
        sg[sg == 0] = 1
        q2 = q2 * sg
        qC = q1 + q2
        qC = qC / _nrm(qC)
        rfO = x[i2] - x[i1]
        rfl = _nrm(rfO)
        rf = _rot(_conj(qC), rfO)
        rfh = rf / _nrm(rf)
        fr = Kr * (rfl - Ln) * rfh
        c = np.cross(rih, rfh)
        sgn = _nrm(c)
        cg = np.sum(rih * rfh, -1, keepdims=True)
        gam = np.arctan2(sgn, cg)
        gos = np.where(sgn > 0, gam / np.where(sgn > 0, sgn, 1), 1 / cg)
        gt = c * gos
        fs = Ks * rfl * np.cross(gt, rfh)
        ts = Ks * rfl ** 2 * gt / 2
        rl = _nrm(rf)
        z, xx, yy = rf[:, 2:3], rf[:, 0:1], rf[:, 1:2]
        zero = np.zeros_like(z)
        m0 = np.concatenate([rl + z, -yy, xx, zero], -1) / np.sqrt(2 * rl * np.maximum(rl + z, L(1e-300)))
        m1 = np.concatenate([-yy, rl - z, zero, xx], -1) / np.sqrt(2 * rl * np.maximum(rl - z, L(1e-300)))
        m = np.where(z >= 0, m0, m1)
        u = _qmul(_qmul(_conj(m), _qmul(_conj(qC), q2)), m)
        tn = np.sqrt(u[:, :1] ** 2 + u[:, 3:] ** 2)
        psi = 4 * np.arctan2(u[:, 3:] / tn, u[:, :1] / tn)
        t2c = np.concatenate([u[:, :1] / tn, zero, zero, -u[:, 3:] / tn], -1)
        bq = _qmul(_qmul(t2c, _qmul(u, u)), t2c)
        bq = bq * np.where(bq[:, :1] < 0, -1, 1)
        bv = bq[:, 1:]
        sb = _nrm(bv)
        th = 2 * np.arctan2(sb, bq[:, :1])
        thb = bv * np.where(sb > 0, th / np.where(sb > 0, sb, 1), 2 / bq[:, :1])
        tbt = Kb * thb
        tbt[:, 2:3] += Kt * psi
        F = _rot(qC, fr + fs)
        TS = _rot(qC, ts)
        TB = _rot(_qmul(qC, m), tbt)
        np.add.at(f, i1, F)
        np.add.at(f, i2, -F)
        np.add.at(t, i1, TS + TB)
        np.add.at(t, i2, TS - TB)
    mw = _rot(q, s.m_body.astype(L))
    t += np.cross(mw, np.broadcast_to(s.B.astype(L), mw.shape))
    if with_dipole and s.dipole_mode == 1:
        c = L(s.mu0_over_4pi)
        for i in range(n):
            r = x[i] - x
            r2 = np.sum(r * r, -1)
            r2[i] = 1
            rl = np.sqrt(r2)
            r3 = r2 * rl
            r5 = r3 * r2
            r7 = r5 * r2
            a = r @ mw[i]
            bb = np.sum(mw * r, -1)
            dd = mw @ mw[i]
            Fij = 3 * c * ((a[:, None] * mw + bb[:, None] * mw[i] + dd[:, None] * r) / r5[:, None]
                           - 5 * (a * bb)[:, None] * r / r7[:, None])
            Bj = c * (3 * bb[:, None] * r / r5[:, None] - mw / r3[:, None])
            Fij[i] = 0
            Bj[i] = 0
            f[i] += Fij.sum(0)
            t[i] += np.cross(mw[i], Bj.sum(0))
    return f.astype(np.float64), t.astype(np.float64)


def bond_scales(orc):
    """Per-particle stiffness scales of the bond terms: s_f = sum over the
    particle's bonds of (K_r + K_s) L and s_t = sum of K_s L^2 + K_t + K_b.
    A bond's force carries an absolute rounding error of order eps * s_f:
    its unit bond vector, rotated into the central frame, is only known to a
    few eps in absolute terms however small the shear angle is."""
    n = orc.n
    K = orc.bond_K
    Lb = np.linalg.norm(orc.bond_ri, axis=1)
    sf = np.zeros(n)
    st = np.zeros(n)
    p1 = orc._keep["p1"][: len(K)]
    p2 = orc._keep["p2"][: len(K)]
    bf = (K[:, 0] + K[:, 1]) * Lb
    bt = K[:, 1] * Lb * Lb + K[:, 2] + K[:, 3]
    np.add.at(sf, p1, bf)
    np.add.at(sf, p2, bf)
    np.add.at(st, p1, bt)
    np.add.at(st, p2, bt)
    return sf, st


def fp64_tolerance(reference, scale, rel=1e-12, k_eps=2.0):
    """Norm-wise FP64 parity bound: rel * |reference| + k_eps * eps * |scale|."""
    return rel * np.linalg.norm(reference) + k_eps * EPS64 * np.linalg.norm(scale)
