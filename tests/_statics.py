"""Static equilibrium of a clamped rod by Newton iteration on oracle forces
(used by the cantilever pins; test helper, CPU only)."""
import numpy as np

from paper_2603_27279_gb300 import workloads as W


def rot_quat(phi):
    a = np.linalg.norm(phi)
    if a == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[np.cos(a / 2)], np.sin(a / 2) * phi / a])


def qmul(a, b):
    w1, v1 = a[0], a[1:]
    w2, v2 = b[0], b[1:]
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


def rot_quats(phi):
    """Batch of rotation vectors [k,3] -> unit quaternions [k,4]."""
    a = np.linalg.norm(phi, axis=1)
    out = np.zeros((len(phi), 4))
    out[:, 0] = np.cos(a / 2)
    nz = a > 0
    out[nz, 1:] = (np.sin(a[nz] / 2) / a[nz])[:, None] * phi[nz]
    out[~nz, 0] = 1.0
    return out


def qmul_batch(a, b):
    w1, v1 = a[:, :1], a[:, 1:]
    w2, v2 = b[:, :1], b[:, 1:]
    return np.concatenate([w1 * w2 - np.sum(v1 * v2, axis=1, keepdims=True),
                           w1 * v2 + w2 * v1 + np.cross(v1, v2)], axis=1)


def cantilever_system(n_bonds, L=1.0, h=0.01, w=0.01, E=1.0, nu=0.5):
    """Planar rectangular beam (bending about z) clamped at particle 0."""
    l = L / n_bonds
    n = n_bonds + 1
    x = np.zeros((n, 3))
    x[:, 0] = l * np.arange(n)
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    clamped = np.zeros(n, dtype=np.uint8)
    clamped[0] = 1
    s = W.RodSystem(name="cantilever", rod_offset=np.array([0, n], dtype=np.int64), x=x.copy(), q=q.copy(),
                    v=np.zeros((n, 3)), omega=np.zeros((n, 3)), mass=np.ones(n), radius=np.full(n, 0.5),
                    m_body=np.zeros((n, 3)), clamped=clamped, x_rest=x.copy(), q_rest=q.copy(),
                    E=np.array([E]), nu=np.array([nu]), d=np.array([h]), dipole_mode=0, damping=0.0)
    A = w * h
    I = w * h ** 3 / 12.0
    G = E / (2 * (1 + nu))
    Jt = w * h ** 3 / 3.0  # torsion constant of a thin strip (unused in planar bending)
    K = np.array([E * A / l, 12 * E * I / l ** 3, G * Jt / l, E * I / l])
    return s, K, I


def static_solve(orc, f_ext, tol=1e-13, max_iter=60, x0=None, q0=None):
    """Newton on free particles' (x, rotation vector) with a central-FD Jacobian.

    Only bonds couple particles here (no dipoles), so the residual of particle
    p depends on p-1, p, p+1: columns of particles three apart are perturbed
    together (a 3-colouring of the band) and separated afterwards."""
    n = orc.n
    free = np.where(orc.sys.clamped == 0)[0]
    x = (orc.x.reshape(-1, 3) if x0 is None else x0).copy()
    q = (orc.q.reshape(-1, 4) if q0 is None else q0).copy()
    zeros = np.zeros((n, 3))

    def resid(x, q):
        f, t = orc.forces(x=x, q=q, v=zeros, w=zeros)
        return np.concatenate([(f + f_ext)[free].ravel(), t[free].ravel()])

    def apply(x, q, du):
        x2 = x.copy()
        q2 = q.copy()
        k = len(free)
        dx = du[:3 * k].reshape(k, 3)
        dp = du[3 * k:].reshape(k, 3)
        x2[free] += dx
        q2[free] = qmul_batch(rot_quats(dp), q[free])
        return x2, q2

    scale = np.abs(orc.bond_K).max()
    for _ in range(max_iter):
        r = resid(x, q)
        if np.abs(r).max() < tol * scale * 1e-6 + 1e-300:
            break
        m = len(r)
        k = len(free)
        Jm = np.zeros((m, m))
        h = 1e-7
        pos = np.arange(k)
        for color in range(3):
            sel = pos[pos % 3 == color]
            for comp in range(6):
                cols = (sel * 3 + comp) if comp < 3 else (3 * k + sel * 3 + comp - 3)
                e = np.zeros(m)
                e[cols] = h
                xp, qp = apply(x, q, e)
                xm, qm = apply(x, q, -e)
                dr = (resid(xp, qp) - resid(xm, qm)) / (2 * h)
                # rows of particle p belong to the perturbed column of the
                # colour-class member nearest to p (members are 3 apart)
                owner = np.clip(np.rint((pos - color) / 3.0).astype(int), 0, len(sel) - 1)
                near = np.abs(sel[owner] - pos) <= 1
                pp = pos[near]
                cc = cols[owner[near]]
                for a in range(3):
                    Jm[3 * pp + a, cc] = dr[3 * pp + a]
                    Jm[3 * k + 3 * pp + a, cc] = dr[3 * k + 3 * pp + a]
        du = np.linalg.solve(Jm, -r)
        x, q = apply(x, q, du)
        if np.abs(du).max() < 1e-15:
            break
    return x, q
