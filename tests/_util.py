"""Small numpy helpers for tests (test code only; not the method)."""
import math

import numpy as np


def qexp(phi):
    """Unit quaternion of the rotation vector phi (angle |phi| about phi^)."""
    phi = np.asarray(phi, dtype=np.float64)
    a = float(np.linalg.norm(phi))
    if a == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[math.cos(a / 2)], math.sin(a / 2) * phi / a])


def qmul(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.concatenate([[a[0] * b[0] - a[1:] @ b[1:]],
                           a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:])])


def qrot_matrix(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_quat(rng):
    g = rng.standard_normal(4)
    return g / np.linalg.norm(g)


def default_K(E=1e4, nu=0.3, d=1.0, L=1.0):
    """Spring constants of a cylindrical bond (used only to pick magnitudes)."""
    G = E / (2 * (1 + nu))
    A = math.pi * d * d / 4
    I = math.pi * d ** 4 / 64
    J = math.pi * d ** 4 / 32
    return np.array([E * A / L, 12 * E * I / L ** 3, G * J / L, E * I / L])


def read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    lines = [ln.split("#")[0].strip() for ln in open(path)]
    return [ln for ln in lines if ln]
