"""Cantilever pins (SI "Cantilever beam under static loading"): the linear
BPM reproduces Euler-Bernoulli exactly at the nodes for a tip load, and the
energy errors printed in the SI at 10% tip deflection are reproduced."""
import numpy as np
import pytest

from oracle import Oracle

from _statics import cantilever_system, static_solve
from _util import read_golden

E, L = 1.0, 1.0


def _golden():
    return {ln.split()[0]: float(ln.split()[1]) for ln in read_golden("cantilever_energy.txt")}


def _solve_for_tip(o, n_bonds, load_vec_of, target, p0):
    """Secant-free fixed point on the load amplitude so that the tip
    deflection equals target (deflection is nearly linear in the load)."""
    x = q = None
    p = p0
    for _ in range(40):
        x, q = static_solve(o, load_vec_of(p), x0=x, q0=q)
        d = x[-1, 1]
        if abs(d - target) < 1e-12:
            break
        p *= target / d
    return p, x, q


def _bond_energy(o, x, q):
    z = np.zeros_like(x)
    return o.forces(x=x, q=q, v=z, w=z, want_energy=True)[2][0]


@pytest.mark.parametrize("n_bonds", [4, 9])
def test_small_tip_load_matches_euler_bernoulli_at_nodes(n_bonds):
    s, K, I = cantilever_system(n_bonds)
    o = Oracle(s)
    o.bond_K[:] = K
    P = 1e-5 * 3 * E * I / L ** 3        # tip deflection 1e-5 L
    fe = np.zeros((n_bonds + 1, 3))
    fe[-1, 1] = P
    x, q = static_solve(o, fe)
    xs = np.linspace(0.0, L, n_bonds + 1)
    y_eb = P * xs ** 2 * (3 * L - xs) / (6 * E * I)
    assert np.abs(x[:, 1] - y_eb).max() < 1e-8 * y_eb[-1]


def test_point_load_energy_error_printed_in_si():
    g = _golden()
    n = int(g["point_load_N"])
    s, K, I = cantilever_system(n)
    o = Oracle(s)
    o.bond_K[:] = K

    def load(p):
        fe = np.zeros((n + 1, 3))
        fe[-1, 1] = p
        return fe

    P, x, q = _solve_for_tip(o, n, load, 0.1 * L, 0.3 * E * I / L ** 2)
    err = abs(_bond_energy(o, x, q) - P ** 2 * L ** 3 / (6 * E * I)) / (P ** 2 * L ** 3 / (6 * E * I))
    assert err == pytest.approx(g["point_load_rel_error"], abs=g["point_load_tolerance"])
    # "does not decrease further" with more bonds
    s2, K2, _ = cantilever_system(4 * n)
    o2 = Oracle(s2)
    o2.bond_K[:] = K2

    def load2(p):
        fe = np.zeros((4 * n + 1, 3))
        fe[-1, 1] = p
        return fe

    P2, x2, q2 = _solve_for_tip(o2, 4 * n, load2, 0.1 * L, P)
    err2 = abs(_bond_energy(o2, x2, q2) - P2 ** 2 * L ** 3 / (6 * E * I)) / (P2 ** 2 * L ** 3 / (6 * E * I))
    assert err2 >= err * 0.95


def test_uniform_load_needs_128_bonds_for_one_percent():
    """Uniform load applied as equal forces q L / N on every free particle
    (this reading of the SI's loading reproduces its convergence statement)."""
    g = _golden()
    errs = {}
    for n in (int(g["uniform_load_N_above_1pct"]), int(g["uniform_load_N_below_1pct"])):
        s, K, I = cantilever_system(n)
        o = Oracle(s)
        o.bond_K[:] = K
        ell = L / n

        def load(qq, n=n, ell=ell):
            fe = np.zeros((n + 1, 3))
            fe[1:, 1] = qq * ell
            return fe

        qq, x, q = _solve_for_tip(o, n, load, 0.1 * L, 0.8 * E * I / L ** 3)
        U_theo = qq ** 2 * L ** 5 / (40 * E * I)
        errs[n] = abs(_bond_energy(o, x, q) - U_theo) / U_theo
    assert errs[int(g["uniform_load_N_above_1pct"])] > 0.01
    assert errs[int(g["uniform_load_N_below_1pct"])] < 0.01
