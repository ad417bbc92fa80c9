"""Pins of the oracle's bond-level damping (Methods, "Damping"; reading R10 of
the oracle's header).

Each test sets up a free dimer along z in one pure deformation mode.  By
symmetry the mode stays pure, and in the small-amplitude limit its coordinate
y obeys a damped oscillator  y'' + c y' + k y = 0  with k = a K and c = a g,
where K is the bond's spring constant of that mode, g its damping factor and
a the inverse effective inertia of the mode:

* radial (stretch s):            a = 2/m
* twist  (relative angle about z): a = 2/I
* bend   (relative angle about x): a = 2/I
* shear  (eta = u/L + alpha, u the transverse offset, alpha the common
  rotation of both particles): a = 2/m + L^2/(2 I)

The oracle's trajectory must converge to the closed-form solution at first
order in dt (the radial term uses the half-step velocity; the angular rates
are backward differences, both lagging by dt/2).  A wrong sign, a missing
factor r_f or 1/2 in the shear torque, or a wrong direction of a term leaves
an O(1) error that does not shrink with dt.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _util import qexp

MASS = 1.0
RADIUS = 0.5
INERTIA = 0.4 * MASS * RADIUS ** 2
L = 1.7
ZETA = 0.1
AMP = 1e-3


def _dimer(mode, g, dt):
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, L]])
    q = np.tile([1.0, 0.0, 0.0, 0.0], (2, 1))
    if mode == "radial":
        x[1, 2] += AMP
    elif mode == "twist":
        q[0], q[1] = qexp([0, 0, -AMP / 2]), qexp([0, 0, AMP / 2])
    elif mode == "bend":
        q[0], q[1] = qexp([-AMP / 2, 0, 0]), qexp([AMP / 2, 0, 0])
    elif mode == "shear":
        q[0] = q[1] = qexp([AMP, 0, 0])
    s = W.RodSystem(name="dimer_" + mode, rod_offset=np.array([0, 2], dtype=np.int64), x=x, q=q,
                    v=np.zeros((2, 3)), omega=np.zeros((2, 3)), mass=np.full(2, MASS),
                    radius=np.full(2, RADIUS), m_body=np.zeros((2, 3)), clamped=np.zeros(2, np.uint8),
                    x_rest=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, L]]), q_rest=np.tile([1.0, 0, 0, 0], (2, 1)),
                    E=np.full(1, 1e4), nu=np.full(1, 0.3), d=np.ones(1), dipole_mode=0, damping=0.0,
                    bond_damping=np.asarray(g, dtype=float).reshape(1, 4), dt=dt)
    return Oracle(s)


def _angle_about(q, axis):
    return 2.0 * math.atan2(q[axis + 1], q[0])


def _coordinate(mode, o):
    x, q, _, _, _ = o.state()
    if mode == "radial":
        return float(np.linalg.norm(x[1] - x[0]) - L)
    if mode == "twist":
        return _angle_about(q[1], 2) - _angle_about(q[0], 2)
    if mode == "bend":
        return _angle_about(q[1], 0) - _angle_about(q[0], 0)
    # shear: rotation of the central frame about x plus the bond's tilt
    qc = q[0] + q[1]
    alpha = _angle_about(qc / np.linalg.norm(qc), 0)
    d = x[1] - x[0]
    return alpha + math.atan2(d[1], d[2])


def _mode_constants(mode, K):
    a = {"radial": 2 / MASS, "twist": 2 / INERTIA, "bend": 2 / INERTIA,
         "shear": 2 / MASS + L * L / (2 * INERTIA)}[mode]
    Kmode = {"radial": K[0], "shear": K[1], "twist": K[2], "bend": K[3]}[mode]
    return a, Kmode


def _damping_factors(K):
    """g per mode for damping ratio ZETA: c = 2 zeta sqrt(k) -> g = 2 zeta sqrt(K/a)."""
    g = np.zeros(4)
    for idx, mode in enumerate(["radial", "shear", "twist", "bend"]):
        a, Km = _mode_constants(mode, K)
        g[idx] = 2 * ZETA * math.sqrt(Km / a)
    return g


def _closed_form(t, k, c, y0):
    wd = math.sqrt(k - c * c / 4)
    return np.exp(-c * t / 2) * (y0 * np.cos(wd * t) + (c * y0 / (2 * wd)) * np.sin(wd * t))


def _max_error(mode, dt, periods=2.0):
    probe = _dimer(mode, np.zeros(4), dt)
    K = probe.bond_K[0].copy()
    g = _damping_factors(K)
    o = _dimer(mode, g, dt)
    a, Km = _mode_constants(mode, K)
    gm = g[{"radial": 0, "shear": 1, "twist": 2, "bend": 3}[mode]]
    k, c = a * Km, a * gm
    T = periods * 2 * math.pi / math.sqrt(k)
    every = max(1, int(round(T / dt / 200)))
    n_chunks = int(round(T / dt)) // every
    ts, ys = [0.0], [_coordinate(mode, o)]
    for _ in range(n_chunks):
        o.run(every)
        ts.append(o.state()[4])
        ys.append(_coordinate(mode, o))
    ts, ys = np.array(ts), np.array(ys)
    return float(np.max(np.abs(ys - _closed_form(ts, k, c, ys[0])))) / AMP, ts, ys


@pytest.mark.parametrize("mode", ["radial", "shear", "twist", "bend"])
def test_damped_mode_converges_to_closed_form(mode):
    k_base = _dimer(mode, np.zeros(4), 1e-4).bond_K[0]
    a, Km = _mode_constants(mode, k_base)
    dt = 0.02 / math.sqrt(a * Km)   # omega dt = 0.02
    e1, _, ys = _max_error(mode, dt)
    e2, _, _ = _max_error(mode, dt / 2)
    # the mode decays (by exp(-2 pi zeta) per period)
    assert abs(ys[-1]) < 0.5 * AMP
    assert e1 < 0.05, (mode, e1)
    ratio = e1 / e2
    assert 1.6 < ratio < 2.6, (mode, e1, e2, ratio)


@pytest.mark.parametrize("mode", ["radial", "shear", "twist", "bend"])
def test_wrong_damping_factor_is_visible(mode):
    """The closed form with g doubled misses the oracle's trajectory by far
    more than the discretisation error: the pins above resolve a factor 2."""
    k_base = _dimer(mode, np.zeros(4), 1e-4).bond_K[0]
    a, Km = _mode_constants(mode, k_base)
    dt = 0.02 / math.sqrt(a * Km)
    err, ts, ys = _max_error(mode, dt)
    g = _damping_factors(k_base)[{"radial": 0, "shear": 1, "twist": 2, "bend": 3}[mode]]
    wrong = float(np.max(np.abs(ys - _closed_form(ts, a * Km, 2 * a * g, ys[0])))) / AMP
    assert wrong > 5 * err, (mode, err, wrong)


def test_undamped_factors_change_nothing():
    """g = 0 reproduces the elastic forces bit for bit, history or not."""
    o0 = _dimer("bend", np.zeros(4), 1e-4)
    s = o0.sys.copy()
    s.bond_damping = None
    o1 = Oracle(s)
    o0.run(7)
    o1.run(7)
    for a, b in zip(o0.state(), o1.state()):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_history_levels_and_standalone_reproduction():
    """A stand-alone evaluation after a run reproduces the forces the last step
    ended with (rates against the previous level; g_r = 0 here because the
    step evaluated its radial term with the half-step velocity); the levels
    shift once per step and a reset empties them."""
    g = np.array([0.0, 2.0, 0.5, 0.7])
    o = _dimer("bend", g, 1e-4)
    rng = np.random.default_rng(5)
    o.v[:] = rng.standard_normal(6) * 1e-2
    o.w[:] = rng.standard_normal(6)
    assert np.isnan(o.bond_history).all()
    o.forces()
    h = o.bond_history
    assert np.isnan(h[0, 0]).all() and np.isfinite(h[0, 1]).all()
    o.run(3)
    h3 = o.bond_history
    assert np.isfinite(h3).all()
    f, tau = o.forces()
    assert np.array_equal(f.ravel(), o.f) and np.array_equal(tau.ravel(), o.tau)
    assert np.array_equal(o.bond_history, h3)        # stand-alone: no shift
    o.run(1)
    assert np.array_equal(o.bond_history[0, 0], h3[0, 1])
    o.reset_history()
    assert np.isnan(o.bond_history).all()


def test_radial_term_uses_relative_velocity():
    """Rigid translation and rigid rotation of the dimer are not damped."""
    g = np.array([50.0, 0.0, 0.0, 0.0])
    o = _dimer("radial", g, 1e-4)
    o.x[:] = np.array([0, 0, 0, 0, 0, L])
    o.v[:] = np.array([0.3, -0.2, 0.5, 0.3, -0.2, 0.5])   # translation
    f, _ = o.forces()
    assert np.abs(f).max() < 1e-12
    o.v[:] = np.array([-0.5, 0, 0, 0.5, 0, 0])             # perpendicular to the bond
    f, _ = o.forces()
    assert np.abs(f).max() < 1e-12
    o.v[:] = np.array([0, 0, -0.5, 0, 0, 0.5])             # separating at 1
    f, _ = o.forces()
    assert f[0] == pytest.approx([0, 0, 50.0], abs=1e-12)
    assert f[1] == pytest.approx([0, 0, -50.0], abs=1e-12)
