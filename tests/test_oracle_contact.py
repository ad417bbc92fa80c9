"""Pins of the oracle's Hertz-Mindlin contact (Methods, "Contact"; reading
R11 of the oracle's header) against closed forms of contact mechanics.

* Head-on collision of two equal elastic spheres (Hertz): the maximum overlap
  delta_m = (15 m* v0^2 / (16 E* sqrt(R*)))^(2/5), the contact time
  t_c = (4/5) B(2/5, 1/2) delta_m / v0 = 2.9432 delta_m / v0, and a rebound
  at the incoming speed.
* A sphere held between two clamped spheres at overlap delta_0 (centre
  distance h) has decoupled small-amplitude modes.  Along the line of centres
  the stiffness is 2 dF/d(delta) = 4 E* a_0.  Tangential translation has
  stiffness 2 k_t - 2 F_n / h (the preload tilts with the displacement) and
  rotation about the tangent has 2 k_t R^2, with Mindlin's k_t = 8 G* a_0 and
  a_0 = sqrt(R* delta_0).  The damping of these modes is 2 gamma_n (normal)
  and 2 gamma_t (tangential translation).  A sphere sliding between them
  decelerates at 2 mu F_n / m.

A dropped factor, a wrong sign of a velocity term or a wrong effective modulus
moves at least one of these numbers far outside its tolerance.
"""
import math

import numpy as np
import pytest
from scipy.special import beta

from oracle import Oracle, contact_pair
from paper_2603_27279_gb300 import workloads as W

E, NU = 1e4, 0.3
ESTAR = E / (2 * (1 - NU * NU))
GSTAR = E / (2 * (1 + NU)) / (2 * (2 - NU))


def spheres(x, v=None, w=None, R=0.5, m=1.0, clamped=None, contact=None, dt=1e-4, rods=None):
    x = np.asarray(x, dtype=float)
    N = len(x)
    offs = np.arange(N + 1, dtype=np.int64) if rods is None else np.asarray(rods, dtype=np.int64)
    Rn = len(offs) - 1
    return W.RodSystem(name="spheres", rod_offset=offs, x=x, q=np.tile([1.0, 0, 0, 0], (N, 1)),
                       v=np.zeros((N, 3)) if v is None else np.asarray(v, float),
                       omega=np.zeros((N, 3)) if w is None else np.asarray(w, float),
                       mass=np.full(N, m), radius=np.full(N, R), m_body=np.zeros((N, 3)),
                       clamped=np.zeros(N, np.uint8) if clamped is None else np.asarray(clamped, np.uint8),
                       x_rest=x.copy(), q_rest=np.tile([1.0, 0, 0, 0], (N, 1)), E=np.full(Rn, 1e4),
                       nu=np.full(Rn, 0.3), d=np.full(Rn, 0.5), dipole_mode=0, damping=0.0,
                       contact=contact or W.ContactParams(E=E, nu=NU, mu=0.5), dt=dt)


def test_hertz_head_on_collision():
    R, m, v0 = 0.5, 1.0, 0.4
    Rs, ms = R / 2, m / 2
    dm = (15 * ms * v0 ** 2 / (16 * ESTAR * math.sqrt(Rs))) ** 0.4
    tc = 0.8 * beta(0.4, 0.5) * dm / v0
    dt = tc / 400
    gap = 1e-3
    s = spheres([[-R - gap / 2, 0, 0], [R + gap / 2, 0, 0]], v=[[v0 / 2, 0, 0], [-v0 / 2, 0, 0]], dt=dt)
    o = Oracle(s)
    t_in = t_out = None
    min_dist = 10.0
    t = 0.0
    for _ in range(4000):
        o.run(1)
        t += dt
        d = np.linalg.norm(o.x[3:6] - o.x[0:3])
        min_dist = min(min_dist, d)
        if d < 2 * R and t_in is None:
            t_in = t
        if t_in is not None and d >= 2 * R:
            t_out = t
            break
    assert t_out is not None
    assert abs((t_out - t_in) - tc) <= 2 * dt, (t_out - t_in, tc)
    assert (2 * R - min_dist) == pytest.approx(dm, rel=1e-4)
    vrel = o.v[0] - o.v[3]
    assert -vrel == pytest.approx(v0, rel=1e-5)            # elastic rebound
    assert np.abs(o.w).max() == 0.0                          # head-on: no tangential force


def sandwich(delta0, v=None, w=None, mu=10.0, gamma_n=0.0, gamma_t=0.0, dt=None):
    R = 0.5
    h = 2 * R - delta0
    cp = W.ContactParams(E=E, nu=NU, mu=mu, gamma_n=gamma_n, gamma_t=gamma_t)
    a0 = math.sqrt(R / 2 * delta0)
    dt = dt or 0.02 / math.sqrt(5 * 8 * GSTAR * a0)
    s = spheres([[0, 0, 0], [0, 0, -h], [0, 0, h]], v=[v or [0, 0, 0], [0, 0, 0], [0, 0, 0]],
                w=[w or [0, 0, 0], [0, 0, 0], [0, 0, 0]], clamped=[0, 1, 1], contact=cp, dt=dt)
    return Oracle(s), a0, dt


def _period(ts, ys):
    """Mean period from upward zero crossings (linear interpolation)."""
    idx = np.where((ys[:-1] < 0) & (ys[1:] >= 0))[0]
    tz = ts[idx] - ys[idx] * (ts[idx + 1] - ts[idx]) / (ys[idx + 1] - ys[idx])
    return float(np.mean(np.diff(tz)))


def _trace(o, steps, get):
    ts, ys = [], []
    for k in range(steps):
        o.run(1)
        ts.append((k + 1) * o.sys.dt)
        ys.append(get(o))
    return np.array(ts), np.array(ys)


@pytest.mark.parametrize("mode", ["normal", "tangential", "rotation"])
def test_sandwich_mode_frequencies(mode):
    delta0 = 0.01
    if mode == "normal":
        o, a0, dt = sandwich(delta0, v=[0, 0, 1e-4])
        k, inert = 4 * ESTAR * a0, 1.0
        get = lambda o: o.x[2]  # noqa: E731
    elif mode == "tangential":
        o, a0, dt = sandwich(delta0, v=[0, 1e-4, 0])
        Fn, h = 4 / 3 * ESTAR * a0 * delta0, 1.0 - delta0
        k, inert = 2 * 8 * GSTAR * a0 - 2 * Fn / h, 1.0
        get = lambda o: o.x[1]  # noqa: E731
    else:
        o, a0, dt = sandwich(delta0, w=[1e-4, 0, 0])
        k, inert = 2 * 8 * GSTAR * a0 * 0.25, 0.4 * 0.25
        get = lambda o: o.w[0]  # noqa: E731
    T = 2 * math.pi / math.sqrt(k / inert)
    ts, ys = _trace(o, int(5 * T / dt), get)
    if mode == "rotation":
        ys = ys - ys.mean()
    assert _period(ts, ys) == pytest.approx(T, rel=2e-3), (mode, _period(ts, ys), T)
    # the other coordinates stay at rest (decoupled modes)
    if mode != "normal":
        assert abs(o.x[2]) < 1e-9
    if mode != "rotation":
        assert np.abs(o.w[:3]).max() < 1e-12


@pytest.mark.parametrize("which", ["gamma_n", "gamma_t"])
def test_sandwich_damping_rates(which):
    delta0, g = 0.01, 0.5
    if which == "gamma_n":
        o, a0, dt = sandwich(delta0, v=[0, 0, 1e-4], gamma_n=g)
        get = lambda o: o.x[2]  # noqa: E731
    else:
        o, a0, dt = sandwich(delta0, v=[0, 1e-4, 0], gamma_t=g)
        get = lambda o: o.x[1]  # noqa: E731
    ts, ys = _trace(o, 20000, get)
    # the envelope decays as exp(-(2 g / m) t / 2); half the peak-to-trough
    # swing is free of the constant offset a new contact's first increment
    # v_t dt leaves in xi
    pk = np.where((ys[1:-1] > ys[:-2]) & (ys[1:-1] >= ys[2:]))[0] + 1
    tr = np.where((ys[1:-1] < ys[:-2]) & (ys[1:-1] <= ys[2:]))[0] + 1
    m = min(len(pk), len(tr))
    amp = 0.5 * (ys[pk[:m]] - ys[tr[:m]])
    tm = 0.5 * (ts[pk[:m]] + ts[tr[:m]])
    slope = np.polyfit(tm, np.log(amp), 1)[0]
    assert slope == pytest.approx(-g, rel=1e-2), slope


def test_coulomb_sliding_deceleration():
    """v0 = 0.06: the contacts stick for about 30 steps, then slide until
    rest after about 190 steps.  While sliding, dv/dt = -2 mu F_n / m plus the
    lateral push 2 F_n y / (h m) of the tilted normal forces (below 1% of the
    friction here); the velocity change over the sliding window must match the
    integral of that law over the measured y(t)."""
    delta0, mu = 0.01, 0.1
    o, a0, dt = sandwich(delta0, v=[0, 0.06, 0], mu=mu)
    Fh, h = 4 / 3 * ESTAR * a0 * delta0, 1.0 - delta0
    ys, vs = [], []
    for _ in range(200):
        o.run(1)
        ys.append(o.x[1])
        vs.append(o.v[1])
    ys, vs = np.array(ys), np.array(vs)
    k0, k1 = 60, 170
    assert vs[k1] > 0.005
    accel = -2 * mu * Fh + 2 * Fh * ys / h
    dv_model = dt * (0.5 * accel[k0] + accel[k0 + 1:k1].sum() + 0.5 * accel[k1])
    dv = vs[k1] - vs[k0]
    assert dv == pytest.approx(dv_model, rel=2e-3), (dv, dv_model, -2 * mu * Fh * (k1 - k0) * dt)
    assert np.abs(o.w[:3]).max() < 1e-12    # the friction torques cancel


def test_pair_law_direct_values():
    """Hertz force and Mindlin stiffness at one overlap, and the Coulomb cap."""
    cp = W.ContactParams(E=E, nu=NU, mu=0.3)
    R, delta = 0.5, 0.02
    xi, xj = np.zeros(3), np.array([0.0, 0.0, -(2 * R - delta)])
    z = np.zeros(3)
    fi, ti, tj, xn = contact_pair(cp, xi, xj, z, z, z, z, R, R, None, 1e-3)
    a = math.sqrt(R / 2 * delta)
    assert fi == pytest.approx([0, 0, 4 / 3 * ESTAR * a * delta], rel=1e-13)
    assert np.abs(ti).max() == 0 and np.abs(tj).max() == 0
    # a stored tangential displacement below the cap: F_t = -8 G* a xi
    small = np.array([1e-7, 0, 0])
    fi, ti, tj, xn = contact_pair(cp, xi, xj, z, z, z, z, R, R, small, 1e-3)
    assert fi[0] == pytest.approx(-8 * GSTAR * a * 1e-7, rel=1e-12)
    assert np.allclose(xn, small, rtol=0, atol=1e-22)
    # torque on each sphere: (-R n) x F_t with n = +z for i, contact on both
    assert ti == pytest.approx(np.cross([0, 0, -R], [fi[0], 0, 0]), rel=1e-12)
    assert tj == pytest.approx(np.cross([0, 0, -R], [fi[0], 0, 0]), rel=1e-12)
    # far above the cap: |F_t| = mu F_n and xi is pulled back to the cap
    big = np.array([1.0, 0, 0])
    fi, ti, tj, xn = contact_pair(cp, xi, xj, z, z, z, z, R, R, big, 1e-3)
    Fn = 4 / 3 * ESTAR * a * delta
    assert abs(fi[0]) == pytest.approx(0.3 * Fn, rel=1e-13)
    assert xn[0] == pytest.approx(0.3 * Fn / (8 * GSTAR * a), rel=1e-12)
    # apart: no contact
    assert contact_pair(cp, xi, np.array([0, 0, -1.001]), z, z, z, z, R, R, None, 1e-3) is None


def test_bonded_neighbours_are_excluded():
    """A rod with overlapping neighbours (spacing 0.8 < 2R) folded back so that
    particles 0 and 5 overlap: with exclude = 3 only (0, 5) is a contact, with
    exclude = 5 none, and without rods' bonds every overlapping pair is."""
    pts = np.array([[0, 0, 0], [0.8, 0, 0], [1.6, 0, 0], [1.6, 0.8, 0], [0.8, 0.8, 0], [0.0, 0.85, 0]])
    for excl, expect in ((3, {(0, 5), (5, 0)}), (5, set())):
        s = spheres(pts, rods=[0, 6], contact=W.ContactParams(E=E, nu=NU, exclude=excl))
        o = Oracle(s)
        o.forces()
        assert set(o.contacts("current")) == expect, excl
    s = spheres(pts, contact=W.ContactParams(E=E, nu=NU, exclude=3))   # six one-particle rods
    o = Oracle(s)
    o.forces()
    pairs = {p for p in o.contacts("current") if p[0] < p[1]}
    assert pairs == {(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (0, 5), (1, 4)}


def test_history_levels_and_antisymmetry():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 2.2, (30, 3))
    s = spheres(x, v=rng.standard_normal((30, 3)) * 0.1, w=rng.standard_normal((30, 3)),
                contact=W.ContactParams(E=E, nu=NU, mu=0.4, gamma_n=0.2, gamma_t=0.1), dt=1e-4)
    o = Oracle(s)
    assert o.contacts("current") is None and o.contacts("previous") is None
    f, _ = o.forces()
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).max()     # f_j = -f_i
    cur = o.contacts("current")
    assert cur and o.contacts("previous") is None
    o.run(5)
    cur, prev = o.contacts("current"), o.contacts("previous")
    assert cur and prev
    for (i, j), xi in cur.items():
        assert np.array_equal(cur[(j, i)], -xi)
    o.forces()                                   # stand-alone: no shift
    assert o.contacts("current").keys() == cur.keys()
    o.run(1)
    assert o.contacts("previous").keys() == cur.keys()
    o.reset_history()
    assert o.contacts("current") is None
    assert not o.contact_overflow


@pytest.mark.parametrize("Ri,Rj", [(0.5, 0.5), (0.4, 0.7)])
def test_meshing_rotation_does_not_slip(Ri, Rj):
    """Spheres spinning like meshing gears (R_i w_i = -R_j w_j about an axis
    normal to the line of centres) have equal contact-point velocities: no
    tangential force.  Spinning the same way, they slip at 2 R w: the
    tangential damping force is then -gamma_t v_t."""
    cp = W.ContactParams(E=E, nu=NU, mu=10.0, gamma_t=0.3)      # below the Coulomb limit
    xi, xj = np.zeros(3), np.array([-(Ri + Rj - 0.01), 0.0, 0.0])
    z = np.zeros(3)
    w = 2.0
    fi, ti, tj, xn = contact_pair(cp, xi, xj, z, z, [0, 0, w / Ri], [0, 0, -w / Rj], Ri, Rj, None, 1e-3)
    assert abs(fi[1]) < 1e-12 and abs(fi[2]) < 1e-12 and np.abs(xn).max() < 1e-15
    fi, ti, tj, xn = contact_pair(cp, xi, xj, z, z, [0, 0, w / Ri], [0, 0, w / Rj], Ri, Rj, None, 1e-3)
    # v_rel = -(R_i w_i + R_j w_j) x n = -(2 w z) x x = -2 w y
    assert xn == pytest.approx([0, -2 * w * 1e-3, 0], abs=1e-15)
    a = math.sqrt(Ri * Rj / (Ri + Rj) * 0.01)
    assert fi[1] == pytest.approx(8 * GSTAR * a * 2 * w * 1e-3 + 0.3 * 2 * w, rel=1e-12)


def test_history_follows_a_rotated_contact_plane():
    """A stored tangential displacement carried into a contact plane rotated
    by 30 degrees keeps its length and lies in the new plane."""
    cp = W.ContactParams(E=E, nu=NU, mu=10.0)
    R = 0.5
    z = np.zeros(3)
    xi_old = np.array([2e-4, 0.0, 0.0])          # in the plane normal to z
    ang = math.radians(30)
    n1 = np.array([math.sin(ang), 0.0, math.cos(ang)])
    xj = -n1 * (2 * R - 0.01)
    fi, ti, tj, xn = contact_pair(cp, z, xj, z, z, z, z, R, R, xi_old, 1e-3)
    assert np.linalg.norm(xn) == pytest.approx(2e-4, rel=1e-13)
    assert abs(xn @ n1) < 1e-18


def test_sampled_search_matches_the_full_pass():
    """The sampled brute-force search (used at full size) equals the full
    evaluation of a fresh state on the sampled particles."""
    s = W.granular(7, 5, 6, seed=9)
    o = Oracle(s)
    f, t = o.forces()
    idx = np.arange(0, s.n, 5)
    fs, ts = Oracle(s).contact_sample(idx)
    assert np.array_equal(fs, f[idx]) and np.array_equal(ts, t[idx])
