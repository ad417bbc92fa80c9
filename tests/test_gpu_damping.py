"""GPU parity of bond-level damping (Methods, "Damping") against the oracle.

The angular damping terms use backward-difference rates of the recorded
measures; both sides keep the measures of the previous and of the current
state per bond (oracle header, reading R10).  Compared here: the forces of a
fresh state (radial term only), trajectories through CUDA-graph replays and
split calls, the stand-alone evaluation after a run (which reproduces the
angular damping the last step ended with), the reset by set_state, and the
mixed-precision path.  Tolerances: the forces of one state within 1e-12
norm-wise (the per-particle check of tests/_parity.py leaves out bond damping
terms, so it is not applied here), 1e-9 relative on states after a
trajectory.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import TOL64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def damped(lengths, seed, g=(20.0, 0.5, 0.5, 0.5), **kw):
    sysm = W.random_rods(lengths, seed=seed, **kw)
    rng = np.random.default_rng(seed + 1000)
    sysm.bond_damping = np.asarray(g)[None, :] * rng.uniform(0.5, 1.5, (sysm.n_rods, 4))
    return sysm


def check_fp64(f, t, fo, to, orc):
    assert rel(f, fo) <= TOL64, rel(f, fo)
    assert rel(t, to) <= TOL64, rel(t, to)


@pytest.mark.parametrize("mode", [W.DIPOLE_OFF, W.DIPOLE_GLOBAL, W.DIPOLE_PER_ROD])
def test_fresh_state_forces(bpm, mode):
    """No measures yet: radial damping only, on the state's velocities."""
    sysm = damped([2, 3, 31, 32, 33, 130], seed=21, dipole_mode=mode)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        f, t = sim.forces()
    o = Oracle(sysm)
    fo, to = o.forces()
    check_fp64(f, t, fo, to, o)
    # non-vacuous: the radial term changes the forces well above the bound
    s0 = sysm.copy()
    s0.bond_damping = None
    f0, _ = Oracle(s0).forces()
    assert rel(f0, fo) > 1e-6


@pytest.mark.parametrize("mode", [W.DIPOLE_OFF, W.DIPOLE_PER_ROD])
def test_trajectory_split_calls(bpm, mode):
    """50 steps as 1 + 16 + 33: graph chunks, single steps and the closing
    kick all carry the measure history; then the stand-alone forces."""
    sysm = damped([3, 40, 70, 33], seed=22, dipole_mode=mode, damping=0.02)
    o = Oracle(sysm)
    o.run(50)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        for n in (1, 16, 33):
            sim.step(n)
        x, q, v, w, t = sim.get_state()
        f, tau = sim.forces()
    xo, qo, vo, wo, to_ = o.state()
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-8 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-8 * np.abs(wo).max()
    fo, tauo = o.forces()
    assert rel(f, fo) <= 1e-9 and rel(tau, tauo) <= 1e-9, (rel(f, fo), rel(tau, tauo))


def test_standalone_reproduces_step_and_set_state_forgets(bpm):
    """With g_r = 0 and no global damping the forces of a stand-alone call
    after a run are those the last step ended with (angular rates against
    the previous level); repeated calls do not shift the levels; set_state
    forgets the measures (zero angular rates)."""
    sysm = damped([20, 45], seed=23, g=(0.0, 0.5, 0.5, 0.5), dipole_mode=W.DIPOLE_OFF, damping=0.0)
    o = Oracle(sysm)
    o.run(12)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        sim.step(12)
        f1, t1 = sim.forces()
        f2, t2 = sim.forces()
        assert np.array_equal(f1, f2) and np.array_equal(t1, t2)
        fo, to = o.forces()
        assert np.array_equal(fo.ravel(), o.f) and np.array_equal(to.ravel(), o.tau)
        assert rel(f1, fo) <= 1e-9 and rel(t1, to) <= 1e-9, (rel(f1, fo), rel(t1, to))
        # set_state with the same state: measures forgotten on both sides
        x, q, v, w, t = sim.get_state()
        sim.set_state(x, q, v, w, t)
        f3, t3 = sim.forces()
        o.reset_history()
        fo3, to3 = o.forces()
        assert rel(f3, fo3) <= 1e-9 and rel(t3, to3) <= 1e-9
        # the angular damping was active before the reset
        assert rel(t3, t1) > 1e-6


def test_mixed_precision_with_damping(bpm):
    sysm = damped([33, 100, 257], seed=24, precision=W.PRECISION_MIXED)
    o = Oracle(sysm)
    with bpm.Simulation(sysm) as sim:
        f, t = sim.forces()
        fo, to = o.forces()
        assert rel(f, fo) <= 1e-5 and rel(t, to) <= 1e-5
        sim.step(20)
        o.run(20)
        f, t = sim.forces()
    fo, to = o.forces()
    assert rel(f, fo) <= 1e-5 and rel(t, to) <= 1e-5, (rel(f, fo), rel(t, to))


def test_bond_damping_descriptions(bpm):
    sysm = damped([5, 6], seed=25)
    bad = sysm.copy()
    bad.bond_damping = bad.bond_damping.copy()
    bad.bond_damping[1, 2] = -1.0
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    bad.bond_damping[1, 2] = np.nan
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    # zero factors: bitwise the undamped system
    zero = sysm.copy()
    zero.bond_damping = np.zeros((2, 4))
    plain = sysm.copy()
    plain.bond_damping = None
    with bpm.Simulation(zero) as a, bpm.Simulation(plain) as b:
        a.step(5)
        b.step(5)
        for u, w in zip(a.get_state(), b.get_state()):
            assert np.array_equal(np.asarray(u), np.asarray(w))
    # the adjoint does not differentiate bond damping
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        with pytest.raises(bpm.BpmError):
            sim.adjoint_begin(4, 2)
