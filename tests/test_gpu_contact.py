"""GPU parity of the Hertz-Mindlin contact (Methods, "Contact"; reading R11
of the oracle) against the oracle's brute-force all-pairs search.

Compared: forces and torques of a fresh state (new contacts only), of a
state reached through graph-replayed steps (history carried through both
levels), stand-alone evaluations after a run and after set_state, rods whose
bonded neighbours overlap (exclusion), mixed precision, determinism, and the
capacity error.  Tolerances: the forces of one state norm-wise within 1e-12;
states after a trajectory within 1e-9 of their scale.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

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


CASES = {
    "granular_9x7x5": lambda: W.granular(9, 7, 5, seed=51),
    "granular_ragged_radii": lambda: W.granular(11, 3, 13, seed=52, rmin=0.3, rmax=0.6, spacing=0.8),
    "crossing_rods_per_rod_dipoles": lambda: W.crossing_rods(seed=53),
    "crossing_rods_global_dipoles": lambda: W.crossing_rods(seed=54, dipole_mode=W.DIPOLE_GLOBAL),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fresh_state_forces(bpm, case):
    sysm = CASES[case]()
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        f, t = sim.forces()
    o = Oracle(sysm)
    fo, to = o.forces()
    assert rel(f, fo) <= 1e-12 and rel(t, to) <= 1e-12, (rel(f, fo), rel(t, to))
    # non-vacuous: contact changes the forces
    s0 = sysm.copy()
    s0.contact = None
    f0, _ = Oracle(s0).forces()
    assert rel(f0, fo) > 1e-3


@pytest.mark.parametrize("case", ["granular_9x7x5", "crossing_rods_per_rod_dipoles"])
def test_trajectory_split_calls(bpm, case):
    sysm = CASES[case]()
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
    assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    fo, tauo = o.forces()
    assert rel(f, fo) <= 1e-9 and rel(tau, tauo) <= 1e-9, (rel(f, fo), rel(tau, tauo))


def test_set_state_forgets_histories(bpm):
    sysm = CASES["granular_9x7x5"]()
    o = Oracle(sysm)
    o.run(20)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        sim.step(20)
        f1, t1 = sim.forces()
        x, q, v, w, t = sim.get_state()
        sim.set_state(x, q, v, w, t)
        f2, t2 = sim.forces()
    o.reset_history()
    fo2, to2 = o.forces()
    assert rel(f2, fo2) <= 1e-9 and rel(t2, to2) <= 1e-9
    assert rel(t2, t1) > 1e-6      # the history mattered


def test_mixed_precision_with_contact(bpm):
    sysm = CASES["crossing_rods_global_dipoles"]()
    sysm.precision = W.PRECISION_MIXED
    with bpm.Simulation(sysm) as sim:
        f, t = sim.forces()
    fo, to = Oracle(sysm).forces()
    assert rel(f, fo) <= 1e-5 and rel(t, to) <= 1e-5


def test_deterministic_and_pairwise_balanced(bpm):
    sysm = W.granular(10, 10, 10, seed=55)
    runs = []
    for _ in range(2):
        with bpm.Simulation(sysm) as sim:
            sim.step(7)
            runs.append(sim.get_state() + sim.forces())
    for a, b in zip(*runs):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    # contact only, no other force: the pair terms cancel in the sum
    f = runs[0][-2]
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()


def test_capacity_error_is_reported(bpm):
    sysm = W.granular(6, 6, 6, seed=56, contact=W.ContactParams(cap=2))
    with bpm.Simulation(sysm) as sim:
        with pytest.raises(bpm.BpmError) as e:
            sim.forces()
        assert e.value.code == bpm.BPM_ERR_CAPACITY
    bad = W.granular(3, 3, 3, contact=W.ContactParams(cap=65))
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    bad = W.granular(3, 3, 3, contact=W.ContactParams(nu=0.5))
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    with bpm.Simulation(W.granular(3, 3, 3)) as sim:
        with pytest.raises(bpm.BpmError):
            sim.adjoint_begin(4, 2)


def test_full_size_granular_sampled(bpm):
    """The 128^3 = 2,097,152-sphere granular workload (the bench's contact
    workload, largest supported size 2^21): forces of a fresh state on 1024
    sampled particles against the oracle's brute-force search over all
    particles, and pairwise balance of the whole force field."""
    sysm = W.granular(128, 128, 128)
    with bpm.Simulation(sysm) as sim:
        f, t = sim.forces()
    idx = np.linspace(0, sysm.n - 1, 1024).astype(np.int64)
    fo, to = Oracle(sysm).contact_sample(idx)
    assert rel(f[idx], fo) <= 1e-12 and rel(t[idx], to) <= 1e-12, (rel(f[idx], fo), rel(t[idx], to))
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()
