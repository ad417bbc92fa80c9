"""Bond and dipole kernels at the same time (bpm_set_overlap).

The concurrent form computes m = q m~ q* in its own kernel, runs the dipole
kernel on the handle's stream and the bond kernel on a second stream, and
joins them before the finish kernel.  The arithmetic of every kernel is the
one of the sequential form, so forces, torques and trajectories must be
bitwise equal to it, in captured graphs and in eager launches alike; with
that, the form inherits the oracle parity of the sequential one, which a
direct comparison below checks once more.
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


def _damped_cilia():
    s = W.cilia(2, 3, 40)
    s.bond_damping = np.tile([0.05, 0.02, 0.002, 0.002], (s.n_rods, 1))
    return s


CASES = {
    "batched_12_mixed": (lambda: W.batched_rods(12, 16, 300), W.PRECISION_MIXED),
    "random_rods_per_rod_ff": (lambda: W.random_rods([5, 40, 129, 300], seed=8, per_rod_field=True,
                                                     dipole_mode=W.DIPOLE_PER_ROD), W.PRECISION_FF),
    "helix_1000_fp64": (lambda: W.helix(1000), W.PRECISION_FP64),
    "cilia_2x3x40_mixed_bond_damping": (_damped_cilia, W.PRECISION_MIXED),
}


def _run(bpm, sysm, precision, mode, steps, timing):
    with bpm.Simulation(sysm, precision=precision) as sim:
        sim.set_overlap(mode)
        sim.set_timing(timing)
        f0, t0 = sim.forces()
        on = sim.overlap()
        sim.step(steps)
        x, q, v, w, _ = sim.get_state()
        f1, t1 = sim.forces()
    return on, (f0, t0, x, q, v, w, f1, t1)


@pytest.mark.parametrize("timing", [False, True], ids=["graphs", "eager"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_overlap_is_bitwise_the_sequential_form(bpm, case, timing):
    make, precision = CASES[case]
    sysm = make()
    on1, a = _run(bpm, sysm, precision, 1, 20, timing)
    on0, b = _run(bpm, sysm, precision, 0, 20, timing)
    assert on1[0] == 1 and on1[1] > 0 and on1[2] > 0
    assert on0 == (0, 0, 0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("plan", [(1, 100), (2, 0)], ids=["ordered", "warp_tiles"])
def test_capped_forms_are_bitwise_the_sequential_form(bpm, plan):
    """The register-capped kernels of the concurrent form (the ordered
    FP32-pair kernel at 144 registers, the bond kernel at 112) give the
    sequential form's bits, in graphs, for a plan fixed to each FP32-pair
    kernel that runs beside the bond kernel."""
    sysm = W.batched_rods(24, 16, 500)
    res = []
    for mode in (1, 0):
        with bpm.Simulation(sysm, precision=W.PRECISION_MIXED) as sim:
            sim.set_dipole_plan(*plan)
            sim.set_overlap(mode)
            f0, t0 = sim.forces()
            on = sim.overlap()
            sim.step(20)
            x, q, v, w, _ = sim.get_state()
            res.append((on, (f0, t0, x, q, v, w)))
    assert res[0][0][0] == 1 and res[1][0] == (0, 0, 0)
    for u, v in zip(res[0][1], res[1][1]):
        assert np.array_equal(u, v)


def test_overlap_forces_match_oracle(bpm):
    """FP32-pair bound (1e-5, norm-wise) of the concurrent form on ragged
    batched rods."""
    sysm = W.batched_rods(12, 16, 300)
    with bpm.Simulation(sysm, precision=W.PRECISION_MIXED) as sim:
        sim.set_overlap(1)
        f, t = sim.forces()
        assert sim.overlap()[0] == 1
    fo, to = Oracle(sysm).forces()
    assert np.linalg.norm(f - fo) <= 1e-5 * np.linalg.norm(fo)
    assert np.linalg.norm(t - to) <= 1e-5 * np.linalg.norm(to)


def test_automatic_choice_is_bitwise_the_sequential_form(bpm):
    """Mode -1 times the forms and keeps one; either way the results are
    those of the sequential form."""
    sysm = W.batched_rods(40, 16, 400)
    on, a = _run(bpm, sysm, W.PRECISION_MIXED, -1, 5, False)
    _, b = _run(bpm, sysm, W.PRECISION_MIXED, 0, 5, False)
    assert on[0] in (0, 1)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_energy_and_contact_handles(bpm):
    """Energy evaluations run sequentially and agree bitwise across modes;
    a handle with contact never takes the concurrent form."""
    sysm = W.batched_rods(6, 16, 100)
    e = []
    for mode in (1, 0):
        with bpm.Simulation(sysm, precision=W.PRECISION_MIXED) as sim:
            sim.set_overlap(mode)
            sim.step(3)
            e.append(sim.energy())
    assert np.array_equal(e[0], e[1])
    with bpm.Simulation(W.crossing_rods(), precision=W.PRECISION_MIXED) as sim:
        sim.set_overlap(1)
        sim.forces()
        assert sim.overlap() == (0, 0, 0)


def test_bad_overlap_mode_is_rejected(bpm):
    with bpm.Simulation(W.straight_rod()) as sim:
        for mode in (-2, 2):
            with pytest.raises(bpm.BpmError):
                sim.set_overlap(mode)
