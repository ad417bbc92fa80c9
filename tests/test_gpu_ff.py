"""GPU parity of the float-float dipole path (BPM_FF) against the CPU FP64
oracle.

The float-float path is held to the FP64 parity bounds of tests/_parity.py:
norm-wise relative force and torque error <= 1e-12 (5e-12 on the twisted
helix) and, per particle, |dF_i| <= 1e-12 times the sum of the magnitudes of
the particle's force terms.  Its own rounding (a few 2^-48 per pair term,
against 2^-53 for FP64) stays inside those bounds on every workload here;
against the FP64 GPU path it is checked at 1e-12 norm-wise on the small
cases.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import TOL64, TOL64_HELIX, check_fp64, rel

pytestmark = pytest.mark.gpu

TOL_VS_FP64 = 1e-12


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


CASES = {
    "straight_rod_64": lambda: W.straight_rod(),
    "random_rods_ragged_global": lambda: W.random_rods([1, 2, 3, 31, 32, 33, 61, 130, 257], seed=7),
    "random_rods_per_rod_field": lambda: W.random_rods([5, 40, 129, 300], seed=8, per_rod_field=True,
                                                       dipole_mode=W.DIPOLE_PER_ROD),
    "helix_300": lambda: W.helix(300),
    "helix_2000": lambda: W.helix(2000),
    "cilia_2x3x40": lambda: W.cilia(2, 3, 40),
    "batched_12": lambda: W.batched_rods(12, 16, 100),
}


def _shifted(sysm, offset):
    s = sysm.copy()
    s.x = s.x + np.asarray(offset)
    if s.x_rest is not None:
        s.x_rest = s.x_rest + np.asarray(offset)
    return s


def _far_apart():
    """Two rods 2e5 apart: the finest position digit is then 2^-46, coarser
    than the FP64 spacing of coordinates near 1, and still far below what
    the pair forces resolve."""
    s = W.random_rods([40, 57], seed=12)
    s.x[40:] += np.array([2e5, -1e5, 5e4])
    if s.x_rest is not None:
        s.x_rest[40:] += np.array([2e5, -1e5, 5e4])
    return s


# translated systems: other position quanta, negative coordinates
CASES["helix_300_shifted"] = lambda: _shifted(W.helix(300), (3000.0, -2000.0, 500.0))
CASES["random_rods_far_apart"] = _far_apart
# autotuned, and the symmetric kernel with warp tiles of 32 and 1, 2 and 8 tiles per supertile
PLANS = {"auto": (0, 0), "symw": (2, 0), "sym1": (2, 1), "sym2": (2, 2), "sym8": (2, 8)}


@pytest.mark.parametrize("plan", sorted(PLANS))
@pytest.mark.parametrize("case", sorted(CASES))
def test_ff_forces_match_oracle(bpm, case, plan):
    sysm = CASES[case]()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        sim.set_dipole_plan(*PLANS[plan])
        f, t = sim.forces()
        f2, t2 = sim.forces()
    o = Oracle(sysm)
    fo, to = o.forces()
    check_fp64(f, t, fo, to, o, norm_rel=TOL64_HELIX if case.startswith("helix") else TOL64)
    # the same decomposition gives the same bits
    assert np.array_equal(f, f2) and np.array_equal(t, t2)


@pytest.mark.parametrize("case", sorted(CASES))
def test_ff_agrees_with_fp64_gpu_path(bpm, case):
    sysm = CASES[case]()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        f, t = sim.forces()
    with bpm.Simulation(sysm, precision=bpm.BPM_FP64) as sim:
        f6, t6 = sim.forces()
    assert rel(f, f6) <= TOL_VS_FP64, rel(f, f6)
    assert rel(t, t6) <= TOL_VS_FP64, rel(t, t6)


def test_ff_trajectory_straight_rod_1000_steps(bpm):
    """The 64-particle rod over its 1000-step horizon, with the bounds of the
    FP64 path's trajectory test: state within 1e-9 of the oracle's, relative
    to the state's scale."""
    sysm = W.straight_rod()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        sim.step(1000)
        x, q, v, w, t = sim.get_state()
    o = Oracle(sysm)
    o.run(1000)
    xo, qo, vo, wo, _ = o.state()
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-9 * max(np.abs(vo).max(), 1e-3)
    assert np.abs(w - wo).max() <= 1e-9 * max(np.abs(wo).max(), 1e-3)


def test_ff_full_size_helix_forces_and_10_steps(bpm):
    """The 16384-particle helix in the bench's launch configuration: step-1
    forces within the FP64 bound and a 10-step trajectory with the bounds of
    the FP64 full-size test."""
    sysm = W.helix()
    o = Oracle(sysm)
    fo, to = o.forces()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        f, t = sim.forces()
        check_fp64(f, t, fo, to, o, norm_rel=TOL64_HELIX)
        sim.step(10)
        x, q, v, w, tt = sim.get_state()
    o.run(10)
    xo, qo, vo, wo, _ = o.state()
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-10
    assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()


def test_ff_full_size_cilia_sampled(bpm):
    """131072 particles (1.7e10 pairs): 96 sampled particles whose dipole sums
    the oracle computes one by one over all partners, plus the oracle's O(N)
    bond and Zeeman terms."""
    sysm = W.cilia(precision=W.PRECISION_FF)
    with bpm.Simulation(sysm) as sim:
        f, t = sim.forces()
    rng = np.random.default_rng(0)
    idx = np.sort(np.concatenate([rng.choice(sysm.n, 90, replace=False), [0, 1, 255, 256, sysm.n - 2, sysm.n - 1]]))
    nodip = sysm.copy()
    nodip.dipole_mode = W.DIPOLE_OFF
    o = Oracle(nodip)
    fb, tb, m = o.forces(want_m=True)
    od = Oracle(sysm)
    Fd, Td, _ = od.dipole_sample(idx, m=m)
    check_fp64(f[idx], t[idx], fb[idx] + Fd, tb[idx] + Td, od, idx=idx)


def test_ff_full_size_batched(bpm):
    """2048 rods of lengths U{16..1024}, per-rod dipoles: the whole force
    field against the oracle."""
    sysm = W.batched_rods(precision=W.PRECISION_FF)
    with bpm.Simulation(sysm) as sim:
        f, t = sim.forces()
    o = Oracle(sysm)
    fo, to = o.forces()
    check_fp64(f, t, fo, to, o, sample=8192)


def test_ff_position_out_of_range_is_reported(bpm):
    """The finest position digit is fixed at create from the initial extent;
    a particle moved far beyond it makes the step report non-finite forces,
    and the handle works again after a state inside the range."""
    sysm = W.straight_rod()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        x = sysm.x.copy()
        x[5, 0] = 1e9
        sim.set_state(x=x, q=sysm.q, v=sysm.v, omega=sysm.omega, t=0.0)
        with pytest.raises(bpm.BpmError) as e:
            sim.step(2)
        assert e.value.code == bpm.BPM_ERR_NONFINITE
        sim.set_state(x=sysm.x, q=sysm.q, v=sysm.v, omega=sysm.omega, t=0.0)
        sim.step(2)
        f, t = sim.forces()
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(t))


def test_ff_rejects_ordered_plan(bpm):
    sysm = W.straight_rod()
    with bpm.Simulation(sysm, precision=bpm.BPM_FF) as sim:
        with pytest.raises(bpm.BpmError) as e:
            sim.set_dipole_plan(bpm.BPM_PLAN_ORDERED, 2)
        assert e.value.code == bpm.BPM_ERR_ARG


def test_ff_all_terms_with_fluid(bpm):
    """Every optional term at once (contact, bond damping, per-rod and global
    dipoles, field, fluid) with float-float dipole pairs: forces and a
    45-step trajectory across LBM cycles and graph replays, with the bounds
    of the FP64 combined test."""
    from test_gpu_combined import combined
    for mode in (W.DIPOLE_PER_ROD, W.DIPOLE_GLOBAL):
        s = combined(seed=74, mode=mode, precision=W.PRECISION_FF)
        o = Oracle(s)
        f0o, t0o = o.forces()
        o.run(45)
        with bpm.Simulation(s) as sim:
            f0, t0 = sim.forces()
            assert rel(f0, f0o) <= 1e-12 and rel(t0, t0o) <= 1e-12, (rel(f0, f0o), rel(t0, t0o))
            for k in (7, 16, 22):
                sim.step(k)
            x, q, v, w, t = sim.get_state()
            r, u = sim.lbm_fields()
        xo, qo, vo, wo, to_ = o.state()
        assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
        assert np.abs(q - qo).max() <= 1e-9
        assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()
        ro, uo = o.lbm_macro()
        assert np.abs(u - uo).max() <= 1e-9 * np.abs(uo).max()
