"""GPU parity of the lattice-Boltzmann fluid and its penalty coupling
(Methods, "Lattice Boltzmann method", "Immersed boundary coupling"; reading
R12 of the oracle) against the oracle.

Compared: the fluid alone (density and velocity fields after several LBM
steps, FP64 and FP32 storage); rods immersed in the fluid through whole and
partial LBM cycles split across calls (particle states, fluid fields, the
stand-alone forces with the penalty term); argument checks.  The momentum
balance between particles and fluid is pinned on the oracle
(test_oracle_lbm.py) and carried here by parity.  Tolerances: FP64 fields within
1e-12 of their scale after a few steps, 1e-9 after trajectories (the
reaction is summed with atomics, reproducible to rounding), the same for
FP64 storage with the float-float collision (BPM_FF handles); FP32 storage
within 1e-6 of the velocity scale.
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


def fluid_only(n=(20, 12, 17), n_sub=2, tau=0.75, seed=61, body=(3e-5, -1e-5, 2e-5)):
    s = W.fluid_rods(n=n, rods=(3,), n_sub=n_sub, tau=tau, seed=seed, body=body)
    s.lbm.coupled = np.zeros(s.n, np.uint8)
    return s


@pytest.mark.parametrize("precision,tol", [(W.PRECISION_FP64, 1e-12), (W.PRECISION_FF, 1e-12),
                                           (W.PRECISION_MIXED, 1e-6)])
def test_fluid_alone_matches_oracle(bpm, precision, tol):
    s = fluid_only()
    s.precision = precision
    o = Oracle(s)
    with bpm.Simulation(s) as sim:
        r0, u0 = sim.lbm_fields()
        ro, uo = o.lbm_macro()
        assert np.abs(r0 - ro).max() <= tol and np.abs(u0 - uo).max() <= tol * np.abs(uo).max()
        sim.step(2 * 7)                    # 7 LBM steps
        r, u = sim.lbm_fields()
    o.run(14)
    ro, uo = o.lbm_macro()
    assert np.abs(r - ro).max() <= tol * 10, np.abs(r - ro).max()
    assert np.abs(u - uo).max() <= tol * 10 * np.abs(uo).max(), np.abs(u - uo).max() / np.abs(uo).max()


@pytest.mark.parametrize("mode", [W.DIPOLE_PER_ROD, W.DIPOLE_GLOBAL])
def test_rods_in_fluid_split_calls(bpm, mode):
    """n_sub = 10: 37 steps as 3 + 14 + 20 cross cycle boundaries inside and
    between calls."""
    s = W.fluid_rods(dipole_mode=mode)
    o = Oracle(s)
    o.run(37)
    with bpm.Simulation(s, precision=W.PRECISION_FP64) as sim:
        for k in (3, 14, 20):
            sim.step(k)
        x, q, v, w, t = sim.get_state()
        r, u = sim.lbm_fields()
        f, tau = sim.forces()
    xo, qo, vo, wo, to_ = o.state()
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    ro, uo = o.lbm_macro()
    assert np.abs(r - ro).max() <= 1e-9 and np.abs(u - uo).max() <= 1e-9 * np.abs(uo).max()
    fo, tauo = o.forces()
    assert rel(f, fo) <= 1e-9 and rel(tau, tauo) <= 1e-9, (rel(f, fo), rel(tau, tauo))
    # non-vacuous: the coupling matters
    s0 = s.copy()
    s0.lbm.coupled = np.zeros(s.n, np.uint8)
    o0 = Oracle(s0)
    o0.run(37)
    assert np.abs(o0.state()[2] - vo).max() > 1e-4 * np.abs(vo).max()


def test_fluid_arguments(bpm):
    s = fluid_only()
    bad = s.copy()
    bad.dt = 0.3
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    bad = s.copy()
    bad.lbm.tau = 0.5
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)
    with bpm.Simulation(s) as sim:
        with pytest.raises(bpm.BpmError):
            sim.adjoint_begin(4, 2)
    plain = W.straight_rod()
    with bpm.Simulation(plain) as sim:
        with pytest.raises(bpm.BpmError):
            bpm.bpm_lbm_fields(sim.h, 8)


@pytest.mark.parametrize("precision,tol", [(W.PRECISION_FP64, 1e-10), (W.PRECISION_FF, 1e-10),
                                           (W.PRECISION_MIXED, 1e-5)])
def test_full_size_fluid_cilia_one_cycle(bpm, precision, tol):
    """The bench's fluid workload at full size (256 x 256 x 128 lattice,
    8,388,608 nodes; 256 cilia of 64 particles): one whole cycle (10 steps
    and the LBM step) against the oracle, all particles and all nodes."""
    s = W.fluid_cilia(precision=precision)
    o = Oracle(s)
    o.run(10)
    with bpm.Simulation(s) as sim:
        sim.step(10)
        x, q, v, w, t = sim.get_state()
        r, u = sim.lbm_fields()
    xo, qo, vo, wo, to_ = o.state()
    assert np.abs(x - xo).max() <= tol * np.abs(xo).max()
    assert np.abs(v - vo).max() <= tol * np.abs(vo).max() * 10
    ro, uo = o.lbm_macro()
    assert np.abs(r - ro).max() <= tol, np.abs(r - ro).max()
    assert np.abs(u - uo).max() <= tol * np.abs(uo).max(), np.abs(u - uo).max() / np.abs(uo).max()
