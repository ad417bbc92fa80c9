"""Every optional term at once against the oracle: overlapping rods with
contact and bond damping, dipoles and a field, immersed in the fluid (lattice
units, soft materials).  Split calls cross LBM cycles and CUDA-graph
replays; timing mode (per-kernel launches) must give the same trajectory as
the graph path to rounding (the fluid reaction is summed with atomics)."""
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


def combined(seed=71, mode=W.DIPOLE_PER_ROD, precision=W.PRECISION_FP64):
    s = W.crossing_rods(seed=seed, dipole_mode=mode, dt=0.1)
    s.precision = precision
    s.E = np.full(s.n_rods, 1.0)
    s.m_body = 0.02 * s.m_body
    s.B = 0.05 * s.B
    s.contact = W.ContactParams(E=20.0, nu=0.3, mu=0.4, gamma_n=0.05, gamma_t=0.02, exclude=3)
    rng = np.random.default_rng(seed)
    s.bond_damping = np.tile([0.05, 0.02, 0.002, 0.002], (s.n_rods, 1))
    lo = s.x.min(axis=0) - 4
    s.x = s.x - lo
    s.x_rest = s.x_rest - lo
    n = tuple(int(v) for v in np.ceil(s.x.max(axis=0) + 4))
    s.lbm = W.LbmParams(nx=n[0], ny=n[1], nz=n[2], n_sub=10, tau=0.8, body_force=np.array([1e-5, 0, 0]),
                        u0=W._smooth_field(rng, n, amp=0.005))
    return s


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("mode", [W.DIPOLE_PER_ROD, W.DIPOLE_GLOBAL])
def test_all_terms_split_calls(bpm, mode):
    s = combined(mode=mode)
    o = Oracle(s)
    f0o, t0o = o.forces()
    o.run(45)
    with bpm.Simulation(s) as sim:
        f0, t0 = sim.forces()
        assert rel(f0, f0o) <= 1e-12 and rel(t0, t0o) <= 1e-12
        for k in (7, 16, 22):
            sim.step(k)
        x, q, v, w, t = sim.get_state()
        r, u = sim.lbm_fields()
        e = sim.energy()
    xo, qo, vo, wo, to_ = o.state()
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()
    assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
    ro, uo = o.lbm_macro()
    assert np.abs(u - uo).max() <= 1e-9 * np.abs(uo).max()
    eo = o.energy()
    assert np.allclose(e, eo, rtol=1e-9, atol=1e-12 * np.abs(eo).max())


def test_timing_mode_matches_graphs(bpm):
    s = combined(seed=72)
    runs = []
    for timing in (False, True):
        with bpm.Simulation(s) as sim:
            sim.set_timing(timing)
            sim.step(13)
            sim.step(12)
            runs.append(sim.get_state()[:4])
            if timing:
                tm = sim.timing()
                assert {"bond", "dipole", "integrate", "contact", "lbm"} <= set(tm)
                assert tm["lbm"]["launches"] == 2
    for a, b in zip(*runs):
        assert np.abs(np.asarray(a) - np.asarray(b)).max() <= 1e-12 * max(np.abs(np.asarray(b)).max(), 1e-30)


def test_all_terms_mixed_precision(bpm):
    s = combined(seed=73, mode=W.DIPOLE_GLOBAL, precision=W.PRECISION_MIXED)
    o = Oracle(s)
    with bpm.Simulation(s) as sim:
        f, t = sim.forces()
        fo, to = o.forces()
        assert rel(f, fo) <= 1e-5 and rel(t, to) <= 1e-5
        sim.step(20)
        o.run(20)
        x = sim.get_state()[0]
        r, u = sim.lbm_fields()
    xo = o.state()[0]
    ro, uo = o.lbm_macro()
    assert np.abs(x - xo).max() <= 1e-6 * np.abs(xo).max()
    assert np.abs(u - uo).max() <= 1e-4 * np.abs(uo).max()
