"""GPU parity: the CUDA library (through the C ABI) against the CPU FP64 oracle
on the same seeded inputs.

Tolerances: FP64 path, norm-wise relative force and torque error <= 1e-12
(5e-12 on the twisted helix) and, per particle, |dF_i| <= 1e-12 times the sum
of the magnitudes of the particle's force terms (tests/_parity.py);
FP32-pair (mixed) path <= 1e-5 norm-wise.  Trajectories are compared over a
stated horizon with the bound written in each test.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import TOL64_HELIX, check_fp64, rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-5


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


def forces_both(bpm, sysm, precision=None, plan=None):
    with bpm.Simulation(sysm, precision=precision) as sim:
        if plan is not None:
            sim.set_dipole_plan(*plan)
        f, t = sim.forces()
    fo, to = Oracle(sysm).forces()
    return f, t, fo, to


FP64_CASES = {
    "straight_rod_64": lambda: W.straight_rod(),
    "random_rods_ragged_global": lambda: W.random_rods([1, 2, 3, 31, 32, 33, 61, 130, 257], seed=7),
    "random_rods_per_rod_field": lambda: W.random_rods([5, 40, 129, 300], seed=8, per_rod_field=True,
                                                       dipole_mode=W.DIPOLE_PER_ROD),
    "random_rods_no_dipole": lambda: W.random_rods([17, 64, 65], seed=9, dipole_mode=W.DIPOLE_OFF),
    "helix_300": lambda: W.helix(300),
    "cilia_2x3x40_fp64": lambda: W.cilia(2, 3, 40, precision=W.PRECISION_FP64),
    "batched_12_fp64": lambda: W.batched_rods(12, 16, 100, precision=W.PRECISION_FP64),
}


# dipole work decompositions: autotuned, ordered pairs with a j-split, and
# the symmetric kernel with warp tiles of 32 and 1, 2 and 8 tiles per supertile
PLANS = {"auto": (0, 0), "ordered3": (1, 3), "symw": (2, 0), "sym1": (2, 1), "sym2": (2, 2), "sym8": (2, 8)}


@pytest.mark.parametrize("plan", sorted(PLANS))
@pytest.mark.parametrize("case", sorted(FP64_CASES))
def test_fp64_forces_match_oracle(bpm, case, plan):
    sysm = FP64_CASES[case]()
    kind, param = PLANS[plan]
    if kind == 1 and sysm.dipole_mode == W.DIPOLE_PER_ROD:
        param = 50  # j-chunk length in particles
    f, t, fo, to = forces_both(bpm, sysm, precision=W.PRECISION_FP64, plan=(kind, param))
    check_fp64(f, t, fo, to, Oracle(sysm), norm_rel=TOL64_HELIX if case.startswith("helix") else TOL64)


MIXED_CASES = {
    "cilia_2x3x40": lambda: W.cilia(2, 3, 40),
    "batched_12": lambda: W.batched_rods(12, 16, 300),
    "helix_2000": lambda: W.helix(2000),
    "random_rods_ragged": lambda: W.random_rods([1, 2, 33, 257, 600], seed=10),
}


MIXED_PLANS = {"auto": (0, 0), "ordered2": (1, 2), "symw": (2, 0), "sym1": (2, 1), "sym2": (2, 2)}


@pytest.mark.parametrize("plan", sorted(MIXED_PLANS))
@pytest.mark.parametrize("case", sorted(MIXED_CASES))
def test_mixed_forces_match_oracle(bpm, case, plan):
    sysm = MIXED_CASES[case]()
    kind, param = MIXED_PLANS[plan]
    if kind == 1 and sysm.dipole_mode == W.DIPOLE_PER_ROD:
        param = 100
    f, t, fo, to = forces_both(bpm, sysm, precision=W.PRECISION_MIXED, plan=(kind, param))
    assert rel(f, fo) <= TOLMIX, rel(f, fo)
    assert rel(t, to) <= TOLMIX, rel(t, to)


@pytest.mark.parametrize("case", ["straight_rod_64", "random_rods_ragged_global", "random_rods_per_rod_field"])
def test_energy_matches_oracle(bpm, case):
    sysm = FP64_CASES[case]()
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        e = sim.energy()
    eo = Oracle(sysm).energy()
    scale = np.abs(eo).max()
    assert np.allclose(e, eo, rtol=1e-11, atol=1e-12 * scale), (e, eo)


def test_trajectory_straight_rod_1000_steps(bpm):
    """Config-1 rod over its full 1000-step horizon: state within 1e-9 of
    the oracle (relative to the state's scale; rounding differences grow
    only mildly in this damped system)."""
    sysm = W.straight_rod()
    o = Oracle(sysm)
    o.run(1000)
    with bpm.Simulation(sysm) as sim:
        sim.step(1000)
        x, q, v, w, t = sim.get_state()
    xo, qo, vo, wo, to_ = o.state()
    assert t == pytest.approx(to_, rel=1e-15)
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-9 * max(np.abs(vo).max(), 1e-3)
    assert np.abs(w - wo).max() <= 1e-9 * max(np.abs(wo).max(), 1e-3)


def test_trajectory_random_rods_split_calls(bpm):
    """50 steps as 1 + 16 + 33 (graph chunks, single steps and the closing
    half kick) against the oracle's 50 steps."""
    sysm = W.random_rods([3, 40, 70], seed=11, damping=0.05)
    o = Oracle(sysm)
    o.run(50)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        for n in (1, 16, 33):
            sim.step(n)
        x, q, v, w, t = sim.get_state()
    xo, qo, vo, wo, to_ = o.state()
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-9
    assert np.abs(v - vo).max() <= 1e-8 * np.abs(vo).max()


def test_state_roundtrip_with_rest_orientations(bpm):
    sysm = W.random_rods([4, 9], seed=12)
    with bpm.Simulation(sysm) as sim:
        x, q, v, w, t = sim.get_state()
        assert np.array_equal(x, sysm.x)
        qn = sysm.q / np.linalg.norm(sysm.q, axis=1, keepdims=True)
        assert np.abs(q - qn).max() < 1e-15
        assert np.array_equal(v, sysm.v) and t == sysm.t0
        # set_state then forces equals a fresh handle on the new state
        s2 = sysm.copy()
        s2.x = sysm.x + 0.01
        sim.set_state(x=s2.x, q=s2.q, v=s2.v, omega=s2.omega, t=s2.t0)
        f, tau = sim.forces()
    o2 = Oracle(s2)
    fo, to = o2.forces()
    check_fp64(f, tau, fo, to, o2)


def test_set_field_and_dipoles(bpm):
    sysm = W.random_rods([20, 33], seed=13, with_gradient=False)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        sim.forces()
        s2 = sysm.copy()
        s2.B = np.array([0.1, -0.7, 0.3])
        s2.m_body = sysm.m_body[::-1].copy()
        sim.set_field(B=s2.B)
        sim.set_dipoles(s2.m_body)
        f, t = sim.forces()
    o2 = Oracle(s2)
    fo, to = o2.forces()
    check_fp64(f, t, fo, to, o2)


@pytest.mark.parametrize("precision,plan", [(W.PRECISION_MIXED, None), (W.PRECISION_MIXED, (2, 1)),
                                            (W.PRECISION_MIXED, (2, 0)), (W.PRECISION_FP64, (2, 1)),
                                            (W.PRECISION_FP64, (1, 4))])
def test_deterministic_bitwise(bpm, precision, plan):
    sysm = W.helix(1000)
    out = []
    for _ in range(2):
        with bpm.Simulation(sysm, precision=precision) as sim:
            if plan:
                sim.set_dipole_plan(*plan)
            sim.step(3)
            out.append(sim.forces())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_plans_agree_and_bad_plans_are_rejected(bpm):
    sysm = W.random_rods([40, 300, 7], seed=21)
    res = []
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as sim:
        for plan in [(1, 2), (2, 1), (2, 4), (2, 0), (0, 0)]:
            sim.set_dipole_plan(*plan)
            res.append(sim.forces())
        with pytest.raises(bpm.BpmError):
            sim.set_dipole_plan(2, 9)
        with pytest.raises(bpm.BpmError):
            sim.set_dipole_plan(7, 1)
    for f, t in res[1:]:
        assert rel(f, res[0][0]) < 1e-13 and rel(t, res[0][1]) < 1e-13
    # FP32 pairs: the warp tiles (64 particles) agree with the other plans
    res = []
    with bpm.Simulation(sysm, precision=W.PRECISION_MIXED) as sim:
        for plan in [(1, 2), (2, 1), (2, 0)]:
            sim.set_dipole_plan(*plan)
            res.append(sim.forces())
    for f, t in res[1:]:
        assert rel(f, res[0][0]) < 1e-6 and rel(t, res[0][1]) < 1e-6
    # warp tiles: not beyond 255 tiles per set
    with bpm.Simulation(W.helix(8192 + 64), precision=W.PRECISION_FP64) as sim:
        with pytest.raises(bpm.BpmError):
            sim.set_dipole_plan(2, 0)
    with bpm.Simulation(W.helix(16384 + 64), precision=W.PRECISION_MIXED) as sim:
        with pytest.raises(bpm.BpmError):
            sim.set_dipole_plan(2, 0)


def test_tuned_plan_is_reused_by_a_second_handle(bpm):
    """The autotuner's choice is cached per work shape: a second handle on
    the same system reports the same, valid plan and sums in the same order
    (per-rod systems, whose ordered candidates include chunk lengths above
    1000 and the whole rod)."""
    for seed, lengths in ((41, [1500, 3000]), (42, [700, 2100, 40]), (43, [5, 9, 12])):
        sysm = W.random_rods(lengths, seed=seed, dipole_mode=W.DIPOLE_PER_ROD)
        with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as a:
            fa, ta = a.forces()
            pa = a.dipole_plan()
        with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as b:
            fb, tb = b.forces()
            pb = b.dipole_plan()
        assert pa == pb, (pa, pb)
        kind, param = pa
        assert kind in (1, 2)
        if kind == 2:
            assert 0 <= param <= 8  # 0: warp tiles of 32
        assert np.array_equal(fa, fb) and np.array_equal(ta, tb)


def test_device_pointer_outputs(bpm):
    torch = pytest.importorskip("torch")
    sysm = W.random_rods([30, 31], seed=14)
    with bpm.Simulation(sysm) as sim:
        fh, th = sim.forces()
        fd = torch.zeros((sysm.n, 3), dtype=torch.float64, device="cuda")
        td = torch.zeros((sysm.n, 3), dtype=torch.float64, device="cuda")
        sim.forces(fd, td)
        torch.cuda.synchronize()
        assert np.array_equal(fd.cpu().numpy(), fh) and np.array_equal(td.cpu().numpy(), th)
        xd = torch.zeros((sysm.n, 3), dtype=torch.float64, device="cuda")
        bpm.bpm_get_state(sim.h, x=xd)
        assert np.array_equal(xd.cpu().numpy(), sysm.x)


def test_edge_sizes(bpm):
    # empty system
    empty = W.random_rods([1], seed=1)
    empty.rod_offset = np.array([0], dtype=np.int64)
    for k in ("x", "v", "omega", "m_body", "x_rest"):
        setattr(empty, k, np.zeros((0, 3)))
    for k in ("q", "q_rest"):
        setattr(empty, k, np.zeros((0, 4)))
    for k in ("mass", "radius"):
        setattr(empty, k, np.zeros(0))
    empty.clamped = np.zeros(0, np.uint8)
    empty.E = empty.nu = empty.d = np.zeros(0)
    empty.B_rod = None
    with bpm.Simulation(empty) as sim:
        f, t = sim.forces()
        assert f.shape == (0, 3)
        sim.step(3)
        assert np.array_equal(sim.energy(), np.zeros(5))
    for prec in (W.PRECISION_FF, W.PRECISION_MIXED):
        with bpm.Simulation(empty, precision=prec) as sim:
            f, t = sim.forces()
            assert f.shape == (0, 3)
            sim.step(3)
    # single particles and two-particle rods, every precision and the
    # symmetric plans with warp tiles and with supertiles
    for lengths in ([1], [1, 1, 1], [2], [1, 2, 1]):
        sysm = W.random_rods(lengths, seed=15)
        o = Oracle(sysm)
        fo, to = o.forces()
        for prec, plan in ((W.PRECISION_FP64, None), (W.PRECISION_FP64, (2, 0)), (W.PRECISION_FF, None),
                           (W.PRECISION_FF, (2, 0)), (W.PRECISION_FF, (2, 1))):
            f, t, _, _ = forces_both(bpm, sysm, precision=prec, plan=plan)
            check_fp64(f, t, fo, to, o)
        for plan in (None, (2, 0), (2, 1)):
            f, t, _, _ = forces_both(bpm, sysm, precision=W.PRECISION_MIXED, plan=plan)
            assert rel(f, fo) <= TOLMIX and rel(t, to) <= TOLMIX
    with bpm.Simulation(W.straight_rod()) as sim:
        sim.step(0)


@pytest.mark.parametrize("mode", [W.DIPOLE_GLOBAL, W.DIPOLE_PER_ROD])
@pytest.mark.parametrize("lengths", [[63], [64], [65], [127, 128, 129], [64, 1, 65, 33]])
def test_mixed_warp_tiles_at_tile_boundaries(bpm, lengths, mode):
    """FP32 pairs in 64-particle warp tiles (two i per lane, j halves 32
    apart) with particle counts around the tile size, in one interacting set
    and per rod, against the oracle; the supertile plan alongside."""
    sysm = W.random_rods(lengths, seed=23, dipole_mode=mode)
    o = Oracle(sysm)
    fo, to = o.forces()
    for plan in ((2, 0), (2, 1)):
        f, t, _, _ = forces_both(bpm, sysm, precision=W.PRECISION_MIXED, plan=plan)
        assert rel(f, fo) <= TOLMIX, (plan, rel(f, fo))
        assert rel(t, to) <= TOLMIX, (plan, rel(t, to))


def test_bad_descriptions_are_rejected(bpm):
    sysm = W.straight_rod()
    bad = sysm.copy()
    bad.x_rest = sysm.x_rest.copy()
    bad.x_rest[5] = bad.x_rest[4]
    with pytest.raises(bpm.BpmError) as e:
        bpm.Simulation(bad)
    assert e.value.code == bpm.BPM_ERR_SINGULAR
    bad = sysm.copy()
    bad.dt = 0.0
    with pytest.raises(bpm.BpmError) as e:
        bpm.Simulation(bad)
    assert e.value.code == bpm.BPM_ERR_ARG
    bad = sysm.copy()
    bad.rod_offset = np.array([0, 10], dtype=np.int64)
    with pytest.raises(bpm.BpmError):
        bpm.Simulation(bad)


def test_nonfinite_state_is_reported(bpm):
    """A NaN injected into host input is caught on the device and reported
    by bpm_step with BPM_ERR_NONFINITE; the handle stays usable."""
    sysm = W.straight_rod()
    with bpm.Simulation(sysm) as sim:
        x = sysm.x.copy()
        x[7, 1] = np.nan
        sim.set_state(x=x, q=sysm.q, v=sysm.v, omega=sysm.omega, t=0.0)
        with pytest.raises(bpm.BpmError) as e:
            sim.step(5)
        assert e.value.code == bpm.BPM_ERR_NONFINITE
        sim.set_state(x=sysm.x, q=sysm.q, v=sysm.v, omega=sysm.omega, t=0.0)
        sim.step(2)
        f, t = sim.forces()
        assert np.all(np.isfinite(f))


# ---------------------------------------------------------------- full sizes

@pytest.mark.parametrize("plan", [None, (2, 1), (1, 8)])
def test_full_size_helix_forces_and_10_steps(bpm, plan):
    """The 16384-particle helix (268M pairs per step) in the bench's launch
    configuration (autotuned plan) and in the symmetric and ordered plans:
    step-1 forces and a 10-step trajectory against the oracle."""
    sysm = W.helix()
    o = Oracle(sysm)
    fo, to = o.forces()
    with bpm.Simulation(sysm) as sim:
        if plan:
            sim.set_dipole_plan(*plan)
        f, t = sim.forces()
        check_fp64(f, t, fo, to, o, norm_rel=TOL64_HELIX)
        sim.step(10)
        x, q, v, w, tt = sim.get_state()
    o.run(10)
    xo, qo, vo, wo, _ = o.state()
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()
    assert np.abs(q - qo).max() <= 1e-10
    assert np.abs(v - vo).max() <= 1e-9 * np.abs(vo).max()


@pytest.mark.parametrize("plan", [None, (2, 1), (1, 8)])
def test_full_size_helix_mixed_forces(bpm, plan):
    sysm = W.helix()
    f, t, fo, to = forces_both(bpm, sysm, precision=W.PRECISION_MIXED, plan=plan)
    assert rel(f, fo) <= TOLMIX and rel(t, to) <= TOLMIX


@pytest.mark.parametrize("precision,tol", [(W.PRECISION_MIXED, TOLMIX), (W.PRECISION_FP64, TOL64)])
def test_full_size_cilia_sampled(bpm, precision, tol):
    """131072 particles (1.7e10 pairs): 96 sampled particles, whose dipole
    sums the oracle computes one by one over all partners, plus the oracle's
    O(N) bond and Zeeman terms."""
    sysm = W.cilia()
    with bpm.Simulation(sysm, precision=precision) as sim:
        f, t = sim.forces()
    rng = np.random.default_rng(0)
    idx = np.sort(np.concatenate([rng.choice(sysm.n, 90, replace=False), [0, 1, 255, 256, sysm.n - 2, sysm.n - 1]]))
    nodip = sysm.copy()
    nodip.dipole_mode = W.DIPOLE_OFF
    o = Oracle(nodip)
    fb, tb, m = o.forces(want_m=True)
    od = Oracle(sysm)
    Fd, Td, _ = od.dipole_sample(idx, m=m)
    fo = fb[idx] + Fd
    to = tb[idx] + Td
    if precision == W.PRECISION_FP64:
        check_fp64(f[idx], t[idx], fo, to, od, idx=idx)
    else:
        assert rel(f[idx], fo) <= tol, rel(f[idx], fo)
        assert rel(t[idx], to) <= tol, rel(t[idx], to)


@pytest.mark.parametrize("plan", [None, (2, 0)])
def test_full_size_batched_mixed(bpm, plan):
    """2048 rods, lengths U{16..1024}: the whole force field against the
    oracle (per-rod pairs ~7.3e8), in the tuned plan and in 64-particle warp
    tiles."""
    sysm = W.batched_rods()
    f, t, fo, to = forces_both(bpm, sysm, precision=W.PRECISION_MIXED, plan=plan)
    assert rel(f, fo) <= TOLMIX and rel(t, to) <= TOLMIX


def test_handles_with_other_plans_in_one_process():
    """Plans of different shared-memory sizes on several handles of one fresh
    process, in every precision, the smaller plan's kernel set up last: each
    handle still launches (a kernel's shared-memory limit is shared by all
    handles, so it must not follow the last plan set up)."""
    import subprocess
    import sys
    import os
    code = r"""
import sys
sys.path.insert(0, %r)
from paper_2603_27279_gb300 import bpm, workloads as W
for prec in (W.PRECISION_MIXED, W.PRECISION_FF, W.PRECISION_FP64):
    s = W.helix(3000, precision=prec)
    live = []
    for g in (8, 3, 1, 2, 8, 5):
        sim = bpm.Simulation(s)
        sim.set_dipole_plan(2, g)
        sim.forces()
        live.append(sim)
    for sim in live:
        sim.forces()
        sim.close()
print("ok")
""" % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
