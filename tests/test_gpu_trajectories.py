"""Trajectories of the full-size workloads against the CPU FP64 oracle.

* The 2048 batched rods (1.07M particles) over their 200-step horizon,
  replayed from CUDA graphs as bpm_step(200) does: the rods do not interact
  (per-rod dipoles), so the oracle runs 16 rods cut out of the batch and
  those rods are compared.
* The cilia array (131072 particles, 1.7e10 pairs per step) over steps 1 and
  2: the oracle runs the whole system (three force passes on the host cores),
  and both the FP64 and the FP32-pair paths are compared, positions and
  velocities as displacements from the initial state.

Bounds: FP64 and float-float paths, the change of position and orientation
from the initial state within 1e-9 of the largest change, the velocity within
1e-9 of the largest velocity; FP32-pair path, 1e-4 of the same scales (its
forces carry up to 1e-5 relative error).
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


def _change_error(a, ao, a0):
    """max |(a - a0) - (ao - a0)| over max |ao - a0|: the error of the change
    from the initial state, relative to the largest change."""
    return np.abs(a - ao).max() / np.abs(ao - a0).max()


def _compare(s0, x, xo, v, vo, q, qo, tol, what):
    ex = _change_error(x, xo, s0.x)
    eq = _change_error(q, qo, s0.q / np.linalg.norm(s0.q, axis=1, keepdims=True))
    ev = np.abs(v - vo).max() / np.abs(vo).max()
    assert ex <= tol and ev <= tol and eq <= tol, \
        f"{what}: displacement {ex:.3e}, velocity {ev:.3e}, rotation {eq:.3e} (bound {tol:.0e})"
    return ex, ev, eq


@pytest.fixture(scope="module")
def batched_oracle():
    sysm = W.batched_rods(precision=W.PRECISION_FP64)
    rng = np.random.default_rng(3)
    lens = np.diff(sysm.rod_offset)
    # the shortest and the longest rods and a random 14
    rods = np.unique(np.concatenate([[int(np.argmin(lens)), int(np.argmax(lens)), 0, sysm.n_rods - 1],
                                     rng.choice(sysm.n_rods, 12, replace=False)]))
    sub = W.subset_rods(sysm, rods)
    o = Oracle(sub)
    o.run(sysm.n_steps)
    offs = sysm.rod_offset
    idx = np.concatenate([np.arange(offs[r], offs[r + 1]) for r in rods])
    return sysm, idx, sub, o.state()


@pytest.mark.parametrize("precision,tol", [(W.PRECISION_FP64, 1e-9), (W.PRECISION_MIXED, 1e-4),
                                           (W.PRECISION_FF, 1e-9)])
def test_batched_rods_200_graph_steps(bpm, batched_oracle, precision, tol):
    sysm, idx, sub, (xo, qo, vo, wo, to_) = batched_oracle
    with bpm.Simulation(sysm, precision=precision) as sim:
        sim.step(sysm.n_steps)  # graph chunks of 16 steps, single-step graphs, closing half kick
        x, q, v, w, t = sim.get_state()
    assert t == pytest.approx(to_, rel=1e-14)
    _compare(sub, x[idx], xo, v[idx], vo, q[idx], qo, tol, f"batched rods, precision {precision}")


@pytest.fixture(scope="module")
def cilia_oracle():
    sysm = W.cilia(precision=W.PRECISION_FP64)
    o = Oracle(sysm)
    o.run(2)
    return sysm, o.state()


@pytest.mark.parametrize("precision,tol", [(W.PRECISION_FP64, 1e-9), (W.PRECISION_MIXED, 1e-4)])
def test_cilia_steps_1_and_2(bpm, cilia_oracle, precision, tol):
    sysm, (xo, qo, vo, wo, to_) = cilia_oracle
    with bpm.Simulation(sysm, precision=precision) as sim:
        sim.step(2)
        x, q, v, w, t = sim.get_state()
    _compare(sysm, x, xo, v, vo, q, qo, tol, f"cilia, precision {precision}")
    ew = np.abs(w - wo).max() / np.abs(wo).max()
    assert ew <= tol, ew
