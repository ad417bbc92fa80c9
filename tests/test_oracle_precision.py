"""Rounding floor of FP64 force evaluation (measured on the oracle).

The twisted helix carries large absolute particle rotations; each bond force
then has an absolute FP64 rounding error of order eps * (K_r + K_s) L,
independent of how small the deformation is.  These tests measure the
oracle's FP64 error against a longdouble evaluation of the same equations:
norm-wise it stays within that floor; per particle it stays within a quarter
of the 1e-12 condition-aware bound of the GPU parity tests (tests/_parity.py),
which therefore needs no floor."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import per_particle_error
from _xprec import bond_scales, forces_extended, fp64_tolerance


@pytest.mark.parametrize("make", [lambda: W.helix(300), lambda: W.straight_rod(),
                                  lambda: W.random_rods([2, 33, 64], seed=7, with_gradient=False,
                                                        with_rotating=False, vel_sigma=0.0)])
def test_oracle_fp64_error_within_rounding_floor(make):
    s = make()
    s.damping = 0.0
    s.v[:] = 0.0
    s.omega[:] = 0.0
    o = Oracle(s)
    f, t = o.forces()
    fx, tx = forces_extended(s)
    sf, st = bond_scales(o)
    assert np.linalg.norm(f - fx) <= fp64_tolerance(fx, sf, rel=1e-13, k_eps=1.0)
    assert np.linalg.norm(t - tx) <= fp64_tolerance(tx, st, rel=1e-13, k_eps=1.0)
    # per particle, against the sum of the magnitudes of the force terms
    Sf, St = o.term_scales()
    assert per_particle_error(f, fx, Sf) <= 2.5e-13
    assert per_particle_error(t, tx, St) <= 2.5e-13


def test_helix_needs_the_floor():
    """The plain 1e-12 relative bar is below FP64's own rounding for the
    twisted helix: the oracle's error against longdouble exceeds 1e-13 |F|."""
    s = W.helix(300)
    f, _ = Oracle(s).forces()
    fx, _ = forces_extended(s)
    assert np.linalg.norm(f - fx) > 1e-13 * np.linalg.norm(fx)


def test_term_scales_bound_the_summed_force():
    """The condition scale of a particle is the sum of the magnitudes of the
    terms its force adds up, so it bounds |F_i| (triangle inequality); a lone
    pair of dipoles has the force scale |F_12| and the torque scale
    |m_1| |B_2(x_1)| exactly."""
    s = W.random_rods([3, 40, 17], seed=31)
    o = Oracle(s)
    f, t = o.forces()
    Sf, St = o.term_scales()
    assert np.all(np.linalg.norm(f, axis=1) <= Sf * (1 + 1e-12))
    assert np.all(np.linalg.norm(t, axis=1) <= St * (1 + 1e-12))
    pair = W.random_rods([1, 1], seed=32, with_gradient=False, with_rotating=False, vel_sigma=0.0)
    pair.damping = 0.0
    pair.B = np.zeros(3)
    pair.B_rod = None
    op = Oracle(pair)
    fp, tp, mp = op.forces(want_m=True)
    Sp, Tp = op.term_scales()
    _, _, H = op.dipole_sample(np.arange(2), m=mp)
    assert np.allclose(Sp, np.linalg.norm(fp, axis=1), rtol=1e-14)
    assert np.allclose(Tp, np.linalg.norm(mp, axis=1) * np.linalg.norm(H, axis=1), rtol=1e-14)
    assert np.all(np.linalg.norm(tp, axis=1) <= Tp * (1 + 1e-14))
