"""Rounding floor of FP64 force evaluation (measured on the oracle).

The twisted helix carries large absolute particle rotations; each bond force
then has an absolute FP64 rounding error of order eps * (K_r + K_s) L,
independent of how small the deformation is.  These tests measure the
oracle's FP64 error against a longdouble evaluation of the same equations and
check it against that floor; the GPU parity tests use the same bound."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

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


def test_helix_needs_the_floor():
    """The plain 1e-12 relative bar is below FP64's own rounding for the
    twisted helix: the oracle's error against longdouble exceeds 1e-13 |F|."""
    s = W.helix(300)
    f, _ = Oracle(s).forces()
    fx, _ = forces_extended(s)
    assert np.linalg.norm(f - fx) > 1e-13 * np.linalg.norm(fx)
