"""The FP64 parity check of the GPU tests (tests/_parity.py) exercised on the
CPU: a single wrong particle that a whole-system norm would let through is
caught per particle, and the oracle compared with itself passes."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import TOL64_HELIX, check_fp64, rel


def test_one_wrong_particle_is_caught_per_particle():
    s = W.helix(2000)
    o = Oracle(s)
    fo, to = o.forces()
    check_fp64(fo.copy(), to.copy(), fo, to, o, norm_rel=TOL64_HELIX)
    # an interior particle of the helix nets a force ~50x below its terms:
    # an error of 2e-12 of its terms stays under the norm-wise bound
    Sf, _ = o.term_scales()
    i = int(np.argmax(Sf / np.maximum(np.linalg.norm(fo, axis=1), 1e-300)))
    bad = fo.copy()
    bad[i, 0] += 2e-12 * Sf[i]
    assert rel(bad, fo) <= TOL64_HELIX
    with pytest.raises(AssertionError, match="per-particle"):
        check_fp64(bad, to.copy(), fo, to, o, norm_rel=TOL64_HELIX)


def test_sampled_per_particle_check_uses_the_sampled_rows():
    s = W.cilia(2, 3, 40, precision=W.PRECISION_FP64)
    o = Oracle(s)
    fo, to = o.forces()
    idx = np.array([0, 5, 39, 40, 200, s.n - 1])
    check_fp64(fo[idx].copy(), to[idx].copy(), fo[idx], to[idx], o, idx=idx)
    bad = fo[idx].copy()
    Sf, _ = o.term_scales(idx)
    bad[3, 2] += 3e-12 * Sf[3]
    with pytest.raises(AssertionError, match="per-particle"):
        check_fp64(bad, to[idx].copy(), fo[idx], to[idx], o, idx=idx, norm_rel=1.0)
