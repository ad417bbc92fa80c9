"""FP64 parity bounds of the GPU tests against the CPU FP64 oracle.

Two checks on the same state, for forces and torques separately:

* norm-wise relative error ||dF|| <= rel ||F||, with rel = 1e-12 (the FP64
  target) on every workload but the twisted helix, where rel = 5e-12.  The
  helix carries particle rotations of up to 4 pi, so each bond's unit vector
  rotated into the central frame is only known to a few eps in absolute
  terms; the oracle itself sits 9.7e-13 from a longdouble evaluation of the
  300-particle helix (tests/test_oracle_precision.py), and the GPU 2.5e-12
  from the oracle at 16384 particles;
* per particle, condition-aware: |dF_i| <= 1e-12 S_i, where S_i is the sum of
  the magnitudes of every term that particle i's force adds up (each bond end,
  Zeeman, each dipole pair, damping; ``Oracle.term_scales``).  The magnetic
  torque m_i x B(x_i) is the cross product of a summed field, so its terms
  count as |m_i| |B_j(x_i)|: along a chain the near neighbours' fields are
  almost parallel to m_i, and m_i x B_j alone would hide the cancellation
  inside the field sum.  The oracle sits at most 2.5e-13 S_i from longdouble
  on the helices, so this needs no rounding floor on any workload, and one
  wrong particle cannot hide in a norm over the whole system.
"""
import numpy as np

TOL64 = 1e-12
TOL64_HELIX = 5e-12
TOL64_PARTICLE = 1e-12


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def per_particle_error(a, b, scale):
    """max_i |a_i - b_i| / scale_i (0 where both the difference and the scale
    vanish)."""
    d = np.linalg.norm(np.asarray(a) - np.asarray(b), axis=1)
    s = np.asarray(scale, dtype=np.float64)
    out = np.zeros_like(d)
    nz = s > 0
    out[nz] = d[nz] / s[nz]
    out[~nz & (d > 0)] = np.inf
    return float(out.max()) if len(out) else 0.0


def check_fp64(f, t, fo, to, orc, idx=None, norm_rel=TOL64, sample=None, seed=0):
    """FP64 parity of (f, t) against the oracle's (fo, to).  ``orc`` is an
    oracle of the whole system holding the compared state; ``idx`` lists the
    particles that f, t, fo, to hold (default: all).  ``sample`` limits the
    per-particle check to that many of them, chosen at random (for systems
    whose term scales would take long on the host)."""
    assert rel(f, fo) <= norm_rel, f"force: norm-wise rel {rel(f, fo):.3e} > {norm_rel:.1e}"
    assert rel(t, to) <= norm_rel, f"torque: norm-wise rel {rel(t, to):.3e} > {norm_rel:.1e}"
    rows = np.arange(len(fo))
    if sample is not None and sample < len(rows):
        rows = np.sort(np.random.default_rng(seed).choice(len(rows), sample, replace=False))
    pidx = rows if idx is None else np.asarray(idx)[rows]
    Sf, St = orc.term_scales(pidx)
    ef = per_particle_error(f[rows], fo[rows], Sf)
    et = per_particle_error(t[rows], to[rows], St)
    assert ef <= TOL64_PARTICLE, f"force: per-particle |dF_i|/S_i {ef:.3e} > {TOL64_PARTICLE:.0e}"
    assert et <= TOL64_PARTICLE, f"torque: per-particle |dT_i|/S_i {et:.3e} > {TOL64_PARTICLE:.0e}"
    return ef, et
