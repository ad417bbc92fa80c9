"""Planted mistakes in copies of the oracle must be caught by its pins.

Each case copies oracle/bpm_oracle.c, replaces one exact line with a
plausible slip (a dropped factor, a swapped composition order, a flipped
sign), builds the copy with gcc into a temporary directory and runs the named
pin tests against it in a child pytest, which loads the copy through the
BPM_ORACLE_LIB variable of oracle/oracle.py.  The pins must fail.  The
untouched oracle passes the same pins in the ordinary run of the suite.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bpm_oracle.c")

# (name, exact original line(s), replacement(s), pytest selection that must
# fail); several lines are given as tuples
MUTATIONS = [
    # SI "Symmetric rotational decomposition": u = t_2 b_2 and u* = t_1 b_1
    # (bend before twist); the slip factors both the other way round,
    # b_2 = u t_2^* and b_1 = u^* t_1^*, which keeps psi, |theta|, the energy
    # and the exchange symmetry
    ("bend_after_twist",
     ("    quat b2 = qmul(qconj(t2), u);", "    quat b1 = qmul(qconj(t1), uc);"),
     ("    quat b2 = qmul(u, qconj(t2));", "    quat b1 = qmul(uc, qconj(t1));"),
     "tests/test_oracle_bond.py::test_combined_bend_and_twist_follow_the_bend_before_twist_decomposition"),
    # Eq. bpm-vector: tau_2 = tau_s - tau_b - tau_t
    ("tau2_sign",
     "    vstore(vsub(TS, TBT), tau2);",
     "    vstore(vadd(TS, TBT), tau2);",
     "tests/test_oracle_bond.py::test_momentum_balance_per_bond"),
    # Eq. bpm-tst: the counter torque carries 1/2 K_s r_f^2
    ("shear_torque_factor",
     "    vec3 ts = vscale(gamma_t, 0.5 * Ks * rf_len * rf_len);   /* 1/2 K_s r_f^2 gamma t^ */",
     "    vec3 ts = vscale(gamma_t, Ks * rf_len * rf_len);   /* 1/2 K_s r_f^2 gamma t^ */",
     "tests/test_oracle_bond.py::test_linear_stiffness_equals_eb_frame_element"),
    # twist angle psi = psi_2 - psi_1
    ("twist_one_sided",
     "    double psi = psi2 - psi1;",
     "    double psi = psi2;",
     "tests/test_oracle_bond.py::test_pure_twist"),
    # the dipole force's 5 a b r / r^7 term
    ("dipole_five",
     "        vec3 Fij = vscale(vsub(vscale(t1, 1.0 / r5), vscale(r, 5.0 * a * b / r7)), 3.0 * c);",
     "        vec3 Fij = vscale(vsub(vscale(t1, 1.0 / r5), vscale(r, 3.0 * a * b / r7)), 3.0 * c);",
     "tests/test_oracle_magnetic.py::test_coaxial_head_to_tail_attraction"),
    # Richardson extrapolation 2 q(2) - q(1)
    ("richardson_plain",
     "    quat qn = qnormalize(qadd(qscale(q2, 2.0), qscale(q1, -1.0)));",
     "    quat qn = qnormalize(q2);",
     "tests/test_oracle_integrator.py::test_richardson_rotor_error_constant"),
]


def _gcc():
    from shutil import which
    return which("gcc")


@pytest.mark.parametrize("name,orig,repl,select", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, orig, repl, select):
    if _gcc() is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    origs = orig if isinstance(orig, tuple) else (orig,)
    repls = repl if isinstance(repl, tuple) else (repl,)
    for o, p in zip(origs, repls):
        assert src.count(o) == 1, f"{name}: {o!r} is not in the oracle exactly once"
        src = src.replace(o, p)
    mutant = tmp_path / "bpm_oracle_mutant.c"
    mutant.write_text(src)
    lib = tmp_path / "libbpm_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mutant), "-lm"], check=True)
    env = dict(os.environ, BPM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", select],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"{name}: the pins did not catch the planted mistake\n{r.stdout[-2000:]}"
