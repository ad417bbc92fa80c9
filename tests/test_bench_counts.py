"""The bench's unit of bond work: the oracle's operation count per bond.

tests/kernels/count_oracle_bond_ops.cpp compiles oracle/bpm_oracle.c with a
number type that counts every FP64 +, -, x and / of one bond's force and
torque; bench.py divides by that count (square roots and atan2 apart)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bond_operation_count_matches_the_oracle(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "count_bond"
    subprocess.run([gxx, "-std=c++17", "-O0", "-w", "-I", os.path.join(ROOT, "oracle"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "kernels", "count_oracle_bond_ops.cpp")], check=True)
    ops, sqrts, atan2s = (int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split())
    import bench
    assert ops == bench.BOND_FLOPS_ORACLE
    assert (sqrts, atan2s) == (9, 4)
