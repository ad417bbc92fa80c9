"""The library's hand-built device math (csrc/bpm_devmath.cuh) against
correctly rounded references: rsqrt_nr and rcp_nr (FP32 hardware seeds made
from the high word, one refinement in FP64) within 2 ulp of 1/sqrt(a) and 1/a
on a million log-uniform inputs over [2^-125, 2^126), the edges of their fast
range and the inputs that take the IEEE fallback; atan_over (the Taylor series
of atan(u)/u for small angles, the library atan2 otherwise) within 4 ulp of
atan2(sqrt(t), c)/sqrt(t) on both sides of its branch points.  References in
numpy longdouble on the host.  The test kernel is built by nvcc from
tests/kernels/devmath_probe.cu."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
L = np.longdouble


@pytest.fixture(scope="module")
def devmath(tmp_path_factory):
    torch = pytest.importorskip("torch")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = tmp_path_factory.mktemp("devmath") / "libdevmath.so"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-o", str(out), os.path.join(HERE, "kernels", "devmath_probe.cu")],
                   check=True)
    lib = ctypes.CDLL(str(out))
    lib.devmath_eval.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5
    lib.devmath_eval.restype = ctypes.c_int

    def run(a, c):
        a_d = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        c_d = torch.from_numpy(np.ascontiguousarray(c, dtype=np.float64)).cuda()
        outs = [torch.empty_like(a_d) for _ in range(3)]
        rc = lib.devmath_eval(len(a), a_d.data_ptr(), c_d.data_ptr(), *[o.data_ptr() for o in outs])
        assert rc == 0, rc
        return [o.cpu().numpy() for o in outs]
    return run


def ulp_err(got, ref):
    """|got - ref| in units of the last place of the FP64 reference."""
    ref64 = ref.astype(np.float64)
    return np.abs(got.astype(L) - ref) / np.spacing(np.abs(ref64)).astype(L)


def test_rsqrt_and_rcp_within_two_ulp(devmath):
    rng = np.random.default_rng(5)
    a = np.exp2(rng.uniform(-125, 126, 1_000_000))
    # the edges of the fast range (high words 0x38200000 and 0x47D00000) and
    # inputs that take the IEEE fallback
    edges = []
    for hi in (0x38200000, 0x47D00000):
        for d in (-2, -1, 0, 1, 2):
            edges.append(np.array([(hi + d) << 32], dtype=np.uint64).view(np.float64)[0])
            edges.append(np.array([((hi + d) << 32) | 0xFFFFFFFF], dtype=np.uint64).view(np.float64)[0])
    edges += [2.0 ** -1000, 2.0 ** -126, 1e-300, 1.0, 1.5, 2.0 ** 126, 2.0 ** 500, 1e300]
    a = np.concatenate([a, np.array(edges)])
    rs, rc, _ = devmath(a, np.ones_like(a))
    aL = a.astype(L)
    e_rs = ulp_err(rs, L(1) / np.sqrt(aL))
    e_rc = ulp_err(rc, L(1) / aL)
    assert e_rs.max() <= 2.0, (e_rs.max(), a[np.argmax(e_rs)])
    assert e_rc.max() <= 2.0, (e_rc.max(), a[np.argmax(e_rc)])


def test_atan_over_within_four_ulp(devmath):
    rng = np.random.default_rng(6)
    c = rng.uniform(0.5, 1.5, 400_000)
    # u^2 = t / c^2 log-uniform over [1e-30, 1]: the 4-term series below
    # 1e-4, the 8-term series below 1e-2, atan2 above, and the branch points
    u2 = np.concatenate([np.exp(rng.uniform(np.log(1e-30), 0.0, 399_980)),
                         np.repeat([1e-4 * (1 - 1e-12), 1e-4, 1e-4 * (1 + 1e-12), 1e-2 * (1 - 1e-12), 1e-2], 4)])
    t = u2 * c * c
    _, _, at = devmath(t, c)
    tL, cL = t.astype(L), c.astype(L)
    s = np.sqrt(tL)
    ref = np.arctan2(s, cL) / s
    e = ulp_err(at, ref)
    assert e.max() <= 4.0, (e.max(), t[np.argmax(e)], c[np.argmax(e)])
    # the limit 1/c at t = 0
    _, _, at0 = devmath(np.zeros(3), np.array([0.5, 1.0, 3.0]))
    assert np.allclose(at0, [2.0, 1.0, 1.0 / 3.0], rtol=1e-15)
