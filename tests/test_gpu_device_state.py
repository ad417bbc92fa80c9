"""Handles over caller-owned device state (bpm_create_device) and the
carrying of forces across a state upload (bpm_set_forces / bpm_get_forces),
through the C ABI, against the CPU FP64 oracle."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

from _parity import TOL64_HELIX, check_fp64, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


def _tensors(torch, sysm):
    """The system's state as (3, N) / (4, N) float64 CUDA tensors."""
    dev = torch.device("cuda")

    def soa(a):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dev).contiguous()

    n = sysm.n
    return {"x": soa(sysm.x), "q": soa(sysm.q), "v": soa(sysm.v), "omega": soa(sysm.omega),
            "f": torch.zeros((3, n), dtype=torch.float64, device=dev),
            "tau": torch.zeros((3, n), dtype=torch.float64, device=dev)}


CASES = {
    "straight_rod_64": lambda: W.straight_rod(),
    "helix_300": lambda: W.helix(300),
    "cilia_2x3x40": lambda: W.cilia(2, 3, 40, precision=W.PRECISION_FP64),
    "batched_12_mixed": lambda: W.batched_rods(12, 16, 100),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_device_state_handle_works_in_place(bpm, case):
    torch = pytest.importorskip("torch")
    sysm = CASES[case]()
    st = _tensors(torch, sysm)
    fp64 = sysm.precision == W.PRECISION_FP64
    o = Oracle(sysm)
    fo, to = o.forces()
    with bpm.Simulation(sysm, device_state=st) as sim:
        f, t = sim.forces()
        torch.cuda.synchronize()
        # the caller's f and tau tensors hold the same forces, component-major
        assert np.array_equal(st["f"].cpu().numpy().T, f) and np.array_equal(st["tau"].cpu().numpy().T, t)
        if fp64:
            check_fp64(f, t, fo, to, o, norm_rel=TOL64_HELIX if case.startswith("helix") else 1e-12)
        else:
            assert rel(f, fo) <= 1e-5 and rel(t, to) <= 1e-5
        sim.step(10)
        x, q, v, w, tt = sim.get_state()
        torch.cuda.synchronize()
        # the state advanced in the caller's tensors
        assert np.array_equal(st["x"].cpu().numpy().T, x) and np.array_equal(st["q"].cpu().numpy().T, q)
        assert np.array_equal(st["v"].cpu().numpy().T, v) and np.array_equal(st["omega"].cpu().numpy().T, w)
        ff, tf = sim.get_forces()
        assert np.array_equal(st["f"].cpu().numpy().T, ff)
    o.run(10)
    xo, qo, vo, wo, _ = o.state()
    tol = 1e-10 if fp64 else 1e-7
    assert np.abs(x - xo).max() <= tol * np.abs(xo).max()
    assert np.abs(q - qo).max() <= tol
    # the handle is gone, the tensors are the caller's and still hold the state
    assert np.array_equal(st["x"].cpu().numpy().T, x)


def test_device_state_handle_matches_the_owning_handle_bitwise(bpm):
    """The same kernels on the same data: a handle over caller tensors and a
    handle that owns its arrays give the same bits over a graph-replayed run."""
    torch = pytest.importorskip("torch")
    sysm = W.random_rods([40, 33, 2, 90], seed=51, damping=0.05)
    sysm.q_rest = np.tile([1.0, 0.0, 0.0, 0.0], (sysm.n, 1))
    st = _tensors(torch, sysm)
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64) as a:
        a.step(37)
        xa, qa, va, wa, _ = a.get_state()
    with bpm.Simulation(sysm, precision=W.PRECISION_FP64, device_state=st) as b:
        b.step(37)
        xb, qb, vb, wb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(qa, qb) and np.array_equal(va, vb) and np.array_equal(wa, wb)


def test_device_state_rejects_host_pointers_and_rest_orientations(bpm):
    torch = pytest.importorskip("torch")
    sysm = W.straight_rod()
    st = _tensors(torch, sysm)
    desc, keep = bpm.make_desc(sysm)
    desc.x = desc.q = desc.v = desc.omega = None
    desc.q_rest = None
    host = np.zeros((3, sysm.n))
    s = bpm.bpm_device_state()
    import ctypes as C
    for k in ("x", "q", "v", "omega", "f", "tau"):
        setattr(s, k, C.cast(C.c_void_p(st[k].data_ptr()), C.POINTER(C.c_double)))
    s.v = host.ctypes.data_as(C.POINTER(C.c_double))
    with pytest.raises(bpm.BpmError) as e:
        bpm.bpm_create_device(desc, s)
    assert e.value.code == bpm.BPM_ERR_ARG and "st->v" in str(e.value)
    s.v = C.cast(C.c_void_p(st["v"].data_ptr()), C.POINTER(C.c_double))
    desc.q_rest = keep[0].ctypes.data_as(C.POINTER(C.c_double))  # any non-NULL pointer
    with pytest.raises(bpm.BpmError) as e:
        bpm.bpm_create_device(desc, s)
    assert e.value.code == bpm.BPM_ERR_ARG
    desc.q_rest = None
    h = bpm.bpm_create_device(desc, s)
    bpm.bpm_destroy(h)
    del keep


@pytest.mark.parametrize("precision", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_restart_with_carried_forces_continues_the_run(bpm, precision):
    """A run stopped after 9 steps and restarted on a fresh handle from the
    saved state and forces (bpm_set_state + bpm_set_forces) continues as the
    uninterrupted run does, without a force evaluation at the restart."""
    sysm = W.random_rods([40, 33, 90], seed=52, damping=0.05, with_gradient=False)
    with bpm.Simulation(sysm, precision=precision) as a:
        a.step(9)
        x, q, v, w, t = a.get_state()
        f, tau = a.get_forces()
        a.step(12)
        xa, qa, va, wa, _ = a.get_state()
    with bpm.Simulation(sysm, precision=precision) as b:
        with pytest.raises(bpm.BpmError):
            b.get_forces()  # nothing evaluated yet
        b.set_state(x, q, v, w, t)
        b.set_forces(f, tau)
        f2, tau2 = b.get_forces()
        assert np.array_equal(f2, f) and np.array_equal(tau2, tau)
        b.step(12)
        xb, qb, vb, wb, _ = b.get_state()
    assert np.abs(xb - xa).max() <= 1e-13 * np.abs(xa).max()
    assert np.abs(qb - qa).max() <= 1e-13
    assert np.abs(vb - va).max() <= 1e-12 * np.abs(va).max()
