"""bpm_dipole_forces_noalloc: the allocation-free dipole entry point.

Some callers cannot call cudaMalloc (a host whose caching allocator already
holds the device memory, or a fixed-latency loop that must not allocate), so
the library offers its FP64 all-pairs dipole kernel with scratch held in a
fixed array of the library's device image.  These tests call it through the
C ABI, two calls in a row for each case, and check each result against the
handle-based entry point (bpm_forces on the same dipoles) within the FP64
parity tolerance of the other GPU tests, and against the CPU FP64 oracle's
dipole sums.  They also check that a warmed-up call changes the device's free
memory by nothing, and that host pointers and short buffers are refused
before any launch.  The file is collected last, and its tests pass both alone
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from _parity import TOL64, rel

pytestmark = pytest.mark.gpu


def _loose_dipoles(n, seed):
    """n unbonded particles (rods of length 1) with random dipoles on a
    jittered grid: bpm_forces then returns the dipole-dipole terms only."""
    from paper_2603_27279_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    side = int(np.ceil(n ** (1 / 3)))
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    x = 1.5 * g + 0.2 * rng.standard_normal((n, 3))
    m = rng.standard_normal((n, 3))
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    s = W.RodSystem(name="loose", rod_offset=np.arange(n + 1, dtype=np.int64), x=x, q=q,
                    v=np.zeros((n, 3)), omega=np.zeros((n, 3)), mass=np.ones(n), radius=np.full(n, 0.5),
                    m_body=m, clamped=np.zeros(n, np.uint8), x_rest=x.copy(), q_rest=q.copy(),
                    E=np.ones(n), nu=np.full(n, 0.3), d=np.ones(n), mu0_over_4pi=1.3,
                    dipole_mode=W.DIPOLE_GLOBAL, damping=0.0)
    return s


@pytest.fixture(scope="module")
def lib():
    pytest.importorskip("torch")
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm
    bpm.load()
    return bpm


def _noalloc(bpm, torch, s):
    n = s.n
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(s.x)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(s.m_body)).to(dev)
    f = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
    t = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
    bpm.bpm_dipole_forces_noalloc(n, x, m, s.mu0_over_4pi, f, t, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy(), t.cpu().numpy()


# pairs of sizes called in a row: the second call of each pair follows one
# with other sizes, so stale scratch from the first is present; n < 4 leaves
# j-chunks empty, whose slots must be written as zeros; 32768 fills the array
SIZE_PAIRS = [(3001, 2500), (1, 2), (3, 129), (32768, 129)]


@pytest.mark.parametrize("sizes", SIZE_PAIRS, ids=[f"{a}_then_{b}" for a, b in SIZE_PAIRS])
def test_noalloc_matches_handle_path_and_oracle_on_two_calls(lib, sizes):
    torch = pytest.importorskip("torch")
    from oracle import Oracle
    bpm = lib
    for call, n in enumerate(sizes):
        s = _loose_dipoles(n, seed=100 + 7 * n + call)
        fn, tn = _noalloc(bpm, torch, s)
        assert np.all(np.isfinite(fn)) and np.all(np.isfinite(tn))
        if n == 1:
            # a lone dipole has no partner
            assert np.array_equal(fn, np.zeros((1, 3))) and np.array_equal(tn, np.zeros((1, 3)))
            continue
        # the existing entry point: bpm_forces of a handle over the same dipoles
        with bpm.Simulation(s, precision=bpm.BPM_FP64) as sim:
            f_ref, t_ref = sim.forces()
        assert rel(fn, f_ref) <= TOL64 and rel(tn, t_ref) <= TOL64, (n, call, rel(fn, f_ref), rel(tn, t_ref))
        # the CPU FP64 oracle: every particle, or a sample at the largest size
        o = Oracle(s)
        idx = np.arange(n) if n <= 4096 else np.sort(np.concatenate(
            [np.random.default_rng(n).choice(n, 120, replace=False), [0, 1, n - 2, n - 1]]))
        Fo, To, _ = o.dipole_sample(idx, m=s.m_body)
        assert rel(fn[idx], Fo) <= TOL64 and rel(tn[idx], To) <= TOL64, (n, call, rel(fn[idx], Fo))


def test_noalloc_allocates_nothing(lib):
    """After a warm-up call, further calls leave the device's free memory and
    torch's reserved memory as they were."""
    torch = pytest.importorskip("torch")
    bpm = lib
    s = _loose_dipoles(4096, seed=5)
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(s.x)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(s.m_body)).to(dev)
    f = torch.empty((s.n, 3), dtype=torch.float64, device=dev)
    t = torch.empty((s.n, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    bpm.bpm_dipole_forces_noalloc(s.n, x, m, 1.0, f, t, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for _ in range(5):
        bpm.bpm_dipole_forces_noalloc(s.n, x, m, 1.0, f, t, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == res0


def test_noalloc_rejects_bad_arguments_before_launching(lib):
    torch = pytest.importorskip("torch")
    bpm = lib
    clib = bpm.load()
    # beyond the array
    rc = clib.bpm_dipole_forces_noalloc(32769, None, None, 1.0, None, None, None)
    assert rc == bpm.BPM_ERR_ARG
    assert b"32768" in clib.bpm_last_error(None)
    # host memory through the C ABI: refused by the library itself
    n = 16
    host = np.zeros((n, 3))
    dev = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    hp = host.ctypes.data
    dp = dev.data_ptr()
    rc = clib.bpm_dipole_forces_noalloc(n, hp, dp, 1.0, dp, dp, None)
    assert rc == bpm.BPM_ERR_ARG and b"not device memory" in clib.bpm_last_error(None)
    rc = clib.bpm_dipole_forces_noalloc(n, dp, dp, 1.0, hp, dp, None)
    assert rc == bpm.BPM_ERR_ARG
    # a buffer whose allocation ends before 3n doubles: the last 100
    # particles' worth of a fresh 12 MB allocation, passed with n = 200
    torch.cuda.empty_cache()
    big = torch.zeros(12 * 2 ** 20 // 8, dtype=torch.float64, device="cuda")
    tail = big[-300:]
    okt = torch.zeros((200, 3), dtype=torch.float64, device="cuda")
    ok = okt.data_ptr()
    rc = clib.bpm_dipole_forces_noalloc(200, ok, ok, 1.0, tail.data_ptr(), ok, None)
    assert rc == bpm.BPM_ERR_ARG and b"shorter than 3n" in clib.bpm_last_error(None)
    torch.cuda.synchronize()
    del big, tail, okt
    # the Python binding refuses numpy arrays, CPU tensors and short tensors
    with pytest.raises(TypeError):
        bpm.bpm_dipole_forces_noalloc(n, host, dev, 1.0, dev, dev)
    with pytest.raises(TypeError):
        bpm.bpm_dipole_forces_noalloc(n, dev.cpu(), dev, 1.0, dev, dev)
    with pytest.raises(ValueError):
        bpm.bpm_dipole_forces_noalloc(n + 1, dev, dev, 1.0, dev, dev)
    torch.cuda.synchronize()
