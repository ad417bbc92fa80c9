"""bpm_dipole_forces_noalloc: the allocation-free dipole entry point.

Some callers cannot call cudaMalloc (a host whose caching allocator already
holds the device memory, or a fixed-latency loop that must not allocate), so
the library offers its FP64 all-pairs dipole kernel with scratch held in a
fixed array of the library's device image.  This test calls it through the C
ABI twice in a row and checks each result against the handle-based path
(bpm_forces on the same dipoles) within the FP64 parity tolerance used by the
other GPU tests.  It lives in its own file, collected last, and passes both
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_handle_path_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm

    # the second call is smaller, so stale scratch from the first is present
    for call, n in enumerate((3001, 2500)):
        s = _loose_dipoles(n, seed=100 + call)
        with bpm.Simulation(s, precision=bpm.BPM_FP64) as sim:
            f_ref, t_ref = sim.forces()
        dev = torch.device("cuda")
        x = torch.from_numpy(np.ascontiguousarray(s.x)).to(dev)
        m = torch.from_numpy(np.ascontiguousarray(s.m_body)).to(dev)
        f = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        t = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        bpm.bpm_dipole_forces_noalloc(n, x, m, s.mu0_over_4pi, f, t, stream)
        torch.cuda.synchronize()
        fn, tn = f.cpu().numpy(), t.cpu().numpy()
        ef = np.linalg.norm(fn - f_ref) / np.linalg.norm(f_ref)
        et = np.linalg.norm(tn - t_ref) / np.linalg.norm(t_ref)
        assert ef <= 1e-12 and et <= 1e-12, (call, ef, et)


def test_noalloc_rejects_sizes_beyond_its_array():
    pytest.importorskip("torch")
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm
    lib = bpm.load()
    rc = lib.bpm_dipole_forces_noalloc(32769, None, None, 1.0, None, None, None)
    assert rc == bpm.BPM_ERR_ARG
    assert b"32768" in lib.bpm_last_error(None)
