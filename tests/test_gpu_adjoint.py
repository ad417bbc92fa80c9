"""Adjoint of the time stepping (bpm_adjoint_begin / bpm_adjoint_end): the
gradient of L = |x_tip(T) - target|^2 with respect to the body-frame dipoles
and the uniform field.

Two checks: (1) central differences with h = 1e-6 on selected components, of
GPU runs and of the CPU FP64 oracle; the trajectory's own rounding differs
between the perturbed runs, which puts a noise floor of order
eps |x| |x - target| / h on each difference, so the bound is 1e-6 of the
largest component plus four times the noise measured as |FD(h) - FD(2h)|;
(2) the directional derivative along a random direction through all
parameters, against a fourth-order five-point difference with h = 1e-4
(truncation and noise both far below 1e-7 relative)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2603_27279_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H = 1e-6


@pytest.fixture(scope="module")
def bpm():
    from paper_2603_27279_gb300 import build
    build.build()
    from paper_2603_27279_gb300 import bpm as B
    B.load()
    return B


def _loss(x, tip, target):
    d = x[tip] - target
    return float(d @ d)


def adjoint_grad(bpm, s, steps, every, tip, target, plan=None, precision=W.PRECISION_FP64):
    with bpm.Simulation(s, precision=precision) as sim:
        if plan is not None:
            sim.set_dipole_plan(*plan)
        sim.adjoint_begin(steps, every)
        x = sim.get_state()[0]
        dL = np.zeros_like(x)
        dL[tip] = 2.0 * (x[tip] - target)
        gm, gB = sim.adjoint_end(dL)
    return _loss(x, tip, target), gm, gB


def gpu_loss(bpm, s, steps, tip, target, precision=W.PRECISION_FP64):
    with bpm.Simulation(s, precision=precision) as sim:
        sim.step(steps)
        return _loss(sim.get_state()[0], tip, target)


def oracle_loss(s, steps, tip, target):
    o = Oracle(s)
    o.run(steps)
    return _loss(o.x.reshape(-1, 3), tip, target)


def _perturbed(s, kind, i, a, delta):
    t = s.copy()
    if kind == "m":
        t.m_body[i, a] += delta
    else:
        t.B[a] += delta
    return t


def fd(loss_fn, s, comps, h=H):
    out = []
    for kind, i, a in comps:
        out.append((loss_fn(_perturbed(s, kind, i, a, h)) - loss_fn(_perturbed(s, kind, i, a, -h))) / (2 * h))
    return np.array(out)


def check_components(g_adj, loss_fn, s, comps):
    """|adjoint - FD(h)| <= 1e-6 max|g| + 4 max|FD(h) - FD(2h)| per component."""
    g_h = fd(loss_fn, s, comps, H)
    g_2h = fd(loss_fn, s, comps, 2 * H)
    noise = np.abs(g_h - g_2h).max()
    bound = 1e-6 * np.abs(g_adj).max() + 4.0 * noise
    err = np.abs(g_adj - g_h).max()
    assert err <= bound, (err, bound, noise, g_adj, g_h)
    return err, noise


def check_direction(gm, gB, loss_fn, s, seed, along_gradient=False):
    """g . d against a five-point fourth-order difference along d (h = 1e-3):
    |g.d - FD5(h)| <= 1e-7 |g.d| + 4 |FD5(h) - FD5(2h)|, and that measured
    noise must itself stay below 1e-5 |g.d| so that the check has teeth."""
    if along_gradient:
        dm, dB = gm.copy(), gB.copy()
    else:
        rng = np.random.default_rng(seed)
        dm, dB = rng.standard_normal(s.m_body.shape), rng.standard_normal(3)
    nrm = np.sqrt((dm ** 2).sum() + (dB ** 2).sum())
    dm, dB = dm / nrm, dB / nrm

    def L_at(eps):
        t = s.copy()
        t.m_body = s.m_body + eps * dm
        t.B = s.B + eps * dB
        return loss_fn(t)

    def fd5(h):
        return (L_at(-2 * h) - 8 * L_at(-h) + 8 * L_at(h) - L_at(2 * h)) / (12 * h)

    f1, f2 = fd5(1e-3), fd5(2e-3)
    g_dir = float((gm * dm).sum() + gB @ dB)
    noise = abs(f1 - f2)
    assert noise <= 1e-5 * abs(g_dir), (noise, g_dir)
    assert abs(g_dir - f1) <= 1e-7 * abs(g_dir) + 4 * noise, (g_dir, f1, f2)


def pick(gm, gB, comps):
    return np.array([gm[i, a] if kind == "m" else gB[a] for kind, i, a in comps])


def comps_for(s, k, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(s.n, size=k, replace=False)
    return [("m", int(i), int(rng.integers(3))) for i in idx] + [("B", 0, a) for a in range(3)]


def _target(bpm, s, steps, tip):
    with bpm.Simulation(s, precision=W.PRECISION_FP64) as sim:
        sim.step(steps)
        return sim.get_state()[0][tip] + np.array([0.01, -0.02, 0.015])


def test_adjoint_matches_gpu_and_oracle_fd_small(bpm):
    s = W.adjoint_rod(48)
    steps, every, tip = 40, 16, s.n - 1   # segments of 16, 16, 8
    target = _target(bpm, s, steps, tip)
    L, gm, gB = adjoint_grad(bpm, s, steps, every, tip, target)
    comps = comps_for(s, 12, 1)
    g_adj = pick(gm, gB, comps)
    assert np.abs(g_adj).max() > 0
    gpu = lambda t: gpu_loss(bpm, t, steps, tip, target)  # noqa: E731
    orc = lambda t: oracle_loss(t, steps, tip, target)  # noqa: E731
    check_components(g_adj, gpu, s, comps)
    check_components(g_adj, orc, s, comps)
    check_direction(gm, gB, gpu, s, 11, along_gradient=True)
    check_direction(gm, gB, gpu, s, 11)
    check_direction(gm, gB, orc, s, 12, along_gradient=True)


def test_adjoint_all_terms(bpm):
    """Random rest orientations (gauge), gradient and rotating fields,
    per-rod dipoles, damping, clamped particles: every term of the force
    function and of the integrator is in the gradient."""
    s = W.random_rods([5, 9, 12], seed=31, dipole_mode=W.DIPOLE_PER_ROD, damping=0.2, vel_sigma=0.05)
    steps, every, tip = 25, 10, 13
    target = _target(bpm, s, steps, tip)
    orc = lambda t: oracle_loss(t, steps, tip, target)  # noqa: E731
    for mode in (W.DIPOLE_PER_ROD, W.DIPOLE_GLOBAL):
        sm = s.copy()
        sm.dipole_mode = mode
        L, gm, gB = adjoint_grad(bpm, sm, steps, every, tip, target)
        comps = comps_for(sm, 10, 2)
        check_components(pick(gm, gB, comps), orc, sm, comps)
        check_direction(gm, gB, orc, sm, 13 + mode, along_gradient=True)
        check_direction(gm, gB, orc, sm, 13 + mode)


def test_adjoint_full_size_16_components(bpm):
    """The 2048-particle clamped rod, 500 steps, checkpoints every 50: 16
    random components of dL/dm~ (and dL/dB) against central differences of
    GPU runs, and the directional derivative along the gradient against a
    fourth-order difference of CPU FP64 oracle runs (8 runs of 500 steps)."""
    s = W.adjoint_rod()
    t2 = W.adjoint_rod(seed=W.SEED_BASE + 33)
    steps, every, tip = s.n_steps, 50, s.n - 1
    # a reachable target: the tip reached with a second seed's magnetisation
    with bpm.Simulation(t2, precision=W.PRECISION_FP64) as sim:
        sim.step(steps)
        target = sim.get_state()[0][tip]
    L, gm, gB = adjoint_grad(bpm, s, steps, every, tip, target)
    comps = comps_for(s, 16, 3)
    gpu = lambda t: gpu_loss(bpm, t, steps, tip, target)  # noqa: E731
    check_components(pick(gm, gB, comps), gpu, s, comps)
    check_direction(gm, gB, gpu, s, 17, along_gradient=True)
    check_direction(gm, gB, gpu, s, 17)
    orc = lambda t: oracle_loss(t, steps, tip, target)  # noqa: E731
    check_direction(gm, gB, orc, s, 18, along_gradient=True)


@pytest.mark.parametrize("case", ["rod_200", "global_rods"])
def test_symmetric_and_ordered_dipole_vjp_agree(bpm, case):
    """The dipole VJP over unordered pairs (both sides of each pair, tiles
    of 32 with a ragged last tile) and over ordered pairs (forced by the
    ordered dipole plan) give the same gradient to rounding; the forward
    trajectories of the two plans differ only by rounding as well."""
    if case == "rod_200":
        s = W.adjoint_rod(200)
        steps, every, tip = 30, 7, s.n - 1
    else:
        s = W.random_rods([40, 3, 57, 33], seed=35, dipole_mode=W.DIPOLE_GLOBAL, vel_sigma=0.05)
        steps, every, tip = 20, 6, 41
    target = _target(bpm, s, steps, tip) if case == "rod_200" else np.zeros(3)
    _, gm_s, gB_s = adjoint_grad(bpm, s, steps, every, tip, target)
    _, gm_o, gB_o = adjoint_grad(bpm, s, steps, every, tip, target, plan=(1, 3))
    scale = max(np.abs(gm_o).max(), np.abs(gB_o).max())
    assert scale > 0
    assert np.abs(gm_s - gm_o).max() <= 1e-9 * scale, np.abs(gm_s - gm_o).max() / scale
    assert np.abs(gB_s - gB_o).max() <= 1e-9 * scale


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function(bpm, device):
    """The torch.autograd.Function with host tensors, and with CUDA tensors
    that cross the C ABI as device pointers."""
    torch = pytest.importorskip("torch")
    from paper_2603_27279_gb300.adjoint import final_positions
    s = W.adjoint_rod(32)
    steps, every, tip = 30, 7, s.n - 1
    target = _target(bpm, s, steps, tip)
    with bpm.Simulation(s, precision=W.PRECISION_FP64) as sim:
        start = sim.get_state()
        m = torch.tensor(s.m_body, dtype=torch.float64, device=device, requires_grad=True)
        B = torch.tensor(s.B, dtype=torch.float64, device=device, requires_grad=True)
        x = final_positions(m, B, sim, start, steps, every)
        assert x.device == m.device
        loss = ((x[tip] - torch.tensor(target, device=device)) ** 2).sum()
        loss.backward()
    L, gm, gB = adjoint_grad(bpm, s, steps, every, tip, target)
    assert float(loss.detach()) == pytest.approx(L, rel=1e-14)
    assert m.grad.device == m.device
    assert np.allclose(m.grad.cpu().numpy(), gm, rtol=1e-12, atol=0)
    assert np.allclose(B.grad.cpu().numpy(), gB, rtol=1e-12)


def test_adjoint_rejects_mixed_and_missing_record(bpm):
    s = W.adjoint_rod(16)
    with bpm.Simulation(s, precision=W.PRECISION_MIXED) as sim:
        with pytest.raises(bpm.BpmError):
            sim.adjoint_begin(5, 2)
    with bpm.Simulation(s, precision=W.PRECISION_FP64) as sim:
        with pytest.raises(bpm.BpmError):
            sim.adjoint_end(np.zeros((s.n, 3)))
        sim.adjoint_begin(5, 2)
        sim.set_field(B=[0.0, 0.1, 0.0])
        with pytest.raises(bpm.BpmError):
            sim.adjoint_end(np.zeros((s.n, 3)))


# ------------------------------------------------------------ float-float
# A BPM_FF handle records its trajectory with float-float dipole pairs and
# evaluates the symmetric dipole VJP in float-float (k_adj_dipole_sym_ff).
# Its gradient is that of its own time stepping, which differs from the FP64
# one by the float-float rounding of the forces (a few 1e-13 relative).

@pytest.mark.parametrize("case", ["rod_200", "global_rods"])
def test_ff_adjoint_agrees_with_fp64(bpm, case):
    if case == "rod_200":
        s = W.adjoint_rod(200)
        steps, every, tip = 30, 7, s.n - 1
    else:
        s = W.random_rods([40, 3, 57, 33], seed=35, dipole_mode=W.DIPOLE_GLOBAL, vel_sigma=0.05)
        steps, every, tip = 20, 6, 41
    target = _target(bpm, s, steps, tip) if case == "rod_200" else np.zeros(3)
    _, gm_6, gB_6 = adjoint_grad(bpm, s, steps, every, tip, target)
    _, gm_f, gB_f = adjoint_grad(bpm, s, steps, every, tip, target, precision=W.PRECISION_FF)
    scale = max(np.abs(gm_6).max(), np.abs(gB_6).max())
    assert scale > 0
    assert np.abs(gm_f - gm_6).max() <= 1e-9 * scale, np.abs(gm_f - gm_6).max() / scale
    assert np.abs(gB_f - gB_6).max() <= 1e-9 * scale


def test_ff_adjoint_matches_ff_finite_differences(bpm):
    """Float-float gradient against central differences of float-float runs,
    with the noise-aware bounds of the FP64 checks."""
    s = W.adjoint_rod(48)
    steps, every, tip = 40, 16, s.n - 1
    target = _target(bpm, s, steps, tip)
    L, gm, gB = adjoint_grad(bpm, s, steps, every, tip, target, precision=W.PRECISION_FF)
    comps = comps_for(s, 10, 5)
    gpu = lambda t: gpu_loss(bpm, t, steps, tip, target, precision=W.PRECISION_FF)  # noqa: E731
    check_components(pick(gm, gB, comps), gpu, s, comps)
    check_direction(gm, gB, gpu, s, 23, along_gradient=True)
    check_direction(gm, gB, gpu, s, 23)


def test_ff_adjoint_full_size(bpm):
    """The 2048-particle rod, 500 steps, checkpoints every 50: the
    float-float gradient against the FP64 one."""
    s = W.adjoint_rod()
    t2 = W.adjoint_rod(seed=W.SEED_BASE + 33)
    steps, every, tip = s.n_steps, 50, s.n - 1
    with bpm.Simulation(t2, precision=W.PRECISION_FP64) as sim:
        sim.step(steps)
        target = sim.get_state()[0][tip]
    _, gm_6, gB_6 = adjoint_grad(bpm, s, steps, every, tip, target)
    _, gm_f, gB_f = adjoint_grad(bpm, s, steps, every, tip, target, precision=W.PRECISION_FF)
    scale = max(np.abs(gm_6).max(), np.abs(gB_6).max())
    assert np.abs(gm_f - gm_6).max() <= 1e-9 * scale, np.abs(gm_f - gm_6).max() / scale
    assert np.abs(gB_f - gB_6).max() <= 1e-9 * scale
