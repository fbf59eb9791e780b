"""Fused Adam (the optimiser step of the training configuration) against the
FP64 oracle: ragged tensor sizes spanning many grid-stride rounds, several
steps in a row, then a full-size run over every parameter array of the
surround-rig scene (9.0M Gaussians, SH3) checked on sampled elements."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(p, m, v, p_ref, m_ref, v_ref):
    """FP32 against FP64 from the same FP32 inputs: p to a few ulp of O(1)
    values (the step itself is lr-sized), the moments to 1e-5 relative with an
    absolute floor at 1e-6 of their largest magnitude (m may cancel)."""
    np.testing.assert_allclose(p, p_ref, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(m, m_ref, rtol=1e-5, atol=1e-6 * np.abs(m_ref).max())
    np.testing.assert_allclose(v, v_ref, rtol=1e-5, atol=1e-6 * np.abs(v_ref).max())


def test_adam_ragged_tensors_several_steps():
    from paper_2503_08217_gb300 import binding, build
    build.build()
    rng = np.random.default_rng(11)
    sizes = [0, 1, 37, 4099, (1 << 20) + 3, 3_000_001]
    host = [rng.standard_normal(n).astype(np.float32) for n in sizes]
    dev_p = [torch.tensor(h, device="cuda") for h in host]
    dev_m = [torch.zeros(n, device="cuda") for n in sizes]
    dev_v = [torch.zeros(n, device="cuda") for n in sizes]
    ref = [(h.astype(np.float64), np.zeros(n), np.zeros(n)) for h, n in zip(host, sizes)]
    # the oracle gets the hyperparameters the kernel receives (float32): 1 - beta2
    # of float32(0.999) differs from 0.001 by 1.3e-5 relative
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1e-2, 0.9, 0.999, 1e-8))
    for step in range(1, 4):
        grads = [(rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1)).astype(np.float32) for n in sizes]
        dev_g = [torch.tensor(g, device="cuda") for g in grads]
        binding.adam_step(dev_p, dev_g, dev_m, dev_v, lr, step, b1, b2, eps)
        ref = [oracle.adam_step(r[0], g, r[1], r[2], lr, step, b1, b2, eps) for r, g in zip(ref, grads)]
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        if n == 0:
            continue
        _check(dev_p[i].cpu().numpy(), dev_m[i].cpu().numpy(), dev_v[i].cpu().numpy(), *ref[i])


def test_adam_full_rig_parameters_sampled():
    """Every parameter array of the 9.0M-Gaussian rig scene plus the instance
    poses in one launch; 20k sampled elements per array against the oracle."""
    from paper_2503_08217_gb300 import binding, build, scenegen
    build.build()
    scene = scenegen.generate("rig", seed=0)
    arrays = [scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
              scene.inst_quat, scene.inst_trans]
    p = [torch.tensor(np.ascontiguousarray(a, dtype=np.float32).reshape(-1), device="cuda") for a in arrays]
    gen = torch.Generator(device="cuda").manual_seed(3)
    m = [torch.randn(t.numel(), device="cuda", generator=gen) * 1e-2 for t in p]
    v = [torch.rand(t.numel(), device="cuda", generator=gen) * 1e-4 for t in p]
    g = [torch.randn(t.numel(), device="cuda", generator=gen) * 1e-2 for t in p]
    rng = np.random.default_rng(2)
    picks = [torch.tensor(rng.integers(0, t.numel(), min(20_000, t.numel())), device="cuda") for t in p]
    before = [tuple(x[i].cpu().numpy() for x in (t, mm, vv, gg)) for t, mm, vv, gg, i in zip(p, m, v, g, picks)]
    assert sum(t.numel() for t in p) > 400_000_000
    lr, b1, b2, eps = (float(np.float32(x)) for x in (1.6e-4, 0.9, 0.999, 1e-8))
    binding.adam_step(p, g, m, v, lr, 7, b1, b2, eps)
    torch.cuda.synchronize()
    for t, mm, vv, i, (p0, m0, v0, g0) in zip(p, m, v, picks, before):
        pr, mr, vr = oracle.adam_step(p0, g0, m0, v0, lr, 7, b1, b2, eps)
        _check(t[i].cpu().numpy(), mm[i].cpu().numpy(), vv[i].cpu().numpy(), pr, mr, vr)


def test_adam_unaligned_views():
    """Arrays that start 4 bytes past a 16-byte boundary take the one-element
    path; mixed with aligned tensors in the same launch."""
    from paper_2503_08217_gb300 import binding, build
    build.build()
    rng = np.random.default_rng(12)
    n = 100_003
    bufs = [torch.tensor(rng.standard_normal(n + 1).astype(np.float32), device="cuda") for _ in range(2)]
    p_un, g_un = bufs[0][1:], bufs[1][1:]
    m_un = torch.zeros(n + 1, device="cuda")[1:]
    v_un = torch.zeros(n + 1, device="cuda")[1:]
    p_al = torch.tensor(rng.standard_normal(777).astype(np.float32), device="cuda")
    g_al = torch.tensor(rng.standard_normal(777).astype(np.float32), device="cuda")
    m_al, v_al = torch.zeros(777, device="cuda"), torch.zeros(777, device="cuda")
    p0 = [p_un.cpu().numpy().copy(), p_al.cpu().numpy().copy()]
    g0 = [g_un.cpu().numpy().copy(), g_al.cpu().numpy().copy()]
    lr, b1, b2, eps = (float(np.float32(x)) for x in (3e-3, 0.9, 0.999, 1e-8))
    binding.adam_step([p_un, p_al], [g_un, g_al], [m_un, m_al], [v_un, v_al], lr, 1, b1, b2, eps)
    torch.cuda.synchronize()
    for (p, m, v), pi, gi in zip(((p_un, m_un, v_un), (p_al, m_al, v_al)), p0, g0):
        ref = oracle.adam_step(pi, gi, np.zeros_like(pi), np.zeros_like(pi), lr, 1, b1, b2, eps)
        _check(p.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), *ref)


def test_fused_adam_class_two_steps():
    from paper_2503_08217_gb300 import build
    from paper_2503_08217_gb300.render import FusedAdam
    build.build()
    rng = np.random.default_rng(13)
    host = [rng.standard_normal(s).astype(np.float32) for s in ((1000, 3), (1000,), (1000, 16, 3))]
    params = [torch.tensor(h, device="cuda") for h in host]
    opt = FusedAdam(params, lr=float(np.float32(1e-3)))
    ref = [(h.astype(np.float64), np.zeros(h.shape), np.zeros(h.shape)) for h in host]
    b1, b2, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-8))
    for step in (1, 2):
        grads = [rng.standard_normal(h.shape).astype(np.float32) for h in host]
        opt.step([torch.tensor(g, device="cuda") for g in grads])
        ref = [oracle.adam_step(r[0], g, r[1], r[2], opt.lr, step, b1, b2, eps) for r, g in zip(ref, grads)]
    torch.cuda.synchronize()
    for p, m, v, r in zip(params, opt.exp_avg, opt.exp_avg_sq, ref):
        _check(p.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), *r)
