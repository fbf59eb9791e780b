"""NeuralODE poses (Sec. 3.2, Eqs. 3-4) on the GPU against the FP64 oracle,
through the C ABI: the states after every Runge-Kutta step, the poses at the
output times, and the gradients of a loss on the poses w.r.t. the network
parameters, the instance embeddings and the initial states. Then the chain
with the renderer: poses from the model render a timestep, the pose
adjoints of s3r_render_bwd flow back through s3r_ode_poses_bwd, and the
result equals the oracle's chain (its render backward, then its ODE
backward).

Tolerances. The states are FP32 sums of Runge-Kutta increments: each step
rounds at about 1e-7 of the state and the errors add up over the steps, so
states and poses are compared at 2e-5 (1 + |z|) after 46 steps. Gradients:
<= 1e-3 relative per tensor, as everywhere.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ode
from paper_2503_08217_gb300 import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def built():
    from paper_2503_08217_gb300 import binding, build
    build.build()
    binding.load()
    return True


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_ode_poses_and_gradients_match_oracle(built):
    from paper_2503_08217_gb300 import binding
    K, D, S, T = 24, 8, 2, 24
    params, embed, z0 = scenegen.ode_model(3, K, D)
    z0[:, 3:] = np.random.default_rng(4).uniform(-0.4, 0.4, (K, 3)).astype(np.float32)
    times = (-1.0 + 2.0 * np.arange(T) / (T - 1)).astype(np.float32)
    assert binding.ode_param_count(D) == params.size
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    states, quat, trans = binding.ode_poses(cu(params), cu(embed), cu(z0), cu(times), S)
    torch.cuda.synchronize()
    st_o = ode.trajectory(params.astype(np.float64), embed.astype(np.float64), z0.astype(np.float64),
                          times.astype(np.float64), S, 64)
    q_o, t_o = ode.poses(st_o, S)
    st = states.double().cpu().numpy()
    assert np.abs(st_o[-1] - st_o[0]).max() > 0.5          # the states move
    assert (np.abs(st - st_o) <= 2e-5 * (1.0 + np.abs(st_o))).all(), float(np.abs(st - st_o).max())
    np.testing.assert_allclose(quat.double().cpu().numpy(), q_o, rtol=0, atol=2e-5)
    np.testing.assert_allclose(trans.double().cpu().numpy(), t_o, rtol=2e-5, atol=2e-5)

    rng = np.random.default_rng(5)
    gq = rng.standard_normal((T, K, 4)).astype(np.float32)
    gt = rng.standard_normal((T, K, 3)).astype(np.float32)
    g_p = torch.zeros(params.size, device="cuda")
    g_e = torch.zeros((K, D), device="cuda")
    g_z = torch.zeros((K, 6), device="cuda")
    binding.ode_poses_bwd(cu(params), cu(embed), cu(times), S, states, cu(gq), cu(gt), g_p, g_e, g_z)
    torch.cuda.synchronize()
    dp, de, dz = ode.backward(params.astype(np.float64), embed.astype(np.float64),
                              z0.astype(np.float64), times.astype(np.float64), S, 64,
                              gq.astype(np.float64), gt.astype(np.float64))
    for name, a, b in (("params", g_p, dp), ("embed", g_e, de), ("z0", g_z, dz)):
        a = a.double().cpu().numpy()
        assert _rel(a, b) <= 1e-3, (name, _rel(a, b))
        bad = np.abs(a - b) > 1e-3 * np.abs(b) + 1e-5 * np.abs(b).max()
        assert bad.mean() < 1e-3, (name, int(bad.sum()))


def test_ode_poses_drive_the_renderer_and_its_pose_adjoints(built):
    """Poses of the model at a timestep render the tiny scene's instances;
    the pose adjoints of the render's backward go back through the model.
    The oracle runs the same chain in FP64 (its render backward on the same
    FP32 poses, then its ODE backward on its own trajectory)."""
    import copy
    import gpu_helpers
    from paper_2503_08217_gb300 import binding
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    tiny = scenegen.generate("tiny", seed=0)
    K, D, S, T = tiny.n_inst, 4, 2, tiny.n_steps
    step = 5
    params, embed, z0 = scenegen.ode_model(11, K, D, scale=0.3,
                                           z0_positions=tiny.inst_trans[0].astype(np.float64))
    times = tiny.times.astype(np.float32)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    states, quat, trans = binding.ode_poses(cu(params), cu(embed), cu(z0), cu(times), S)
    q_g = quat.cpu().numpy()
    t_g = trans.cpu().numpy()

    # the oracle's render of the timestep with these poses, and the loss weights
    vis, _ = gpu_helpers.sweep_visibility(tiny)
    cams = tiny.cams[step]
    sc = copy.deepcopy(tiny)
    sc.inst_quat = np.repeat(q_g[step][None], T, 0)
    sc.inst_trans = np.repeat(t_g[step][None], T, 0)
    f = oracle.step_forward(sc, step, vis, None, 0.0, cams=cams)
    view = f["views"][0]
    rng = np.random.default_rng(6)
    d = rng.standard_normal((3, cams[0].height, cams[0].width))
    d[:, gpu_helpers.bad_pixels(cams[0], view["rec"], view["flag"])] = 0.0
    g_orc = oracle.step_backward(sc, step, f, [d], 0.0, cams=cams)
    d[:, g_orc["pixel_flags"][0]] = 0.0
    g_orc = oracle.step_backward(sc, step, f, [d], 0.0, cams=cams)

    # the GPU chain
    dev = DeviceScene.from_host(tiny)
    r = Renderer(tiny.n, K, cams)
    bg = torch.zeros(3, device="cuda")
    iq, it = quat[step].contiguous(), trans[step].contiguous()
    out = r.forward(dev, iq, it, cams, float(times[step]), cu(vis), None, 0.0, bg)
    dL = cu(d.astype(np.float32).reshape(-1))
    grads = {k: torch.zeros_like(v) for k, v in zip(("means", "log_scales", "quats", "opacity_logits", "sh"),
                                                   dev.params())}
    grads["inst_quat"] = torch.zeros_like(iq)
    grads["inst_trans"] = torch.zeros_like(it)
    r.backward(dev, iq, it, bg, dL, grads)
    gq = torch.zeros_like(quat)
    gt = torch.zeros_like(trans)
    gq[step] = grads["inst_quat"]
    gt[step] = grads["inst_trans"]
    g_p = torch.zeros(params.size, device="cuda")
    g_e = torch.zeros((K, D), device="cuda")
    g_z = torch.zeros((K, 6), device="cuda")
    binding.ode_poses_bwd(cu(params), cu(embed), cu(times), S, states, gq, gt, g_p, g_e, g_z)
    torch.cuda.synchronize()
    r.sync_status()
    assert out.numel() == 3 * cams[0].width * cams[0].height
    assert _rel(grads["inst_trans"].double().cpu().numpy(), g_orc["inst_trans"]) <= 1e-3
    assert _rel(grads["inst_quat"].double().cpu().numpy(), g_orc["inst_quat"]) <= 1e-3

    gq_o = np.zeros((T, K, 4))
    gt_o = np.zeros((T, K, 3))
    gq_o[step] = g_orc["inst_quat"]
    gt_o[step] = g_orc["inst_trans"]
    dp, de, dz = ode.backward(params.astype(np.float64), embed.astype(np.float64),
                              z0.astype(np.float64), times.astype(np.float64), S, 64, gq_o, gt_o)
    for name, a, b in (("params", g_p, dp), ("embed", g_e, de), ("z0", g_z, dz)):
        a = a.double().cpu().numpy()
        assert np.abs(b).max() > 0, name
        assert _rel(a, b) <= 2e-3, (name, _rel(a, b))
