"""Checkpoint / resume on the GPU: a trainer built on a saved state continues
the run. The forward after the resume is bit-identical to the uninterrupted
run's (including the Eq. 7 draws, numbered by the restored call counter), the
point-life record (Eq. 5) is identical, and gradients and parameters agree up
to the float atomics' summation order."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2503_08217_gb300 import scenegen, train
from paper_2503_08217_gb300.render import DeviceScene, pixel_count

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LODS = {"threshold": {"mode": "threshold", "r": 0.0},
        "eq7": {"mode": "stochastic", "r": 2.0, "p_max": 0.5, "distance": 20.0,
                "offset": (0.05, 0.05, 0.05), "seed": 2025}}


@pytest.fixture(scope="module")
def tiny_and_record():
    import gpu_helpers
    from paper_2503_08217_gb300 import binding, build
    build.build()
    binding.load()
    tiny = scenegen.generate("tiny", seed=0)
    return tiny, gpu_helpers.sweep_visibility(tiny)


def _initial(tiny, vis, life, lod):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()   # noqa: E731
    return train.TrainState.initial(DeviceScene.from_host(tiny), f(tiny.inst_quat),
                                    f(tiny.inst_trans), f(vis), f(life), lod)


@pytest.mark.parametrize("lod", list(LODS))
def test_resume_continues_the_run(tiny_and_record, tmp_path, lod):
    tiny, (vis, life) = tiny_and_record
    lr = 1e-3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    targets = [torch.rand(3 * pixel_count(c), device="cuda", generator=gen) for c in tiny.cams]
    a = train.Trainer(_initial(tiny, vis, life, LODS[lod]), tiny.cams, tiny.times, lr=lr)
    for k in (0, 3, 6):
        a.step(k, targets[k])
    a.save(tmp_path / "ck.pt")
    loss_a, img_a = a.step(8, targets[8])
    torch.cuda.synchronize()

    b = train.Trainer(train.load(tmp_path / "ck.pt"), tiny.cams, tiny.times, lr=lr)
    assert b.state.step == 3 and b.state.epoch == a.state.epoch > 0
    loss_b, img_b = b.step(8, targets[8])
    torch.cuda.synchronize()
    a.renderer.sync_status()
    b.renderer.sync_status()

    assert torch.equal(img_a, img_b)                               # forward: bit-identical
    assert torch.equal(a.state.point_life, b.state.point_life)     # Eq. 5 record
    assert abs(float(loss_a) - float(loss_b)) <= 1e-5 * abs(float(loss_a))
    for name, ga in a.grads.items():
        gb = b.grads[name]
        scale = float(ga.abs().max())
        torch.testing.assert_close(gb, ga, rtol=1e-3, atol=1e-5 * scale, msg=name)
    # an Adam step moves a parameter by a few lr at most: differences in the
    # step's gradients (summation order) stay within that, most far below it
    pa = dict(a.state.tensors())
    pb = dict(b.state.tensors())
    for name in ("scene.means", "scene.quats", "scene.sh", "inst_quat", "inst_trans"):
        d = (pa[name] - pb[name]).abs()
        assert float(d.max()) <= 4 * lr, name
        assert float((d > 1e-6).float().mean()) < 1e-2, name
    assert a.state.adam_steps == b.state.adam_steps == 4
    assert a.state.pose_steps == b.state.pose_steps


def test_a_failed_step_changes_no_parameter(tiny_and_record):
    """A step whose render overflowed the workspace (splats dropped) must not
    reach the optimiser: both Adam updates are gated on the device by the
    latched status, the step raises S3R_ERR_CAPACITY and is not counted, and
    every parameter, moment and pose is unchanged. Without the per-step
    check the device skips the updates all the same."""
    from paper_2503_08217_gb300 import binding
    tiny, (vis, life) = tiny_and_record
    a = train.Trainer(_initial(tiny, vis, life, LODS["threshold"]), tiny.cams, tiny.times,
                      max_splats=100, max_duplicates=50)
    before = {k: v.clone() for k, v in a.state.tensors().items()}
    target = torch.rand(3 * pixel_count(tiny.cams[3]), device="cuda")
    with pytest.raises(binding.S3RError) as e:
        a.step(3, target)
    assert e.value.status == 2                                    # S3R_ERR_CAPACITY
    assert (a.state.step, a.state.adam_steps, a.state.pose_steps[3]) == (0, 0, 0)
    a.step(3, target, check=False)
    a.step(4, target, check=False)
    with pytest.raises(binding.S3RError):
        a.check()
    for k, v in a.state.tensors().items():
        if k != "point_life":                                     # Eq. 5 records as it renders
            assert torch.equal(v, before[k]), k
