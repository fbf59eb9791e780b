"""Checkpoint round trip of the training state on the CPU (no library calls)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2503_08217_gb300 import train
from paper_2503_08217_gb300.render import DeviceScene


def _state(seed=0, n=37, n_inst=2, T=5, sh=16):
    g = torch.Generator().manual_seed(seed)
    r = lambda *s: torch.randn(*s, generator=g)   # noqa: E731
    scene = DeviceScene(means=r(n, 3), log_scales=r(n, 3), quats=r(n, 4), opacity_logits=r(n),
                        sh=r(n, sh * 3), inst_offsets=torch.tensor([0, 20, 30, n], dtype=torch.int64),
                        sh_degree=3)
    st = train.TrainState.initial(scene, r(T, n_inst, 4), r(T, n_inst, 3), r(n, 2), r(n, 2),
                                  lod={"mode": "stochastic", "r": 2.0, "p_max": 0.5,
                                       "distance": 100.0, "offset": (0.1, 0.1, 0.1), "seed": 2025})
    for m in st.exp_avg + st.exp_avg_sq + st.pose_exp_avg + st.pose_exp_avg_sq:
        m.copy_(r(*m.shape).abs())
    st.pose_steps[3] = 7
    st.adam_steps, st.step, st.epoch = 11, 11, 12
    return st


def test_checkpoint_round_trip_is_exact(tmp_path):
    st = _state()
    train.save(tmp_path / "ck.pt", st)
    back = train.load(tmp_path / "ck.pt", device="cpu")
    a, b = st.tensors(), back.tensors()
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].dtype == b[k].dtype and torch.equal(a[k], b[k]), k
    assert (back.pose_steps, back.adam_steps, back.step, back.epoch) == ([0, 0, 0, 7, 0], 11, 11, 12)
    assert back.lod == st.lod and back.scene.sh_degree == 3
    assert back.scene.n == st.scene.n and back.scene.n_inst == 2


def test_checkpoint_holds_every_piece_of_state():
    names = set(_state().tensors())
    for p in train.PARAM_NAMES:
        assert {f"scene.{p}", f"exp_avg.{p}", f"exp_avg_sq.{p}"} <= names
    assert {"inst_quat", "inst_trans", "vis_window", "point_life", "scene.inst_offsets",
            "pose_exp_avg.quat", "pose_exp_avg.trans", "pose_exp_avg_sq.quat",
            "pose_exp_avg_sq.trans"} <= names


def test_initial_state_has_zero_moments_and_no_steps():
    st = _state()
    fresh = train.TrainState.initial(st.scene, st.inst_quat, st.inst_trans, st.vis_window,
                                     st.point_life)
    assert all(float(m.abs().sum()) == 0.0 for m in fresh.exp_avg + fresh.pose_exp_avg_sq)
    assert fresh.pose_steps == [0] * 5 and fresh.adam_steps == fresh.step == fresh.epoch == 0
    assert fresh.lod == {"mode": "threshold", "r": 0.0}
    assert fresh.pose_exp_avg[0].shape == st.inst_quat.shape


def test_a_checkpoint_of_another_format_is_refused(tmp_path):
    train.save(tmp_path / "ck.pt", _state())
    blob = torch.load(tmp_path / "ck.pt", weights_only=True)
    blob["format"] = 99
    torch.save(blob, tmp_path / "bad.pt")
    with pytest.raises(ValueError, match="format"):
        train.load(tmp_path / "bad.pt", device="cpu")
    np.testing.assert_equal(train.FORMAT, 1)
