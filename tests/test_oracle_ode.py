"""Pins of the NeuralODE pose oracle (Sec. 3.2, Eqs. 3-4) against what the
mathematics fixes, independent of the oracle's own code:

  * a constant vector field integrates exactly (z(t) = z0 + b3 (t - t0));
  * the integrator is fourth order: against a high-accuracy solution of the
    same ODE (scipy's DOP853 at tolerance 1e-12), halving the step divides the
    error by about 16 (a wrong Runge-Kutta weight or stage time breaks it);
  * the rotation-vector map gives the textbook quaternion of an axis rotation
    and unit quaternions, continuously through zero;
  * the hand-written reverse mode equals central differences (FP64,
    h = 1e-6) on every parameter, embedding and initial state, and an
    independent float64 PyTorch restatement with autograd.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ode


def _setup(seed, H, D, K, scale=0.6):
    rng = np.random.default_rng(seed)
    n = ode.param_count(H, D)
    params = rng.standard_normal(n) * scale / np.sqrt(H)
    emb = rng.standard_normal((K, D)) * 0.5
    z0 = np.concatenate([rng.uniform(-5, 5, (K, 3)), np.zeros((K, 3))], axis=1)
    return params, emb, z0


def test_constant_field_integrates_exactly():
    H, D, K = 16, 4, 3
    params, emb, z0 = _setup(1, H, D, K)
    net = ode.unpack(params, H, D)
    net["W3"][:] = 0.0
    b3 = np.array([0.3, -1.2, 2.0, 0.05, -0.1, 0.2])
    net["b3"][:] = b3
    times = np.array([-1.0, -0.7, -0.2, 0.5])
    st = ode.trajectory(params, emb, z0, times, 3, H)
    for j, t in enumerate(times):
        np.testing.assert_allclose(st[3 * j], z0 + b3 * (t - times[0]), rtol=0, atol=1e-14)


def test_integrator_is_fourth_order():
    scipy = pytest.importorskip("scipy.integrate")
    H, D, K = 16, 4, 1
    params, emb, z0 = _setup(2, H, D, K, scale=1.0)
    net = ode.unpack(params, H, D)
    times = np.array([-1.0, 1.0])

    def rhs(t, z):
        return ode.f(net, z, t, emb[0])[0]

    ref = scipy.solve_ivp(rhs, (-1.0, 1.0), z0[0], method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for S in (8, 16, 32):
        st = ode.trajectory(params, emb, z0, times, S, H)
        errs.append(np.abs(st[-1, 0] - ref).max())
    assert errs[0] > 1e-9                       # the test field is not trivially integrated
    for a, b in zip(errs, errs[1:]):
        assert 14.0 < a / b < 18.0, errs        # 2^4 = 16 (15.85, 15.93 on this field)


def test_rotation_vector_to_quaternion():
    th = 0.7
    np.testing.assert_allclose(ode.quat_from_rotvec([0.0, 0.0, th]),
                               [np.cos(th / 2), 0.0, 0.0, np.sin(th / 2)], atol=1e-15)
    rng = np.random.default_rng(3)
    for r in rng.standard_normal((20, 3)):
        assert abs(np.linalg.norm(ode.quat_from_rotvec(r)) - 1.0) < 1e-14
    # the rotation of the quaternion turns x towards y by th about z
    w, x, y, z = ode.quat_from_rotvec([0.0, 0.0, th])
    Rx = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    np.testing.assert_allclose(Rx, [np.cos(th), np.sin(th), 0.0], atol=1e-15)
    # continuous through zero
    a = ode.quat_from_rotvec([1e-13, 0.0, 0.0])
    b = ode.quat_from_rotvec([1e-6, 0.0, 0.0])
    np.testing.assert_allclose(a, [1.0, 5e-14, 0.0, 0.0], atol=1e-20)
    np.testing.assert_allclose(b, [1.0 - 1.25e-13, 5e-7, 0.0, 0.0], rtol=1e-12)


def _loss(params, emb, z0, times, S, H, gq, gt):
    st = ode.trajectory(params, emb, z0, times, S, H)
    q, tr = ode.poses(st, S)
    return float((q * gq).sum() + (tr * gt).sum())


def test_gradient_matches_central_differences():
    H, D, K, S = 8, 3, 2, 2
    params, emb, z0 = _setup(4, H, D, K, scale=1.5)
    z0[:, 3:] = np.random.default_rng(9).uniform(-0.5, 0.5, (K, 3))   # a rotation to start with
    times = np.array([-1.0, -0.6, -0.1, 0.4])
    rng = np.random.default_rng(5)
    gq = rng.standard_normal((times.size, K, 4))
    gt = rng.standard_normal((times.size, K, 3))
    dp, de, dz = ode.backward(params, emb, z0, times, S, H, gq, gt)
    eps = 1e-6

    def fd(arr, idx):
        old = arr[idx]
        arr[idx] = old + eps
        up = _loss(params, emb, z0, times, S, H, gq, gt)
        arr[idx] = old - eps
        dn = _loss(params, emb, z0, times, S, H, gq, gt)
        arr[idx] = old
        return (up - dn) / (2 * eps)

    num = np.array([fd(params, i) for i in range(params.size)])
    np.testing.assert_allclose(dp, num, rtol=1e-6, atol=1e-8 * np.abs(num).max())
    num = np.array([fd(emb, ix) for ix in np.ndindex(emb.shape)]).reshape(emb.shape)
    np.testing.assert_allclose(de, num, rtol=1e-6, atol=1e-8 * np.abs(num).max())
    num = np.array([fd(z0, ix) for ix in np.ndindex(z0.shape)]).reshape(z0.shape)
    np.testing.assert_allclose(dz, num, rtol=1e-6, atol=1e-8 * np.abs(num).max())


def test_gradient_matches_torch_autograd_restatement():
    torch = pytest.importorskip("torch")
    H, D, K, S = 64, 8, 3, 3
    params, emb, z0 = _setup(6, H, D, K)
    times = np.array([-1.0, -0.8, -0.55, -0.3])
    rng = np.random.default_rng(7)
    gq = rng.standard_normal((times.size, K, 4))
    gt = rng.standard_normal((times.size, K, 3))
    dp, de, dz = ode.backward(params, emb, z0, times, S, H, gq, gt)

    # the same model written independently with torch tensors and autograd
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    E = torch.tensor(emb, dtype=torch.float64, requires_grad=True)
    Z = torch.tensor(z0, dtype=torch.float64, requires_grad=True)
    I = 7 + D
    o = 0
    W1 = P[o:o + H * I].view(H, I); o += H * I
    b1 = P[o:o + H]; o += H
    W2 = P[o:o + H * H].view(H, H); o += H * H
    b2 = P[o:o + H]; o += H
    W3 = P[o:o + 6 * H].view(6, H); o += 6 * H
    b3 = P[o:o + 6]

    def field(z, t):                                 # [K, 6], scalar
        x = torch.cat([z, torch.full((K, 1), float(t), dtype=torch.float64), E], dim=1)
        return torch.tanh(torch.tanh(x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3

    def quat(r):
        th = torch.sqrt((r * r).sum(1, keepdim=True))
        return torch.cat([torch.cos(th / 2), torch.sin(th / 2) / th * r], dim=1)

    z = Z
    loss = (quat(z[:, 3:] + 1e-30) * torch.tensor(gq[0])).sum() + (z[:, :3] * torch.tensor(gt[0])).sum()
    for j in range(times.size - 1):
        h = (times[j + 1] - times[j]) / S
        for s in range(S):
            t = times[j] + s * h
            k1 = field(z, t)
            k2 = field(z + 0.5 * h * k1, t + 0.5 * h)
            k3 = field(z + 0.5 * h * k2, t + 0.5 * h)
            k4 = field(z + h * k3, t + h)
            z = z + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        loss = loss + (quat(z[:, 3:]) * torch.tensor(gq[j + 1])).sum() + \
            (z[:, :3] * torch.tensor(gt[j + 1])).sum()
    loss.backward()
    # at t0 the rotation is exactly zero: torch's r/|r| limit is taken on a
    # 1e-30 offset, whose derivative equals the small-angle branch's (0.5 I)
    np.testing.assert_allclose(dp, P.grad.numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(de, E.grad.numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dz, Z.grad.numpy(), rtol=1e-9, atol=1e-12)
