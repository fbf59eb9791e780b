"""FP64 oracle of the NeuralODE pose model (Sec. 3.2, Eqs. 3-4).

TEST INFRASTRUCTURE ONLY: used by the tests (and nothing in the product
path) to check the CUDA implementation of the pose model against a plain,
slow NumPy restatement in float64.

The object state is z(t) = [position, rotation] in R^6 (Sec. 3.2: the
refined 3D position and the rotation parameters R_t, initialised to zero).
Its evolution is the ODE of Eq. 3, dz/dt = f(z, t, c), with f a small
multilayer perceptron and c the object's instance embedding; Eq. 4 gives z at
later times by integration from z(t0). Readings (the paper names neither the
network nor the integrator):

  * f(z, t, c) = W3 tanh(W2 tanh(W1 [z, t, c] + b1) + b2) + b3, hidden width
    H, embedding width D;
  * the integral of Eq. 4 is taken with the classical fourth-order
    Runge-Kutta method, `substeps` equal steps between consecutive output
    times;
  * the rotation parameters are a rotation vector r (axis times angle); the
    object pose at time t is the rotation exp(r) as the unit quaternion
    (cos(|r|/2), sin(|r|/2) r/|r|) in (w, x, y, z) order and the translation
    z[0:3] (local -> world, the instance pose W_{t,i2g} of Sec. 3.3).

The parameters travel as one flat vector in the order W1 (H x (7 + D), row
major), b1 (H), W2 (H x H), b2 (H), W3 (6 x H), b3 (6); the embeddings as a
[K, D] array.

The gradient is the exact derivative of this discrete computation (reverse
mode through every Runge-Kutta stage), written out by hand below.
"""
from __future__ import annotations

import numpy as np

STATE = 6


def param_count(hidden: int, embed: int) -> int:
    return hidden * (7 + embed) + hidden + hidden * hidden + hidden + STATE * hidden + STATE


def unpack(params: np.ndarray, hidden: int, embed: int) -> dict:
    """Views of the flat parameter vector (the layout above)."""
    p = np.asarray(params, np.float64)
    H, I = hidden, 7 + embed
    sizes = [("W1", (H, I)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (STATE, H)),
             ("b3", (STATE,))]
    out, o = {}, 0
    for name, shape in sizes:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    assert o == p.size, (o, p.size)
    return out


def f(net: dict, z, t, c):
    """The network of Eq. 3 at one state; returns (dz/dt, cache for the VJP)."""
    x = np.concatenate([z, [t], c])
    h1 = np.tanh(net["W1"] @ x + net["b1"])
    h2 = np.tanh(net["W2"] @ h1 + net["b2"])
    return net["W3"] @ h2 + net["b3"], (x, h1, h2)


def f_vjp(net: dict, cache, ybar, grads: dict):
    """Vector-Jacobian product of f: adds the parameter adjoints to `grads`,
    returns the adjoint of the input x = [z, t, c]."""
    x, h1, h2 = cache
    grads["W3"] += np.outer(ybar, h2)
    grads["b3"] += ybar
    p2 = (net["W3"].T @ ybar) * (1.0 - h2 * h2)
    grads["W2"] += np.outer(p2, h1)
    grads["b2"] += p2
    p1 = (net["W2"].T @ p2) * (1.0 - h1 * h1)
    grads["W1"] += np.outer(p1, x)
    grads["b1"] += p1
    return net["W1"].T @ p1


def rk4_step(net: dict, z, t, h, c):
    """One classical Runge-Kutta step of Eq. 3 from (z, t) over h."""
    k1, _ = f(net, z, t, c)
    k2, _ = f(net, z + 0.5 * h * k1, t + 0.5 * h, c)
    k3, _ = f(net, z + 0.5 * h * k2, t + 0.5 * h, c)
    k4, _ = f(net, z + h * k3, t + h, c)
    return z + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def step_times(times, substeps: int):
    """(start time, step length) of every Runge-Kutta step of the trajectory:
    `substeps` equal steps between consecutive output times."""
    out = []
    for j in range(len(times) - 1):
        h = (float(times[j + 1]) - float(times[j])) / substeps
        for s in range(substeps):
            out.append((float(times[j]) + s * h, h))
    return out


def trajectory(params, embed, z0, times, substeps: int, hidden: int):
    """Eq. 4 for every instance: the states at every Runge-Kutta step
    boundary, [n_steps + 1, K, 6] (the output times are every `substeps`-th)."""
    emb = np.asarray(embed, np.float64)
    net = unpack(params, hidden, emb.shape[1])
    z = np.array(z0, np.float64)
    steps = step_times(times, substeps)
    out = np.zeros((len(steps) + 1,) + z.shape)
    out[0] = z
    for i, (t, h) in enumerate(steps):
        for k in range(z.shape[0]):
            z[k] = rk4_step(net, z[k], t, h, emb[k])
        out[i + 1] = z
    return out


def quat_from_rotvec(r):
    """exp(r) as a unit quaternion (w, x, y, z)."""
    r = np.asarray(r, np.float64)
    th = np.linalg.norm(r)
    if th < 1e-12:
        return np.array([1.0, 0.5 * r[0], 0.5 * r[1], 0.5 * r[2]])
    s = np.sin(0.5 * th) / th
    return np.array([np.cos(0.5 * th), s * r[0], s * r[1], s * r[2]])


def quat_from_rotvec_vjp(r, gq):
    """Adjoint of r given the adjoint gq of quat_from_rotvec(r)."""
    r = np.asarray(r, np.float64)
    th = np.linalg.norm(r)
    if th < 1e-12:
        return 0.5 * np.asarray(gq[1:], np.float64)
    s = np.sin(0.5 * th) / th
    # d cos(th/2)/dr = -sin(th/2)/2 * r/th; d(s r)/dr = s I + r (ds/dth) r^T / th
    ds = (0.5 * np.cos(0.5 * th) * th - np.sin(0.5 * th)) / (th * th)
    g = -0.5 * np.sin(0.5 * th) / th * gq[0] * r
    g = g + s * np.asarray(gq[1:]) + r * (ds / th) * float(np.dot(r, gq[1:]))
    return g


def poses(states, substeps: int):
    """Instance poses at the output times: quaternions [T, K, 4] and
    translations [T, K, 3] from the states at every `substeps`-th boundary."""
    zs = states[::substeps]
    q = np.zeros(zs.shape[:2] + (4,))
    for j in range(zs.shape[0]):
        for k in range(zs.shape[1]):
            q[j, k] = quat_from_rotvec(zs[j, k, 3:6])
    return q, zs[:, :, 0:3].copy()


def backward(params, embed, z0, times, substeps: int, hidden: int, g_quat, g_trans):
    """Exact gradient of sum_t <g_quat[t], quat[t]> + <g_trans[t], trans[t]>
    w.r.t. the flat parameters, the embeddings and z0 (reverse mode through
    every Runge-Kutta stage of `trajectory`)."""
    emb = np.asarray(embed, np.float64)
    D = emb.shape[1]
    net = unpack(params, hidden, D)
    states = trajectory(params, embed, z0, times, substeps, hidden)
    steps = step_times(times, substeps)
    K = states.shape[1]
    gflat = np.zeros(param_count(hidden, D))
    grads = unpack(gflat, hidden, D)   # views into gflat
    gemb = np.zeros_like(emb)
    gz0 = np.zeros((K, STATE))
    for k in range(K):
        c = emb[k]
        abar = np.zeros(STATE)
        for i in range(len(steps), -1, -1):
            if i % substeps == 0:
                j = i // substeps
                abar[0:3] += g_trans[j, k]
                abar[3:6] += quat_from_rotvec_vjp(states[i, k, 3:6], g_quat[j, k])
            if i == 0:
                break
            t, h = steps[i - 1]
            z = states[i - 1, k]
            # forward stages of the step, with their caches
            k1, c1 = f(net, z, t, c)
            u2 = z + 0.5 * h * k1
            k2, c2 = f(net, u2, t + 0.5 * h, c)
            u3 = z + 0.5 * h * k2
            k3, c3 = f(net, u3, t + 0.5 * h, c)
            u4 = z + h * k3
            _, c4 = f(net, u4, t + h, c)
            # z' = z + h/6 (k1 + 2 k2 + 2 k3 + k4)
            zbar = abar.copy()
            kb1 = (h / 6.0) * abar
            kb2 = (h / 3.0) * abar
            kb3 = (h / 3.0) * abar
            kb4 = (h / 6.0) * abar
            x4 = f_vjp(net, c4, kb4, grads)
            gemb[k] += x4[7:]
            zbar += x4[0:6]
            kb3 = kb3 + h * x4[0:6]
            x3 = f_vjp(net, c3, kb3, grads)
            gemb[k] += x3[7:]
            zbar += x3[0:6]
            kb2 = kb2 + 0.5 * h * x3[0:6]
            x2 = f_vjp(net, c2, kb2, grads)
            gemb[k] += x2[7:]
            zbar += x2[0:6]
            kb1 = kb1 + 0.5 * h * x2[0:6]
            x1 = f_vjp(net, c1, kb1, grads)
            gemb[k] += x1[7:]
            zbar += x1[0:6]
            abar = zbar
        gz0[k] = abar
    return gflat, gemb, gz0
