"""Checks that pin the learned-correction oracle to things other than itself:
library routines (PyTorch's bfloat16 conversion, conv2d and autograd in
float64), closed forms of Adam, and special cases that reduce to the plain
MAGPS of the main oracle.  Each takes the learned-oracle module `L` so that
the mutation tests can run them on planted copies."""
from __future__ import annotations

import numpy as np
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def random_theta(L, seed=0, scale=1.0):
    """He-scaled random parameters for every layer, biases included."""
    rng = _rng(seed)
    parts = []
    for ci, co, _, _, _ in L.LAYERS:
        parts.append(rng.normal(0.0, scale * np.sqrt(2.0 / (9 * ci)), co * 9 * ci))
        parts.append(rng.normal(0.0, 0.1, co))
    return np.concatenate(parts)


def bf16_rounding(L):
    """Round-to-nearest-even against PyTorch's float32 -> bfloat16 cast, plus
    the halfway cases written out."""
    x = _rng(1).normal(0, 10, 4096).astype(np.float32)
    x[:4] = [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = L.bf16(x)
    assert np.array_equal(got, ref)
    assert got[1] == 1.0 and got[2] == 1.0 + 2 ** -6 and got[3] == 1.0 + 2 ** -7


def _torch_conv(x, W, b, stride, up):
    xt = torch.from_numpy(np.ascontiguousarray(x.transpose(0, 3, 1, 2)))
    if up > 1:
        xt = xt.repeat_interleave(up, dim=2).repeat_interleave(up, dim=3)
    Wt = torch.from_numpy(np.ascontiguousarray(W.transpose(0, 3, 1, 2)))
    y = torch.nn.functional.conv2d(xt, Wt, torch.from_numpy(b), stride=stride, padding=1)
    return y.numpy().transpose(0, 2, 3, 1)


def conv_matches_library(L):
    """conv3x3 = PyTorch conv2d (float64, padding 1) on the nearest-upsampled
    input, for every (stride, upsample) the network uses."""
    rng = _rng(2)
    for stride, up in ((1, 1), (2, 1), (1, 2), (1, 4)):
        x = rng.normal(size=(2, 8, 8, 5))
        W = rng.normal(size=(3, 3, 3, 5))
        b = rng.normal(size=3)
        assert np.allclose(L.conv3x3(x, W, b, stride, up), _torch_conv(x, W, b, stride, up), atol=1e-12)


def conv_special_cases(L):
    """A centred delta kernel is the identity; a corner delta is a shift with
    zero fill; stride 2 keeps the even outputs of stride 1."""
    rng = _rng(3)
    x = rng.normal(size=(1, 6, 6, 2))
    W = np.zeros((2, 3, 3, 2))
    W[0, 1, 1, 0] = W[1, 1, 1, 1] = 1.0
    assert np.allclose(L.conv3x3(x, W, np.zeros(2), 1, 1), x)
    W = np.zeros((1, 3, 3, 2))
    W[0, 0, 0, 1] = 1.0
    y = L.conv3x3(x, W, np.zeros(1), 1, 1)[0, ..., 0]
    assert np.allclose(y[1:, 1:], x[0, :-1, :-1, 1]) and np.all(y[0] == 0) and np.all(y[:, 0] == 0)
    W = rng.normal(size=(3, 3, 3, 2))
    assert np.allclose(L.conv3x3(x, W, np.ones(3), 2, 1), L.conv3x3(x, W, np.ones(3), 1, 1)[:, ::2, ::2])


def _torch_net(L, theta, x):
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    a = torch.from_numpy(np.ascontiguousarray(x.transpose(0, 3, 1, 2)))
    o = 0
    for ci, co, s, up, relu in L.LAYERS:
        W = th[o:o + co * 9 * ci].reshape(co, 3, 3, ci).permute(0, 3, 1, 2)
        o += co * 9 * ci
        b = th[o:o + co]
        o += co
        if up > 1:
            a = a.repeat_interleave(up, dim=2).repeat_interleave(up, dim=3)
        a = torch.nn.functional.conv2d(a, W, b, stride=s, padding=1)
        if relu:
            a = torch.relu(a)
    return th, a.permute(0, 2, 3, 1)


def network_matches_autograd(L):
    """Forward and backward (no BF16 rounding) = the same network written with
    PyTorch conv2d in float64, gradient by autograd."""
    theta = random_theta(L, 4)
    rng = _rng(5)
    x = rng.normal(size=(2, 8, 8, 4))
    dy = rng.normal(size=(2, 8, 8, 2))
    y, acts = L.forward(theta, x, rounding=False)
    th, yt = _torch_net(L, theta, x)
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-10, atol=1e-10)
    (yt * torch.from_numpy(dy)).sum().backward()
    g = L.backward(theta, acts, dy, rounding=False)
    ref = th.grad.numpy()
    assert np.linalg.norm(g - ref) <= 1e-10 * np.linalg.norm(ref)


def backward_finite_difference(L):
    """<grad, v> against a central difference of <dy, y(theta)> along a random v."""
    theta = random_theta(L, 6)
    rng = _rng(7)
    x = rng.normal(size=(1, 8, 8, 4))
    dy = rng.normal(size=(1, 8, 8, 2))
    v = rng.normal(size=theta.shape)
    _, acts = L.forward(theta, x, rounding=False)
    g = L.backward(theta, acts, dy, rounding=False)
    eps = 1e-6
    fp = np.sum(dy * L.forward(theta + eps * v, x, rounding=False)[0])
    fm = np.sum(dy * L.forward(theta - eps * v, x, rounding=False)[0])
    assert abs((fp - fm) / (2 * eps) - g @ v) <= 1e-6 * abs(g @ v)


def rounded_network_close(L):
    """With BF16 rounding the output stays within the BF16 error growth of
    the unrounded network."""
    theta = random_theta(L, 8)
    x = _rng(9).normal(size=(2, 8, 8, 4))
    y1, _ = L.forward(theta, x, rounding=True)
    y0, _ = L.forward(L.bf16(theta), L.bf16(x), rounding=False)
    assert np.linalg.norm(y1 - y0) <= 0.05 * np.linalg.norm(y0)
    assert not np.array_equal(y1, y0)


def adam_closed_forms(L):
    """Step 1 moves every weight by -lr g / (|g| + eps); a constant gradient
    keeps the bias-corrected moments at (g, g^2), so every step is the same."""
    rng = _rng(10)
    g = rng.normal(size=100)
    th = rng.normal(size=100)
    m = np.zeros(100)
    v = np.zeros(100)
    lr = 1e-3
    th1, m, v = L.adam(th, g, m, v, 1, lr)
    assert np.allclose(th1 - th, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    for t in range(2, 6):
        th2, m, v = L.adam(th1, g, m, v, t, lr)
        assert np.allclose(th2 - th1, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
        th1 = th2
    # a gradient g then 0: the second step's bias-corrected moments are
    # b1 g / (1 + b1) and b2 g^2 / (1 + b2) (Kingma and Ba, Algorithm 1, two
    # steps written out), so it moves by -lr (b1/(1+b1)) g / (sqrt(b2/(1+b2)) |g| + eps)
    b1, b2 = 0.9, 0.999
    th1, m1, v1 = L.adam(th, g, np.zeros(100), np.zeros(100), 1, lr)
    th2, _, _ = L.adam(th1, np.zeros(100), m1, v1, 2, lr)
    expect = -lr * (b1 / (1 + b1)) * g / (np.sqrt(b2 / (1 + b2)) * np.abs(g) + 1e-8)
    assert np.allclose(th2 - th1, expect, rtol=1e-9, atol=0)


def loss_gradient(L):
    """dL/dy of L = 1/2 mean((y-t)^2) against a central difference."""
    rng = _rng(11)
    y = rng.normal(size=(2, 4, 4, 2))
    t = rng.normal(size=y.shape)
    l0, g = L.loss_and_grad(y, t)
    assert np.isclose(l0, 0.5 * np.sum((y - t) ** 2) / y.size)
    v = rng.normal(size=y.shape)
    eps = 1e-6
    d = (L.loss_and_grad(y + eps * v, t)[0] - L.loss_and_grad(y - eps * v, t)[0]) / (2 * eps)
    assert np.isclose(d, np.sum(g * v), rtol=1e-7)


def _window(seed=12, m=32, levels=3):
    rng = _rng(seed)
    Q = synth.make_probe(m).astype(np.complex128)
    zk = (0.8 + 0.2 * rng.random((m, m))) * np.exp(1j * rng.normal(0, 0.5, (m, m)))
    zt = (0.8 + 0.2 * rng.random((m, m))) * np.exp(1j * rng.normal(0, 0.5, (m, m)))
    dk = np.abs(O.fft2(Q * zt)) ** 2
    u = O.rpie_regulariser(Q, 0.1)
    Rk = O.revised_exit_wave(zk, Q, dk)
    return zk, Q, Rk, u, dk, levels


def coarse_state_is_residual_chain(L):
    """The coarse residual gradient of the literal z/R restriction chain equals
    the chain g^(l+1) = W_u^l I_h^H g^l started from g^0 = conj(Q)(R - Q z)
    (first-order consistency of the coarse surrogate), and e_plain is the
    coarsest proximal step of Algorithm MAGPS."""
    zk, Q, Rk, u, _, levels = _window()
    Qs, zs, Rs, us = L.coarse_chain(zk, Q, Rk, u, levels)
    g = np.conj(Q) * (Rk - Q * zk)
    Ql = Q
    for _ in range(levels - 1):
        _, _, _, Wu = O.coarse_weights(Ql)
        g = Wu * O.restrict(g)
        Ql = O.restrict(Ql)
    gH = np.conj(Qs[-1]) * (Rs[-1] - Qs[-1] * zs[-1])
    assert np.allclose(gH, g, atol=1e-12 * np.abs(g).max())
    x, s, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
    step = O.magps(zs[-1], Qs[-1], Rs[-1], us[-1], 1) - zs[-1]
    assert np.allclose(e_plain, step, atol=1e-13)
    assert np.isclose(np.mean(x[..., 2] ** 2 + x[..., 3] ** 2), 1.0)
    assert np.allclose(x[..., 0] + 1j * x[..., 1], zs[-1])


def plain_coarse_step_is_magps(L):
    """Given the plain coarse step, the learned V-cycle is Algorithm MAGPS; a
    zero last layer proposes exactly that step and is accepted (margin 0)."""
    zk, Q, Rk, u, _, levels = _window()
    _, _, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
    ref = O.magps(zk, Q, Rk, u, levels)
    assert np.allclose(L.magps_coarse_given(zk, Q, Rk, u, levels, e_plain), ref, atol=1e-13)
    theta = random_theta(L, 13)
    n_last = 64 * 9 * 2 + 2
    theta[-n_last:] = 0.0
    out, acc, margin = L.learned_window(zk, Q, Rk, u, levels, theta)
    assert acc and margin == 0.0 and np.allclose(out, ref, atol=1e-13)


def acceptance_rule(L):
    """A wild proposal raises the window surrogate and is rejected (the output
    is the plain V-cycle); the plain coarse step scaled slightly is assessed by
    the surrogate values written out."""
    zk, Q, Rk, u, _, levels = _window()
    theta = random_theta(L, 14, scale=30.0)
    out, acc, margin = L.learned_window(zk, Q, Rk, u, levels, theta)
    ref = O.magps(zk, Q, Rk, u, levels)
    assert not acc and margin < 0 and np.allclose(out, ref, atol=1e-13)
    _, _, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
    for f in (0.5, 1.5):
        a = L.magps_coarse_given(zk, Q, Rk, u, levels, f * e_plain)
        lhs = 0.5 * np.sum(np.abs(Q * a - Rk) ** 2)
        assert np.isclose(L.window_surrogate(a, Q, Rk), lhs)


def proposal_in_units_of_the_scale(L):
    """The network's output is in units of the window's scale s (the RMS of
    the plain coarse step): a network whose last layer has zero weights and
    biases (b0, b1) outputs y = b everywhere, and the proposal is then
    e_plain + s (b0 + i b1); the window's margin is the surrogate of the plain
    output minus that of the V-cycle built on that proposal."""
    zk, Q, Rk, u, _, levels = _window()
    theta = random_theta(L, 18)
    theta[-(64 * 9 * 2 + 2):] = 0.0
    theta[-2:] = (0.03, -0.02)
    _, acc, margin = L.learned_window(zk, Q, Rk, u, levels, theta)
    _, s, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
    b = complex(float(np.float32(0.03)), float(np.float32(-0.02)))  # the FP32 output, held in FP64
    prop = L.magps_coarse_given(zk, Q, Rk, u, levels, e_plain + s * b)
    plain = L.magps_coarse_given(zk, Q, Rk, u, levels, e_plain)
    expect = 0.5 * np.sum(np.abs(Q * plain - Rk) ** 2) - 0.5 * np.sum(np.abs(Q * prop - Rk) ** 2)
    assert s > 0 and abs(margin - expect) <= 1e-9 * max(abs(expect), 1e-300), (margin, expect)
    assert acc == (expect >= 0)


def minibatch_reduces_to_plain(L):
    """With a zero last layer the learned minibatch step is the plain one."""
    w = synth.WORKLOADS["tiny"]
    z_true, Q, pos = synth.make_problem(w)
    d = O.forward_intensities(z_true, Q, pos)
    u = O.rpie_regulariser(Q, w.alpha)
    z = np.ones((w.n, w.n), dtype=np.complex128)
    theta = random_theta(L, 15)
    theta[-(64 * 9 * 2 + 2):] = 0.0
    batch = list(range(5))
    zl, acc, _ = L.learned_minibatch_step(z, Q, pos, d, u, w.levels, batch, theta)
    zp = O.minibatch_step(z, Q, pos, d, u, w.levels, batch)
    assert acc.all() and np.allclose(zl, zp, atol=1e-12)


def stacked_windows_are_independent(L):
    """Windows tiled without overlap into one object and updated as one
    minibatch evolve exactly as separate one-window MAGPS problems: the
    trajectories the network is trained on."""
    zk, Q, Rk, u, dk, levels = _window(16)
    zk2, _, _, _, dk2, _ = _window(17)
    m = Q.shape[0]
    z = np.concatenate([zk, zk2], axis=0)
    pos = np.array([[0, 0], [m, 0]])
    d = np.stack([dk, dk2])
    out = O.minibatch_step(z, Q, pos, d, u, levels, [0, 1])
    for i, (zi, di) in enumerate(((zk, dk), (zk2, dk2))):
        ref = O.magps(zi, Q, O.revised_exit_wave(zi, Q, di), u, levels)
        assert np.allclose(out[i * m:(i + 1) * m], ref, atol=1e-12)


def targets_definition(L):
    """A trajectory that moved z_H by exactly the plain step has target 0; one
    that moved it by twice the plain step has target e_plain / s."""
    rng = _rng(18)
    x0 = rng.normal(size=(3, 4, 4, 4))
    s = np.array([0.5, 2.0, 1.0])
    e = (x0[..., 2] + 1j * x0[..., 3]) * s[:, None, None]
    zh_T = np.stack([x0[..., 0] + e.real, x0[..., 1] + e.imag], axis=-1)
    assert np.allclose(L.targets(x0, zh_T, s), 0.0, atol=1e-14)
    zh_T = np.stack([x0[..., 0] + 2 * e.real, x0[..., 1] + 2 * e.imag], axis=-1)
    assert np.allclose(L.targets(x0, zh_T, s), x0[..., 2:4], atol=1e-14)


ALL = [bf16_rounding, conv_matches_library, conv_special_cases, network_matches_autograd,
       backward_finite_difference, rounded_network_close, adam_closed_forms, loss_gradient,
       coarse_state_is_residual_chain, plain_coarse_step_is_magps, acceptance_rule,
       minibatch_reduces_to_plain, stacked_windows_are_independent, targets_definition, proposal_in_units_of_the_scale]
