"""Plant plausible mistakes in copies of the learned-correction oracle and
confirm that its pins notice each one (CPU only)."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import magpie_oracle as O
from tests import learned_pins

FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "learned_oracle.py")


def fresh():
    spec = importlib.util.spec_from_file_location("learned_copy", FILE)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def m_kernel_transposed(L):
    orig = L.conv3x3
    L.conv3x3 = lambda x, W, b, s, up: orig(x, W.transpose(0, 2, 1, 3), b, s, up)


def m_no_relu_mask(L):
    def backward(theta, acts, dy, rounding=True):
        q = L.bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
        grads, dz = [], np.asarray(dy, dtype=np.float64)
        layers = list(zip(L.unpack(theta), L.LAYERS))
        for li in range(len(layers) - 1, -1, -1):
            (W, b), (_, _, s, up, relu) = layers[li]
            dx, dW, db = L.conv3x3_backward(acts[li], q(W), dz, s, up)
            grads.append((dW, db))
            dz = dx
        grads.reverse()
        return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
    L.backward = backward


def m_bf16_truncate(L):
    def bf16(a):
        f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        u = (f.view(np.uint32) >> 16) << 16
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    L.bf16 = bf16


def m_adam_no_bias_correction(L):
    def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        return theta - lr * m / (np.sqrt(v) + eps), m, v
    L.adam = adam


def m_plain_restriction(L):
    def coarse_chain(zk, Q, Rk, u, levels):
        Qs, zs, Rs, us = [Q], [zk], [Rk], [u]
        for _ in range(levels - 1):
            QH, Wz, WR, Wu = O.coarse_weights(Qs[-1])
            zs.append(O.restrict(zs[-1]))
            Rs.append(O.restrict(WR * Rs[-1]))
            us.append(Wu * O.restrict(us[-1]))
            Qs.append(QH)
        return Qs, zs, Rs, us
    L.coarse_chain = coarse_chain


def m_acceptance_inverted(L):
    orig = L.window_surrogate
    L.window_surrogate = lambda x, Q, Rk: -orig(x, Q, Rk)


def m_no_post_smoothing(L):
    def given(zk, Q, Rk, u, levels, eH):
        if levels == 1:
            return zk + eH
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(WR * Rk)
        uH = Wu * O.restrict(u)
        return zk + O.prolong(given(zH, QH, RH, uH, levels - 1, eH) - zH)
    L.magps_coarse_given = given


def m_stride_offset(L):
    def conv(x, W, b, stride, up):
        v = np.repeat(np.repeat(x, up, axis=1), up, axis=2) if up > 1 else x
        n, Hv, _, ci = v.shape
        Ho = Hv // stride
        vp = np.zeros((n, Hv + 3, Hv + 3, ci))
        vp[:, 1:Hv + 1, 1:Hv + 1] = v
        y = np.zeros((n, Ho, Ho, W.shape[0])) + b
        o = 1 if stride > 1 else 0
        for ky in range(3):
            for kx in range(3):
                p = vp[:, ky + o:ky + o + stride * Ho:stride, kx + o:kx + o + stride * Ho:stride, :]
                y += np.einsum("nijc,oc->nijo", p, W[:, ky, kx, :])
        return y
    L.conv3x3 = conv


def m_target_sign(L):
    orig = L.targets
    L.targets = lambda x0, zh_T, s: -orig(x0, zh_T, s)


def m_scale_not_rms(L):
    orig = L.coarse_state
    def cs(zk, Q, Rk, u, levels):
        x, s, e = orig(zk, Q, Rk, u, levels)
        x = x.copy()
        x[..., 2:4] *= 2.0
        return x, 0.5 * s, e
    L.coarse_state = cs


def m_adam_eps_inside_sqrt(L):
    def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** step)
        vh = v / (1.0 - b2 ** step)
        return theta - lr * mh / np.sqrt(vh + eps), m, v
    L.adam = adam


def m_adam_betas_swapped(L):
    orig = L.adam
    L.adam = lambda theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8: orig(theta, g, m, v, step, lr, b2, b1, eps)


def m_loss_grad_sum_not_mean(L):
    def lg(y, t):
        r = y - t
        return 0.5 * float(np.mean(r * r)), r
    L.loss_and_grad = lg


def m_upsample_tiled(L):
    orig = L.conv3x3

    def conv(x, W, b, stride, up):
        if up > 1:
            x = np.tile(x, (1, up, up, 1))
            return orig(x, W, b, stride, 1)
        return orig(x, W, b, stride, up)
    L.conv3x3 = conv


def m_backward_no_bias_grad(L):
    orig = L.conv3x3_backward

    def cb(x, W, dy, stride, up):
        dx, dW, db = orig(x, W, dy, stride, up)
        return dx, dW, np.zeros_like(db)
    L.conv3x3_backward = cb


def m_acceptance_strict(L):
    orig = L.learned_window

    def lw(zk, Q, Rk, u, levels, theta, rounding=True):
        out, acc, margin = orig(zk, Q, Rk, u, levels, theta, rounding)
        if acc and margin == 0.0:
            x, s, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
            return L.magps_coarse_given(zk, Q, Rk, u, levels, e_plain), False, margin
        return out, acc, margin
    L.learned_window = lw


def m_proposal_unscaled(L):
    def lw(zk, Q, Rk, u, levels, theta, rounding=True):
        x, s, e_plain = L.coarse_state(zk, Q, Rk, u, levels)
        plain = L.magps_coarse_given(zk, Q, Rk, u, levels, e_plain)
        if not s > L.O.TINY:
            return plain, False, 0.0
        y, _ = L.forward(theta, x[None], rounding)
        e_nn = e_plain + (y[0, ..., 0] + 1j * y[0, ..., 1])  # the scale s dropped
        learned = L.magps_coarse_given(zk, Q, Rk, u, levels, e_nn)
        margin = L.window_surrogate(plain, Q, Rk) - L.window_surrogate(learned, Q, Rk)
        return (learned, True, margin) if margin >= 0 else (plain, False, margin)
    L.learned_window = lw


def m_surrogate_no_half(L):
    L.window_surrogate = lambda x, Q, Rk: float(np.sum(np.abs(Q * x - Rk) ** 2))


def m_relu_on_output(L):
    orig = L.forward

    def fw(theta, x, rounding=True):
        out, acts = orig(theta, x, rounding)
        return np.maximum(out, 0.0), acts
    L.forward = fw


def m_bias_before_weights(L):
    def unpack(theta):
        out, o = [], 0
        for ci, co, _, _, _ in L.LAYERS:
            b = theta[o:o + co]
            o += co
            W = theta[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
            o += co * 9 * ci
            out.append((W, b))
        return out
    L.unpack = unpack


MUTANTS = [m_kernel_transposed, m_no_relu_mask, m_bf16_truncate, m_adam_no_bias_correction, m_plain_restriction,
           m_acceptance_inverted, m_no_post_smoothing, m_stride_offset, m_target_sign, m_scale_not_rms,
           m_adam_eps_inside_sqrt, m_adam_betas_swapped, m_loss_grad_sum_not_mean, m_upsample_tiled,
           m_backward_no_bias_grad, m_acceptance_strict, m_proposal_unscaled, m_surrogate_no_half,
           m_relu_on_output, m_bias_before_weights]


@pytest.mark.parametrize("mutant", MUTANTS, ids=lambda f: f.__name__)
def test_pins_catch(mutant):
    L = fresh()
    mutant(L)
    failed = []
    for check in learned_pins.ALL:
        try:
            check(L)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"no pin caught {mutant.__name__}"
