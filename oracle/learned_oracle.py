"""FP64 reference of the learned coarse-level correction (test infrastructure,
not product code).

The paper's MAGPS (Algorithm MAGPS) ends its recursion on the coarsest grid
with one proximal step.  The learned form keeps every other step and lets a
small convolutional network propose that coarsest-level correction instead;
the paper has no such network, so everything here is a reading, listed with
its reasons in the design notes of the repository:

  * Network input (4 channels on the coarsest grid, side h = m / 2^(L-1)):
    the coarse object z_H (the paper's weighted restriction chain
    z^(l+1) = I_h^H (W_z^l . z^l)) and the plain coarse step
    e_plain = c^(L-1) . (R^(L-1) - Q^(L-1) z^(L-1)) = g_H / w_H, i.e. the coarse
    residual gradient g_H = conj(Q_H)(R_H - Q_H z_H) scaled by the coarse
    proximal weight w_H = u_H + |Q_H|^2.  e_plain is divided by its RMS s over
    the window, so the network sees unit-scale data.
  * Network output y (2 channels): the proposal is e_nn = e_plain + s . y; with
    a zero last layer the proposal is the plain coarse step.
  * Acceptance: the window's quadratic surrogate of Eq. (quadratic_surrogate),
    Phi~_k(x) = 1/2 || Q . x - R_k(z_k) ||^2 (it majorises Phi_k and equals it
    at z_k), is evaluated at the V-cycle's output with e_nn and with e_plain;
    the learned output is kept only when its value is not larger, otherwise
    the plain V-cycle output is used (the plain coarse solve is both the
    fallback and the yardstick the proposal is measured against).
  * Training target: the change of the window's coarse object z_H between
    the input state and a later state of the plain solver (its final state,
    or T further V-cycles of that window alone with refreshed R), in the
    network's scaled units: t = (z_H^(T) - z_H^(0)) / s - e_plain / s.
  * Arithmetic of the network as the CUDA path does it: BF16 weights and
    BF16 activations between layers, products accumulated in FP32 (here
    FP64), FP32 biases.  `bf16` rounds to nearest even.

Only the test suite and the benchmark's CPU legs may import this module.
"""
from __future__ import annotations

import numpy as np

from oracle import magpie_oracle as O

# -------------------------------------------------------------- architecture
# (c_in, c_out, stride, upsample, relu): 3x3 convolutions with zero padding 1;
# spatial sides h, h, h/2, h/4, h/8, h/4, h.
LAYERS = (
    (4, 32, 1, 1, True),
    (32, 64, 2, 1, True),
    (64, 128, 2, 1, True),
    (128, 512, 2, 1, True),
    (512, 64, 1, 2, True),
    (64, 2, 1, 4, False),
)


def param_count() -> int:
    """Weights [c_out][3][3][c_in] then biases [c_out], layer after layer."""
    return sum(co * 9 * ci + co for ci, co, _, _, _ in LAYERS)


def unpack(theta: np.ndarray):
    """Split the flat parameter vector into per-layer (W [co,3,3,ci], b [co])."""
    out, o = [], 0
    for ci, co, _, _, _ in LAYERS:
        W = theta[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def bf16(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64.  Inputs are first rounded to float32."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    r = r.astype(np.uint32).view(np.float32).astype(np.float64)
    r[nan] = np.nan
    return r


# --------------------------------------------------------------- convolution
def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray, stride: int, up: int) -> np.ndarray:
    """y[n, i, j, co] = b[co] + sum_{ky,kx,ci} W[co,ky,kx,ci] v[n, s i + ky - 1, s j + kx - 1, ci]
    where v is x upsampled by `up` (nearest neighbour) and v = 0 outside.
    x: [n, H, H, ci] -> y: [n, H up / s, H up / s, co]."""
    v = np.repeat(np.repeat(x, up, axis=1), up, axis=2) if up > 1 else x
    n, Hv, _, ci = v.shape
    Ho = Hv // stride
    vp = np.zeros((n, Hv + 2, Hv + 2, ci))
    vp[:, 1:Hv + 1, 1:Hv + 1] = v
    y = np.zeros((n, Ho, Ho, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            patch = vp[:, ky:ky + stride * Ho:stride, kx:kx + stride * Ho:stride, :]
            y += np.einsum("nijc,oc->nijo", patch, W[:, ky, kx, :])
    return y


def conv3x3_backward(x, W, dy, stride: int, up: int):
    """Adjoint of conv3x3 in its input and weights: (dx, dW, db)."""
    v = np.repeat(np.repeat(x, up, axis=1), up, axis=2) if up > 1 else x
    n, Hv, _, ci = v.shape
    Ho = dy.shape[1]
    vp = np.zeros((n, Hv + 2, Hv + 2, ci))
    vp[:, 1:Hv + 1, 1:Hv + 1] = v
    dvp = np.zeros_like(vp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(ky, ky + stride * Ho, stride), slice(kx, kx + stride * Ho, stride), slice(None))
            dW[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, vp[sl])
            dvp[sl] += np.einsum("nijo,oc->nijc", dy, W[:, ky, kx, :])
    dv = dvp[:, 1:Hv + 1, 1:Hv + 1]
    if up > 1:
        H = Hv // up
        dx = dv.reshape(n, H, up, H, up, ci).sum(axis=(2, 4))
    else:
        dx = dv
    return dx, dW, dy.sum(axis=(0, 1, 2))


def forward(theta: np.ndarray, x: np.ndarray, rounding: bool = True):
    """Network output and the stored activations [a0 .. a5] (inputs of the six
    layers).  With `rounding`, weights, the input and each hidden activation
    are rounded to BF16 as the CUDA path stores them; the output stays FP32."""
    q = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    acts = [q(x)]
    a = acts[0]
    for li, ((W, b), (_, _, s, up, relu)) in enumerate(zip(unpack(theta), LAYERS)):
        y = conv3x3(a, q(W), np.asarray(b, dtype=np.float64), s, up)
        if relu:
            a = q(np.maximum(y, 0.0))
            acts.append(a)
        else:
            out = y if not rounding else np.asarray(y, dtype=np.float32).astype(np.float64)
    return out, acts


def backward(theta: np.ndarray, acts, dy: np.ndarray, rounding: bool = True) -> np.ndarray:
    """Gradient of <dy, forward(theta, x)> with respect to theta, through the
    stored activations (ReLU derivative 1 where the activation is > 0; the
    BF16 roundings are passed straight through)."""
    q = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    grads = []
    dz = np.asarray(dy, dtype=np.float64)
    layers = list(zip(unpack(theta), LAYERS))
    for li in range(len(layers) - 1, -1, -1):
        (W, b), (_, _, s, up, relu) = layers[li]
        dx, dW, db = conv3x3_backward(acts[li], q(W), dz, s, up)
        grads.append((dW, db))
        if li > 0:
            dz = dx * (acts[li] > 0)
    grads.reverse()
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


# ----------------------------------------------------------------- training
def loss_and_grad(y: np.ndarray, t: np.ndarray):
    """L = 1/2 mean((y - t)^2) over every output value, and dL/dy."""
    r = y - t
    return 0.5 * float(np.mean(r * r)), r / r.size


def adam(theta, g, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) with bias correction;
    `step` counts from 1.  Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def targets(x0: np.ndarray, zh_T: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Training targets t = (z_H^(T) - z_H^(0)) / s - e_plain / s in the
    network's units; x0 channels are (Re z_H, Im z_H, Re e_plain/s, Im e_plain/s)."""
    s = scale.reshape(-1, 1, 1, 1)
    inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    return (zh_T - x0[..., 0:2]) * inv - x0[..., 2:4]


# ------------------------------------------------------- coarse-level state
def coarse_chain(zk, Q, Rk, u, levels: int):
    """The restriction chain of Algorithm MAGPS down to the coarsest grid:
    lists of (Q^l, z^l, R^l, u^l) for l = 0 .. levels-1."""
    Qs, zs, Rs, us = [Q], [zk], [Rk], [u]
    for _ in range(levels - 1):
        QH, Wz, WR, Wu = O.coarse_weights(Qs[-1])
        zs.append(O.restrict(Wz * zs[-1]))
        Rs.append(O.restrict(WR * Rs[-1]))
        us.append(Wu * O.restrict(us[-1]))
        Qs.append(QH)
    return Qs, zs, Rs, us


def coarse_state(zk, Q, Rk, u, levels: int):
    """Network input x [h, h, 4], the scale s and the plain coarse step
    e_plain of one window (module docstring)."""
    Qs, zs, Rs, us = coarse_chain(zk, Q, Rk, u, levels)
    QH, zH, RH, uH = Qs[-1], zs[-1], Rs[-1], us[-1]
    e_plain = O.safe_div(np.conj(QH), uH + np.abs(QH) ** 2) * (RH - QH * zH)
    s = float(np.sqrt(np.mean(np.abs(e_plain) ** 2)))
    inv = 1.0 / s if s > O.TINY else 0.0
    x = np.stack([zH.real, zH.imag, (e_plain * inv).real, (e_plain * inv).imag], axis=-1)
    return x, s, e_plain


def magps_coarse_given(zk, Q, Rk, u, levels: int, eH):
    """Algorithm MAGPS with the coarsest-level correction replaced by `eH`
    (levels >= 2): restriction, z~ = z + I_H^h e on the way up and one
    post-smoothing proximal step per level, as in the plain algorithm."""
    if levels == 1:
        return zk + eH
    QH, Wz, WR, Wu = O.coarse_weights(Q)
    zH = O.restrict(Wz * zk)
    RH = O.restrict(WR * Rk)
    uH = Wu * O.restrict(u)
    zH_hat = magps_coarse_given(zH, QH, RH, uH, levels - 1, eH)
    z_tilde = zk + O.prolong(zH_hat - zH)
    return O.proximal_step(z_tilde, Q, Rk, u)


def window_surrogate(x, Q, Rk) -> float:
    """Phi~_k(x; z_k) = 1/2 || Q . x - R_k(z_k) ||^2 (Eq. quadratic_surrogate)."""
    return 0.5 * float(np.sum(np.abs(Q * x - Rk) ** 2))


def learned_window(zk, Q, Rk, u, levels: int, theta, rounding: bool = True):
    """One window of the learned V-cycle: (z_hat, accepted, margin), where
    margin = Phi~(plain output) - Phi~(learned output) (accepted iff >= 0)."""
    x, s, e_plain = coarse_state(zk, Q, Rk, u, levels)
    plain = magps_coarse_given(zk, Q, Rk, u, levels, e_plain)
    if not s > O.TINY:
        return plain, False, 0.0
    y, _ = forward(theta, x[None], rounding)
    e_nn = e_plain + s * (y[0, ..., 0] + 1j * y[0, ..., 1])
    learned = magps_coarse_given(zk, Q, Rk, u, levels, e_nn)
    margin = window_surrogate(plain, Q, Rk) - window_surrogate(learned, Q, Rk)
    return (learned, True, margin) if margin >= 0 else (plain, False, margin)


def learned_minibatch_step(z, Q, positions, d, u, levels, batch, theta, rounding: bool = True):
    """The minibatch step of the plain method (same combination with weights
    w = u + |Q|^2) with every window's MAGPS replaced by `learned_window`.
    Returns (z, accepted flags, margins) in batch order."""
    z = np.asarray(z, dtype=np.complex128)
    m = Q.shape[0]
    w = u + np.abs(Q) ** 2
    num = np.zeros(z.shape, dtype=np.complex128)
    den = np.zeros(z.shape, dtype=np.float64)
    acc, margins = [], []
    for k in batch:
        r, c = positions[k]
        zk = z[r:r + m, c:c + m]
        Rk = O.revised_exit_wave(zk, Q, d[k])
        zh, a, mg = learned_window(zk, Q, Rk, u, levels, theta, rounding)
        acc.append(a)
        margins.append(mg)
        num[r:r + m, c:c + m] += w * (zh - zk)
        den[r:r + m, c:c + m] += w
    out = z.copy()
    lit = den > 0
    out[lit] += num[lit] / den[lit]
    return out, np.array(acc), np.array(margins)
