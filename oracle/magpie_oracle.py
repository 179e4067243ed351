"""FP64 reference of the MAGPIE sweep (test infrastructure, not product code).

A plain, slow, NumPy float64/complex128 statement of what the method
computes, written to be checked against the paper by eye.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import
it; the CUDA library never calls it and shares no code with it.

Notation follows the paper: z object, Q probe, P_k the k-th m x m scan
window, d_k measured intensities, R_k the revised exit wave, u the
regulariser, I_h^H the 2x2 averaging restriction and I_H^h = 4 (I_h^H)^T the
prolongation.  F is the unnormalised 2-D DFT and F^{-1} = F^* / m^2
(appendix "Computation for complex gradients").  The 2-D DFT itself is a
library primitive (numpy.fft), pinned against the defining double sum in
the tests.

Readings where the paper is silent (listed with their reasons in the design
notes of the repository):
  * theta(0) := 0 at every iteration (the definition of the revised exit
    wave, footnote).  The recycling rule of Eq. (specification) is available
    through `prev_phase` but is not the default.  -- parity unpinned
  * Division rule: any element-wise quotient whose denominator has modulus
    <= 1e-30 is set to 0 (W_z, W_R, W_u^H and the proximal factor
    conj(Q) / (u + |Q|^2) at coarse levels, where the complex bin mean of Q
    can vanish).  -- parity unpinned
  * Probe step (optional, off by default; the paper keeps Q fixed and names
    blind ptychography as future work): the same surrogate minimised over Q
    with the object fixed, by the symmetry of 1/2 || Q . z_k - R_k ||^2 in Q
    and z_k: Q <- Q + sum_k conj(z_k)(R_k - Q z_k) / sum_k (u_Q,k + |z_k|^2),
    u_Q,k = beta (max |z_k|^2 - |z_k|^2), all windows of the minibatch from the
    same (z, Q).  -- parity pinned only as the exact minimiser of that
    proximal surrogate and by full-batch monotone descent
  * Variants (off by default): the MG/OPT correction term of Algorithm
    MG/OPT on every coarse problem (`magps_mgopt`), and the phase rule of
    Eq. (specification) across visits of a window
    (`minibatch_step_variant`).  -- pinned by their special cases (no
    effect where the probe is constant on every 2x2 bin, resp. where no
    spectrum entry is exactly 0) and by the first-order matching the
    correction term enforces
  * Minibatch step: the paper updates one window at a time (Algorithm
    MAGPIE).  For a minibatch every window starts from the same z; the
    increments Delta_k are combined as z <- z + sum_k P_k^T (w . Delta_k) /
    sum_k P_k^T w with w = u + |Q|^2 (on pixels where the denominator is
    > 0).  For one level this is the exact minimiser of the proximal
    surrogate summed over the minibatch (Eq. proximal_point_method summed
    over k); for a minibatch of one it is Algorithm MAGPIE.  Pinned by those
    two special cases; the multilevel weighting itself is a reading.
"""
from __future__ import annotations

import numpy as np

TINY = 1e-30  # division rule threshold (see module docstring)


# ---------------------------------------------------------------- transforms
def fft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2-D DFT: (Fx)[p,q] = sum_{a,b} x[a,b] e^{-2 pi i (pa+qb)/m}."""
    return np.fft.fft2(x)


def ifft2(x: np.ndarray) -> np.ndarray:
    """F^{-1} = F^* / m^2 (appendix, Parseval argument)."""
    return np.fft.ifft2(x)


# ------------------------------------------- restriction and prolongation
def restrict(a: np.ndarray) -> np.ndarray:
    """I_h^H of Eq. (restriction_operator): mean of each 2x2 bin."""
    return 0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2])


def prolong(b: np.ndarray) -> np.ndarray:
    """I_H^h = 4 (I_h^H)^T of Eq. (prolongation_operator): copy into the bin."""
    return np.repeat(np.repeat(b, 2, axis=0), 2, axis=1)


def safe_div(num, den):
    """Element-wise num / den, 0 where |den| <= TINY (division rule)."""
    num = np.asarray(num)
    den = np.asarray(den)
    ok = np.abs(den) > TINY
    out = np.zeros(np.broadcast(num, den).shape, dtype=np.result_type(num, den, np.float64))
    np.divide(num, den, out=out, where=ok)
    return out


# ------------------------------------------------------------ scan windows
def extract(z: np.ndarray, pos, m: int) -> np.ndarray:
    """z_k = P_k z: the m x m window whose top-left corner is pos = (row, col)."""
    r, c = int(pos[0]), int(pos[1])
    return z[r:r + m, c:c + m].copy()


def extract_adjoint(patch: np.ndarray, pos, shape) -> np.ndarray:
    """P_k^T: an object-sized array that is `patch` on window k and 0 elsewhere."""
    out = np.zeros(shape, dtype=np.result_type(patch, np.complex128))
    r, c = int(pos[0]), int(pos[1])
    m = patch.shape[0]
    out[r:r + m, c:c + m] = patch
    return out


# ----------------------------------------------------------- forward model
def exit_wave(zk: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Q . z_k (Section 2.1)."""
    return Q * zk


def forward_intensities(z: np.ndarray, Q: np.ndarray, positions) -> np.ndarray:
    """Noise-free data d~_k = |F(Q . P_k z)|^2, k = 1..N (Section 2.1)."""
    m = Q.shape[0]
    return np.stack([np.abs(fft2(exit_wave(extract(z, p, m), Q))) ** 2 for p in positions])


def revised_exit_wave(zk, Q, dk, prev_phase=None):
    """R_k(z_k) = F^{-1}(sqrt(d_k) . exp(i theta(F(Q . z_k)))) (Definition REW).

    theta is the principal argument; where F(Q . z_k) is exactly 0 it is 0,
    or the entry of `prev_phase` when one is given (Eq. specification).
    """
    psi = fft2(exit_wave(zk, Q))
    theta = np.angle(psi)
    zero = psi == 0
    theta[zero] = 0.0 if prev_phase is None else prev_phase[zero]
    return ifft2(np.sqrt(dk) * np.exp(1j * theta))


# ------------------------------------------------- objective and gradient
def objective_k(zk, Q, dk) -> float:
    """Phi_k(z_k) = 1/2 || Q . z_k - R_k(z_k) ||^2 (Eq. exit_misfit)."""
    return 0.5 * float(np.sum(np.abs(exit_wave(zk, Q) - revised_exit_wave(zk, Q, dk)) ** 2))


def objective(z, Q, positions, d) -> float:
    """Phi(z) = sum_k Phi_k(P_k z) (Eq. exit_misfit)."""
    m = Q.shape[0]
    return float(sum(objective_k(extract(z, p, m), Q, dk) for p, dk in zip(positions, d)))


def objective_amplitude(z, Q, positions, d) -> float:
    """1/2 sum_k || |F(Q . P_k z)| - sqrt(d_k) ||^2 / m^2.

    The amplitude form of Section 2.1 scaled by 1/m^2, which the appendix
    ("Computation for the misfit derivative") shows equal to the exit-wave
    form for the unnormalised F.
    """
    m = Q.shape[0]
    tot = 0.0
    for p, dk in zip(positions, d):
        tot += float(np.sum((np.abs(fft2(exit_wave(extract(z, p, m), Q))) - np.sqrt(dk)) ** 2))
    return 0.5 * tot / (m * m)


def gradient_k(zk, Q, dk) -> np.ndarray:
    """grad Phi_k = conj(Q) . (Q . z_k - R_k(z_k)) (Eq. misfit_derivative)."""
    return np.conj(Q) * (exit_wave(zk, Q) - revised_exit_wave(zk, Q, dk))


def gradient(z, Q, positions, d) -> np.ndarray:
    """grad Phi(z) = sum_k P_k^T grad Phi_k(P_k z) (Section 2.1)."""
    m = Q.shape[0]
    g = np.zeros(z.shape, dtype=np.complex128)
    for p, dk in zip(positions, d):
        g += extract_adjoint(gradient_k(extract(z, p, m), Q, dk), p, z.shape)
    return g


def surrogate(z, zj, Q, positions, d) -> float:
    """Quadratic surrogate Phi~(z; z^(j)) of Eq. (quadratic_surrogate)."""
    m = Q.shape[0]
    tot = 0.0
    for p, dk in zip(positions, d):
        Rk = revised_exit_wave(extract(zj, p, m), Q, dk)
        tot += 0.5 * float(np.sum(np.abs(exit_wave(extract(z, p, m), Q) - Rk) ** 2))
    return tot


def stop_metric(z, Q, positions, d) -> float:
    """(1/(N m)) sum_k || grad Phi_k(z_k) ||_2, the stopping criterion of Section 5."""
    m = Q.shape[0]
    N = len(positions)
    tot = sum(np.linalg.norm(gradient_k(extract(z, p, m), Q, dk)) for p, dk in zip(positions, d))
    return float(tot) / (N * m)


def rpie_regulariser(Q, alpha: float) -> np.ndarray:
    """u^rPIE = alpha (||Q||_inf^2 J - |Q|^2) (Section 2.1, PIE family)."""
    a2 = np.abs(Q) ** 2
    return alpha * (a2.max() - a2)


# ---------------------------------------------------------------- weights
def coarse_weights(Q):
    """Q_H, W_z, W_R, W_u^H of Eq. (def_weights) for one coarsening.

    Q_H = I_h^H Q; W_z = |Q|^2 / (I_H^h I_h^H |Q|^2);
    W_R = (I_H^h Q_H) . W_z / Q; W_u^H = |Q_H|^2 / (I_h^H |Q|^2).
    """
    a2 = np.abs(Q) ** 2
    QH = restrict(Q)
    S = restrict(a2)
    Wz = safe_div(a2, prolong(S))
    WR = prolong(QH) * safe_div(Wz, Q)
    Wu = safe_div(np.abs(QH) ** 2, S)
    return QH, Wz, WR, Wu


# ------------------------------------------------------------------ MAGPS
def proximal_step(zk, Q, Rk, u):
    """z + conj(Q) / (u + |Q|^2) . (R - Q . z): one proximal point step on
    the surrogate of one window (Eq. rpie_formulation / the coarsest branch
    and the post-smoothing of Algorithm MAGPS)."""
    return zk + safe_div(np.conj(Q), u + np.abs(Q) ** 2) * (Rk - Q * zk)


def magps(zk, Q, Rk, u, levels: int):
    """Algorithm MAGPS on one window, `levels` grids including this one.

    levels == 1 is the coarsest branch (a single proximal step, i.e. rPIE).
    Otherwise: coarse-level preparation (Q_H and the three weights), weighted
    restriction of z and R, the coarse regulariser u_H = W_u^H . I_h^H u, the
    recursive coarse solve, the coarse-to-fine update z~ = z + I_H^h e_H, and
    one post-smoothing proximal step that uses the original fine R.
    """
    if levels == 1:
        return proximal_step(zk, Q, Rk, u)
    QH, Wz, WR, Wu = coarse_weights(Q)
    zH = restrict(Wz * zk)
    RH = restrict(WR * Rk)
    uH = Wu * restrict(u)
    zH_hat = magps(zH, QH, RH, uH, levels - 1)
    eH = zH_hat - zH
    z_tilde = zk + prolong(eH)
    return proximal_step(z_tilde, Q, Rk, u)


def magps_mgopt(zk, Q, Rk, u, levels: int, shift=None):
    """Algorithm MAGPS with the MG/OPT correction term of Algorithm MG/OPT
    (the variant the paper describes before proposing its consistent coarse
    surrogate): every coarse problem is the paper's coarse surrogate minus
    Re<v_H, z_H>, v_H = grad f_H(z_H) - I_h^H grad f_h(z_h), which makes the
    coarse gradient at z_H equal to the restricted fine gradient.  `shift` is
    the linear term this level inherited (the negative gradient of the level's
    objective at zk is conj(Q)(R - Q zk) + shift); each proximal step moves by
    that corrected residual gradient over u + |Q|^2."""
    if shift is None:
        shift = np.zeros_like(zk)

    def step(z):
        return z + safe_div(np.conj(Q) * (Rk - Q * z) + shift, u + np.abs(Q) ** 2)

    if levels == 1:
        return step(zk)
    QH, Wz, WR, Wu = coarse_weights(Q)
    zH = restrict(Wz * zk)
    RH = restrict(WR * Rk)
    uH = Wu * restrict(u)
    g_fine = np.conj(Q) * (Rk - Q * zk) + shift
    shift_H = restrict(g_fine) - np.conj(QH) * (RH - QH * zH)
    zH_hat = magps_mgopt(zH, QH, RH, uH, levels - 1, shift_H)
    return step(zk + prolong(zH_hat - zH))


def revised_exit_wave_recycled(zk, Q, dk, prev_theta):
    """R_k with the phase rule of Eq. (specification): where F(Q . z_k) is
    exactly 0 the phase of the window's previous visit is reused (0 on the
    first visit, prev_theta = None).  Returns R_k and the phases used."""
    psi = fft2(exit_wave(zk, Q))
    theta = np.angle(psi)
    zero = psi == 0
    theta[zero] = 0.0 if prev_theta is None else prev_theta[zero]
    return ifft2(np.sqrt(dk) * np.exp(1j * theta)), theta


def minibatch_step_variant(z, Q, positions, d, u, levels, batch, mgopt: bool = False, phases=None):
    """minibatch_step with the paper's variants switched on: the MG/OPT
    correction term (magps_mgopt) and/or the phase rule of Eq.
    (specification), `phases` a dict window -> phases of its last visit,
    updated in place (None: theta(0) = 0 at every visit)."""
    z = np.asarray(z, dtype=np.complex128)
    m = Q.shape[0]
    w = u + np.abs(Q) ** 2
    num = np.zeros(z.shape, dtype=np.complex128)
    den = np.zeros(z.shape, dtype=np.float64)
    for k in batch:
        r, c = positions[k]
        zk = z[r:r + m, c:c + m]
        if phases is None:
            Rk = revised_exit_wave(zk, Q, d[k])
        else:
            Rk, phases[k] = revised_exit_wave_recycled(zk, Q, d[k], phases.get(k))
        zh = magps_mgopt(zk, Q, Rk, u, levels) if mgopt else magps(zk, Q, Rk, u, levels)
        num[r:r + m, c:c + m] += w * (zh - zk)
        den[r:r + m, c:c + m] += w
    out = z.copy()
    lit = den > 0
    out[lit] += num[lit] / den[lit]
    return out


def rpie_update(zk, Q, dk, u):
    """One window of Algorithm rPIE: z_k + conj(Q)/(u+|Q|^2) . (R_k(z_k) - Q z_k)."""
    Rk = revised_exit_wave(zk, Q, dk)
    return zk + np.conj(Q) / (u + np.abs(Q) ** 2) * (Rk - Q * zk)


# ----------------------------------------------------------- MAGPIE loops
def magpie_sequential(z, Q, positions, d, u, levels, order):
    """One iteration of Algorithm MAGPIE: windows updated one at a time in
    the given permutation, each by MAGPS with its freshly revised exit wave."""
    z = np.array(z, dtype=np.complex128, copy=True)
    m = Q.shape[0]
    for k in order:
        r, c = positions[k]
        zk = z[r:r + m, c:c + m].copy()
        Rk = revised_exit_wave(zk, Q, d[k])
        z[r:r + m, c:c + m] = magps(zk, Q, Rk, u, levels)
    return z


def minibatch_step(z, Q, positions, d, u, levels, batch):
    """One minibatch: every window of `batch` starts from the same z, runs
    R_k and MAGPS, and the increments are combined with weights w = u + |Q|^2
    (module docstring)."""
    z = np.asarray(z, dtype=np.complex128)
    m = Q.shape[0]
    w = u + np.abs(Q) ** 2
    num = np.zeros(z.shape, dtype=np.complex128)
    den = np.zeros(z.shape, dtype=np.float64)
    for k in batch:
        r, c = positions[k]
        zk = z[r:r + m, c:c + m]
        Rk = revised_exit_wave(zk, Q, d[k])
        delta = magps(zk, Q, Rk, u, levels) - zk
        num[r:r + m, c:c + m] += w * delta
        den[r:r + m, c:c + m] += w
    out = z.copy()
    lit = den > 0
    out[lit] += num[lit] / den[lit]
    return out


def probe_step(z, Q, positions, d, beta, batch):
    """Probe update of one minibatch (module docstring, reading R2): every
    window from the same (z, Q); returns the new probe."""
    m = Q.shape[0]
    num = np.zeros(Q.shape, dtype=np.complex128)
    den = np.zeros(Q.shape, dtype=np.float64)
    for k in batch:
        zk = extract(z, positions[k], m)
        Rk = revised_exit_wave(zk, Q, d[k])
        a2 = np.abs(zk) ** 2
        num += np.conj(zk) * (Rk - Q * zk)
        den += beta * (a2.max() - a2) + a2
    out = np.array(Q, dtype=np.complex128, copy=True)
    lit = den > 0
    out[lit] += num[lit] / den[lit]
    return out


def minibatch_step_with_probe(z, Q, positions, d, alpha, levels, batch, beta):
    """Object and probe updated together from the same (z, Q): the object by
    minibatch_step with u = u^rPIE(Q), the probe by probe_step."""
    u = rpie_regulariser(Q, alpha)
    return (minibatch_step(z, Q, positions, d, u, levels, batch),
            probe_step(z, Q, positions, d, beta, batch))


def sweep_with_probe(z, Q, positions, d, alpha, levels, order, minibatch, beta):
    """One iteration over all windows updating object and probe per minibatch."""
    for s in range(0, len(order), minibatch):
        z, Q = minibatch_step_with_probe(z, Q, positions, d, alpha, levels, order[s:s + minibatch], beta)
    return z, Q


def sweep(z, Q, positions, d, u, levels, order, minibatch):
    """One iteration over all windows: consecutive minibatches of `order`."""
    for s in range(0, len(order), minibatch):
        z = minibatch_step(z, Q, positions, d, u, levels, order[s:s + minibatch])
    return z


# ----------------------------------------------------------------- metrics
def illuminated_mask(Q, positions, shape, rel: float = 1e-3) -> np.ndarray:
    """Pixels with sum_k P_k^T |Q|^2 >= rel * max (unlit pixels carry no data)."""
    m = Q.shape[0]
    cov = np.zeros(shape)
    for r, c in positions:
        cov[r:r + m, c:c + m] += np.abs(Q) ** 2
    return cov >= rel * cov.max()


def nrmse(a, b, mask=None) -> float:
    """min_phi || e^{i phi} a - b || / || b || over `mask` (global phase removed)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    if mask is not None:
        a, b = a[mask], b[mask]
    ip = np.vdot(a, b)
    ph = ip / abs(ip) if abs(ip) > 0 else 1.0
    return float(np.linalg.norm(ph * a - b) / np.linalg.norm(b))


def magnitude_error(z, z_true) -> float:
    """|| |z| - |z*| ||_2, the error metric of Section 5."""
    return float(np.linalg.norm(np.abs(z) - np.abs(z_true)))
