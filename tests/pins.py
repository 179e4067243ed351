"""Checks that tie the FP64 oracle to what the paper and the mathematics fix.

Each check takes the oracle module as its argument so that the mutation
tests can run the same checks against copies of the oracle with a planted
mistake and confirm that at least one check notices it.  A check raises
AssertionError when it fails.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _small_problem(O, seed=0, n=24, m=8, step=4, probe="gauss"):
    """A small fully covered problem with a probe that has no zeros."""
    rng = np.random.default_rng(seed)
    z_true = (0.8 + 0.2 * rng.random((n, n))) * np.exp(1j * (rng.random((n, n)) - 0.5))
    c = (m - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
    if probe == "gauss":
        Q = np.exp(-(xx ** 2 + yy ** 2) / (2 * (m / 3.0) ** 2)) * np.exp(0.3j * (xx ** 2 + yy ** 2) / m)
    else:
        Q = _crand(rng, m, m)
    Q = Q / np.abs(Q).max()
    starts = list(range(0, n - m + 1, step))
    pos = np.array([(r, cc) for r in starts for cc in starts], dtype=np.int64)
    d = O.forward_intensities(z_true, Q, pos)
    return z_true, Q, pos, d


# ------------------------------------------------------------------- DFT
def check_dft_defining_sum(O):
    """F equals the defining double sum with kernel e^{-2 pi i (pa+qb)/m}."""
    rng = np.random.default_rng(1)
    for m in (4, 8):
        x = _crand(rng, m, m)
        X = np.zeros((m, m), dtype=np.complex128)
        for p in range(m):
            for q in range(m):
                s = 0j
                for a in range(m):
                    for b in range(m):
                        s += x[a, b] * complex(math.cos(-2 * math.pi * (p * a + q * b) / m),
                                               math.sin(-2 * math.pi * (p * a + q * b) / m))
                X[p, q] = s
        assert _rel(O.fft2(x), X) < 1e-12


def check_dft_parseval_inverse(O):
    """||Fx||^2 = m^2 ||x||^2 and F^{-1} = F^*/m^2 (appendix)."""
    rng = np.random.default_rng(2)
    m = 16
    x = _crand(rng, m, m)
    X = O.fft2(x)
    assert abs(np.sum(np.abs(X) ** 2) - m * m * np.sum(np.abs(x) ** 2)) < 1e-9 * np.sum(np.abs(X) ** 2)
    # F^* X = conj(F(conj X)); the inverse must equal that divided by m^2
    assert _rel(O.ifft2(X), np.conj(O.fft2(np.conj(X))) / (m * m)) < 1e-13
    assert _rel(O.ifft2(X), x) < 1e-13


def check_dft_closed_forms(O):
    """Delta -> all ones; plane wave e^{+2 pi i (p0 a + q0 b)/m} -> m^2 delta at (p0, q0)."""
    m = 8
    x = np.zeros((m, m), dtype=np.complex128)
    x[0, 0] = 1
    assert _rel(O.fft2(x), np.ones((m, m))) < 1e-14
    a, b = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    p0, q0 = 3, 5
    wave = np.exp(2j * np.pi * (p0 * a + q0 * b) / m)
    expect = np.zeros((m, m), dtype=np.complex128)
    expect[p0, q0] = m * m
    assert _rel(O.fft2(wave), expect) < 1e-12


# --------------------------------------------------------- scan operators
def check_scan_adjoint(O):
    """<P_k x, y> = <x, P_k^T y> and the same for A = F diag(Q) P_k."""
    rng = np.random.default_rng(3)
    n, m = 20, 8
    pos = (5, 9)
    x = _crand(rng, n, n)
    y = _crand(rng, m, m)
    lhs = np.vdot(y, O.extract(x, pos, m))
    rhs = np.vdot(O.extract_adjoint(y, pos, (n, n)), x)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    Q = _crand(rng, m, m)
    Ax = O.fft2(Q * O.extract(x, pos, m))
    Aty = O.extract_adjoint(np.conj(Q) * (m * m) * O.ifft2(y), pos, (n, n))
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(Aty, x)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # the window is the one whose top-left corner is pos = (row, col)
    e = np.zeros((n, n))
    e[5, 9] = 1.0
    assert O.extract(e, pos, m)[0, 0] == 1.0


# ---------------------------------------------------- transfer operators
def _matrix_of(f, shape_in):
    cols = []
    for i in range(int(np.prod(shape_in))):
        e = np.zeros(int(np.prod(shape_in)))
        e[i] = 1.0
        cols.append(np.ravel(f(e.reshape(shape_in))))
    return np.array(cols).T


def check_transfer_operators(O):
    """Restriction is the 2x2 mean, prolongation 4 times its transpose;
    <I x, y> = 1/4 <x, P y>; I P = identity; ||I||_2 = 1/2, ||P||_2 = 2,
    both infinity norms 1; Lemma (commutative): B . I(A) = I(P(B) . A)."""
    rng = np.random.default_rng(4)
    x = _crand(rng, 8, 8)
    y = _crand(rng, 4, 4)
    assert abs(np.vdot(y, O.restrict(x)) - 0.25 * np.vdot(O.prolong(y), x)) < 1e-12
    assert _rel(O.restrict(O.prolong(y)), y) < 1e-15
    Rm = _matrix_of(O.restrict, (4, 4))
    Pm = _matrix_of(O.prolong, (2, 2))
    assert np.allclose(Pm, 4 * Rm.T)
    assert abs(np.linalg.norm(Rm, 2) - 0.5) < 1e-12
    assert abs(np.linalg.norm(Pm, 2) - 2.0) < 1e-12
    assert abs(np.abs(Rm).sum(axis=1).max() - 1.0) < 1e-12
    assert abs(np.abs(Pm).sum(axis=1).max() - 1.0) < 1e-12
    A = _crand(rng, 8, 8)
    B = _crand(rng, 4, 4)
    assert _rel(B * O.restrict(A), O.restrict(O.prolong(B) * A)) < 1e-14
    # the restriction of a constant bin is that constant (mean, not sum)
    assert np.allclose(O.restrict(np.full((2, 2), 3.0)), 3.0)


# ------------------------------------------------- objective and gradient
def check_objective_forms(O):
    """Exit-wave objective = amplitude objective / m^2 (appendix); both are
    0 at the true object on noise-free data."""
    z_true, Q, pos, d = _small_problem(O, seed=5)
    rng = np.random.default_rng(5)
    z = z_true + 0.3 * _crand(rng, *z_true.shape)
    a = O.objective(z, Q, pos, d)
    b = O.objective_amplitude(z, Q, pos, d)
    assert abs(a - b) < 1e-10 * a
    assert O.objective(z_true, Q, pos, d) < 1e-20 * a
    assert O.stop_metric(z_true, Q, pos, d) < 1e-10


def check_gradient_fd(O):
    """Central differences of Phi_k and Phi along random complex directions
    match Re <grad, h> with grad = conj(Q)(Q z_k - R_k) (Eq. misfit_derivative)."""
    z_true, Q, pos, d = _small_problem(O, seed=6)
    rng = np.random.default_rng(6)
    z = z_true + 0.3 * _crand(rng, *z_true.shape)
    m = Q.shape[0]
    zk = O.extract(z, pos[3], m)
    eps = 1e-6
    for _ in range(3):
        h = _crand(rng, m, m)
        fd = (O.objective_k(zk + eps * h, Q, d[3]) - O.objective_k(zk - eps * h, Q, d[3])) / (2 * eps)
        an = float(np.real(np.vdot(O.gradient_k(zk, Q, d[3]), h)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
    g = O.gradient(z, Q, pos, d)
    h = _crand(rng, *z.shape)
    fd = (O.objective(z + eps * h, Q, pos, d) - O.objective(z - eps * h, Q, pos, d)) / (2 * eps)
    an = float(np.real(np.vdot(g, h)))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def check_majorization(O):
    """Proposition (Majorization): Phi <= Phi~(.; z^(j)), equality and equal
    gradients at z^(j)."""
    z_true, Q, pos, d = _small_problem(O, seed=7)
    rng = np.random.default_rng(7)
    zj = z_true + 0.4 * _crand(rng, *z_true.shape)
    assert abs(O.surrogate(zj, zj, Q, pos, d) - O.objective(zj, Q, pos, d)) < 1e-12 * O.objective(zj, Q, pos, d)
    for s in (0.05, 0.3, 1.0):
        z = zj + s * _crand(rng, *zj.shape)
        assert O.objective(z, Q, pos, d) <= O.surrogate(z, zj, Q, pos, d) * (1 + 1e-12)
    g = O.gradient(zj, Q, pos, d)
    h = _crand(rng, *zj.shape)
    eps = 1e-6
    fd = (O.surrogate(zj + eps * h, zj, Q, pos, d) - O.surrogate(zj - eps * h, zj, Q, pos, d)) / (2 * eps)
    assert abs(fd - np.real(np.vdot(g, h))) < 1e-6 * max(1.0, abs(fd))
    # Eq. (quadratic_surrogate) is a quadratic in z for fixed z^(j): along a
    # line its second differences are constant and equal 2 * 1/2 sum ||Q . P_k h||^2
    # per unit step squared; Phi itself is not quadratic (R_k moves with z)
    vals = [O.surrogate(zj + t * h, zj, Q, pos, d) for t in (-1.0, 0.0, 1.0, 2.0)]
    curv = sum(float(np.sum(np.abs(Q * O.extract(h, p, Q.shape[0])) ** 2)) for p in pos)
    assert abs((vals[0] - 2 * vals[1] + vals[2]) - curv) < 1e-9 * curv
    assert abs((vals[1] - 2 * vals[2] + vals[3]) - curv) < 1e-9 * curv


def check_full_batch_monotone(O):
    """Proposition (Monotone descent): the full-batch one-level step is the
    exact minimiser of the proximal surrogate, so Phi never increases."""
    z_true, Q, pos, d = _small_problem(O, seed=8)
    rng = np.random.default_rng(8)
    z = z_true + 0.5 * _crand(rng, *z_true.shape)
    for alpha in (0.01, 0.3):
        u = O.rpie_regulariser(Q, alpha)
        zz = z.copy()
        prev = O.objective(zz, Q, pos, d)
        for it in range(8):
            zz = O.minibatch_step(zz, Q, pos, d, u, 1, np.arange(len(pos)))
            cur = O.objective(zz, Q, pos, d)
            assert cur <= prev * (1 + 1e-12)
            prev = cur


def check_minibatch_one_level_is_argmin(O):
    """For one level the minibatch step zeroes the gradient of
    sum_k [Phi~_k(P_k z; z^(j)) + 1/2 u^T |P_k z - P_k z^(j)|^2] (Eq.
    proximal_point_method summed over the minibatch), on covered pixels."""
    z_true, Q, pos, d = _small_problem(O, seed=9)
    rng = np.random.default_rng(9)
    zj = z_true + 0.5 * _crand(rng, *z_true.shape)
    u = O.rpie_regulariser(Q, 0.05)
    batch = np.array([0, 2, 4, 7])
    zp = O.minibatch_step(zj, Q, pos, d, u, 1, batch)
    m = Q.shape[0]
    grad = np.zeros(zj.shape, dtype=np.complex128)
    cover = np.zeros(zj.shape, dtype=bool)
    for k in batch:
        Rk = O.revised_exit_wave(O.extract(zj, pos[k], m), Q, d[k])
        zk = O.extract(zp, pos[k], m)
        gk = np.conj(Q) * (Q * zk - Rk) + u * (zk - O.extract(zj, pos[k], m))
        grad += O.extract_adjoint(gk, pos[k], zj.shape)
        r, c = pos[k]
        cover[r:r + m, c:c + m] = True
    assert np.abs(grad[cover]).max() < 1e-10 * np.abs(zj).max()
    # pixels outside the minibatch's windows do not move
    assert np.array_equal(zp[~cover], zj[~cover])


def check_sublinear_bound(O):
    """Proposition (Sublinear stationarity bound) for the exact full-batch
    surrogate minimiser (u = 0, every pixel covered, probe without zeros),
    L = 1/2 ||sum_k P_k^T |Q|^2||_inf.

    Its proof loses a factor 1/2 on the cross term Re <z - z^(j), grad Phi>
    between two consecutive lines; carried through, the step
    z = z^(j) - grad / (2L) gives Phi(z^(j)) - Phi(z^(j+1)) >= ||grad||^2/(4L),
    so the bound that holds is (1/(4L)) sum_j ||grad Phi(z^(j))||^2 <= Phi(z^(0)).
    The stated constant 1/L fails on this very problem (ratio about 3.2), and
    the check also asserts that, so that the reading stays visible."""
    z_true, Q, pos, d = _small_problem(O, seed=10)
    rng = np.random.default_rng(10)
    z = z_true + 0.5 * _crand(rng, *z_true.shape)
    u = np.zeros(Q.shape)
    cov = np.zeros(z.shape)
    m = Q.shape[0]
    for r, c in pos:
        cov[r:r + m, c:c + m] += np.abs(Q) ** 2
    assert cov.min() > 0
    Lc = 0.5 * cov.max()
    phi0 = O.objective(z, Q, pos, d)
    acc = 0.0
    for it in range(15):
        acc += float(np.sum(np.abs(O.gradient(z, Q, pos, d)) ** 2)) / (4 * Lc)
        assert acc <= phi0 * (1 + 1e-12)
        if it == 0:
            assert 4 * acc > phi0  # the constant as printed does not hold here
        z = O.minibatch_step(z, Q, pos, d, u, 1, np.arange(len(pos)))


# ---------------------------------------------------------------- weights
def check_weight_properties(O):
    """Proposition (Well-definedness): I_h^H W_z = J on lit bins, W_z <= 4,
    |W_R| <= 3/2 (the sharp bound quoted in its proof), W_u^H <= 1; the
    golden 2x2 bin (3,1,1,1) attains |W_R| = 3/2."""
    rng = np.random.default_rng(11)
    probes = [_crand(rng, 16, 16), np.abs(_crand(rng, 16, 16)) ** 3,
              _small_problem(O, seed=11)[1]]
    for Q in probes:
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        assert np.allclose(O.restrict(Wz), 1.0, atol=1e-12)
        assert Wz.max() <= 4 + 1e-12 and Wz.min() >= 0
        assert np.abs(WR).max() <= 1.5 + 1e-12
        assert Wu.max() <= 1 + 1e-12 and Wu.min() >= 0
        # consistency relation W_R . Q = (I_H^h Q_H) . W_z (Section 4.1)
        assert _rel(WR * Q, O.prolong(QH) * Wz) < 1e-12
    with open(os.path.join(GOLDEN, "weights_sharp_bound.json")) as f:
        g = json.load(f)
    QH, Wz, WR, Wu = O.coarse_weights(np.array(g["bin"], dtype=np.complex128))
    assert abs(np.abs(WR).max() - g["max_abs_WR"]) < 1e-14
    assert tuple(np.unravel_index(np.abs(WR).argmax(), WR.shape)) == tuple(g["argmax"])


def check_coarse_step_closed_form(O):
    """Theorem (Descent property): for two levels the coarse increment is
    e_H = -|Q_H|^2 / (I|Q|^2) / (u_H + |Q_H|^2) . I(grad Phi~_k(z')) (Eq.
    coarse_grid_rPIE_update), the MAGPS output is the post-smoothing step
    from z' + I_H^h e_H, and Re <grad, I_H^h e_H> <= 0."""
    rng = np.random.default_rng(12)
    m = 16
    for trial in range(3):
        Q = _crand(rng, m, m) if trial else _small_problem(O, seed=12, m=m)[1]
        zk = _crand(rng, m, m)
        Rk = _crand(rng, m, m)
        u = O.rpie_regulariser(Q, 0.1)
        grad = np.conj(Q) * (Q * zk - Rk)
        QH = O.restrict(Q)
        S = O.restrict(np.abs(Q) ** 2)
        uH = np.abs(QH) ** 2 / S * O.restrict(u)
        eH = -(np.abs(QH) ** 2 / S) / (uH + np.abs(QH) ** 2) * O.restrict(grad)
        zt = zk + O.prolong(eH)
        expect = zt + np.conj(Q) / (u + np.abs(Q) ** 2) * (Rk - Q * zt)
        assert _rel(O.magps(zk, Q, Rk, u, 2), expect) < 1e-12
        assert np.real(np.vdot(grad, O.prolong(eH))) <= 0
        # the same increment in lowest terms: -I(grad) / I(u + |Q|^2)
        assert _rel(eH, -O.restrict(grad) / O.restrict(u + np.abs(Q) ** 2)) < 1e-12


def check_coarse_prox_is_argmin(O):
    """The coarsest MAGPS branch zeroes the gradient of the coarse surrogate
    plus its proximal term (Eq. coarse_proximal)."""
    rng = np.random.default_rng(13)
    m = 8
    Q = _crand(rng, m, m)
    zH = _crand(rng, m, m)
    RH = _crand(rng, m, m)
    uH = rng.random((m, m))
    zh = O.magps(zH, Q, RH, uH, 1)
    g = np.conj(Q) * (Q * zh - RH) + uH * (zh - zH)
    assert np.abs(g).max() < 1e-12


def check_auto_regularisation(O):
    """Proposition (Automatic regularization selection): with
    u_H = W_u^H . I u, (1/(u_H + |Q_H|^2)) . |Q_H|^2 / I|Q|^2 equals
    1 / I(u + |Q|^2); it equals I(1/(u + |Q|^2)) when u + |Q|^2 is constant
    on each bin and is never larger (Jensen)."""
    rng = np.random.default_rng(14)
    Q = _crand(rng, 16, 16)
    u = O.rpie_regulariser(Q, 0.2)
    QH, Wz, WR, Wu = O.coarse_weights(Q)
    uH = Wu * O.restrict(u)
    lhs = (1.0 / (uH + np.abs(QH) ** 2)) * np.abs(QH) ** 2 / O.restrict(np.abs(Q) ** 2)
    assert _rel(lhs, 1.0 / O.restrict(u + np.abs(Q) ** 2)) < 1e-12
    assert np.all(O.restrict(1.0 / (u + np.abs(Q) ** 2)) >= lhs * (1 - 1e-12))
    # bins on which u + |Q|^2 is constant: u = alpha (max - |Q|^2) with alpha = 1
    u1 = O.rpie_regulariser(Q, 1.0)
    uH1 = Wu * O.restrict(u1)
    lhs1 = (1.0 / (uH1 + np.abs(QH) ** 2)) * np.abs(QH) ** 2 / O.restrict(np.abs(Q) ** 2)
    assert _rel(lhs1, O.restrict(1.0 / (u1 + np.abs(Q) ** 2))) < 1e-12


def check_consistency_bounds(O):
    """Proposition (Consistency) on random windows."""
    rng = np.random.default_rng(15)
    m = 16
    for _ in range(4):
        Q = _crand(rng, m, m)
        zk = _crand(rng, m, m)
        Rk = _crand(rng, m, m)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(WR * Rk)
        phi = 0.5 * np.sum(np.abs(Q * zk - Rk) ** 2)
        phiH = 0.5 * np.sum(np.abs(QH * zH - RH) ** 2)
        assert phiH <= 0.25 * np.abs(WR).max() ** 2 * phi * (1 + 1e-12)
        g = np.linalg.norm(np.conj(Q) * (Q * zk - Rk))
        gH = np.linalg.norm(np.conj(QH) * (QH * zH - RH))
        assert gH <= 0.5 * Wu.max() * g * (1 + 1e-12)


def check_residual_form(O):
    """MAGPS depends on (z, R) only through g = conj(Q)(R - Qz), through a
    recursion with real per-level factors: g^{l+1} = W_u^l . I(g^l),
    w^{l+1} = W_u^l . I(w^l) (w = u + |Q|^2), e^{L-1} = g / w on the
    coarsest grid and e^l = (g^l + u^l . I_H^h e^{l+1}) / w^l above it.
    Follows from W_R . Q = (I_H^h Q_H) . W_z and Lemma (commutative)."""
    rng = np.random.default_rng(16)
    m = 16
    for L in (1, 2, 3, 4, 5):
        Q = _crand(rng, m, m)
        zk = _crand(rng, m, m)
        Rk = _crand(rng, m, m)
        u = O.rpie_regulariser(Q, 0.05)
        gs, us, ws = [np.conj(Q) * (Rk - Q * zk)], [u], [u + np.abs(Q) ** 2]
        Ql = Q
        for lvl in range(L - 1):
            QH, Wz, WR, Wu = O.coarse_weights(Ql)
            gs.append(Wu * O.restrict(gs[-1]))
            us.append(Wu * O.restrict(us[-1]))
            ws.append(Wu * O.restrict(ws[-1]))
            Ql = QH
        e = gs[-1] / ws[-1]
        for lvl in range(L - 2, -1, -1):
            e = (gs[lvl] + us[lvl] * O.prolong(e)) / ws[lvl]
        assert _rel(O.magps(zk, Q, Rk, u, L) - zk, e) < 1e-11


def check_special_cases(O):
    """levels = 1 is rPIE (Algorithm rPIE); a minibatch of one is Algorithm
    MAGPIE's sequential update."""
    z_true, Q, pos, d = _small_problem(O, seed=17)
    rng = np.random.default_rng(17)
    z = z_true + 0.3 * _crand(rng, *z_true.shape)
    u = O.rpie_regulariser(Q, 0.1)
    m = Q.shape[0]
    zk = O.extract(z, pos[1], m)
    Rk = O.revised_exit_wave(zk, Q, d[1])
    assert _rel(O.magps(zk, Q, Rk, u, 1), O.rpie_update(zk, Q, d[1], u)) < 1e-14
    order = rng.permutation(len(pos))
    for L in (1, 2, 3):
        a = O.magpie_sequential(z, Q, pos, d, u, L, order)
        b = O.sweep(z, Q, pos, d, u, L, order, 1)
        assert _rel(b, a) < 1e-13


def check_recovery(O):
    """Noise-free data, known probe: the minibatch iteration drives the
    object to the truth up to a global phase (stationarity, Proposition
    Monotone descent) on the illuminated pixels."""
    z_true, Q, pos, d = _small_problem(O, seed=18, n=24, m=8, step=2)
    u = O.rpie_regulariser(Q, 0.2)
    z = np.ones_like(z_true)
    mask = O.illuminated_mask(Q, pos, z.shape, 0.05)
    rng = np.random.default_rng(18)
    first = O.nrmse(z, z_true, mask)
    for it in range(400):
        z = O.magpie_sequential(z, Q, pos, d, u, 2, rng.permutation(len(pos)))
    last = O.nrmse(z, z_true, mask)
    assert last < 1e-6 < first, (first, last)


def check_probe_step(O):
    """Probe step (reading R2): it zeroes the gradient in Q of
    sum_k [1/2 ||Q . z_k - R_k||^2 + 1/2 u_Q,k^T |Q - Q^(j)|^2] with R_k and
    z_k from the current iterate, and a full-batch probe step never increases
    Phi (majorization, with the roles of Q and z_k exchanged)."""
    z_true, Q_true, pos, d = _small_problem(O, seed=19)
    rng = np.random.default_rng(19)
    z = z_true + 0.1 * _crand(rng, *z_true.shape)
    Qj = Q_true * (1 + 0.2 * _crand(rng, *Q_true.shape))
    m = Qj.shape[0]
    beta = 0.3
    batch = np.array([0, 3, 5, 6])
    Qp = O.probe_step(z, Qj, pos, d, beta, batch)
    grad = np.zeros(Qj.shape, dtype=np.complex128)
    for k in batch:
        zk = O.extract(z, pos[k], m)
        Rk = O.revised_exit_wave(zk, Qj, d[k])
        a2 = np.abs(zk) ** 2
        uq = beta * (a2.max() - a2)
        grad += np.conj(zk) * (Qp * zk - Rk) + uq * (Qp - Qj)
    assert np.abs(grad).max() < 1e-10 * np.abs(Qj).max()
    allk = np.arange(len(pos))
    prev = O.objective(z, Qj, pos, d)
    Qc = Qj
    for it in range(5):
        Qc = O.probe_step(z, Qc, pos, d, beta, allk)
        cur = O.objective(z, Qc, pos, d)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def check_mgopt_variant(O):
    """The MG/OPT correction term (Algorithm MG/OPT): (a) it vanishes where
    the probe is constant on every bin of every level (W_u = 1, the coarse
    surrogate is then first-order consistent by itself); (b) for two levels
    the result is the minimiser of the coarse surrogate minus Re<v_H, z_H>,
    v_H = grad f_H(z_H) - I_h^H grad f_h(z), followed by the fine proximal
    step, both solved here from their stationarity conditions with the
    gradients grad f(x) = conj(Q)(Q x - R) of Eq. (misfit_derivative);
    (c) the residual form with the plain restriction g^{l+1} = I_h^H g^l (the
    weights W_u replaced by 1, u^l and w^l unchanged) gives the same step."""
    rng = np.random.default_rng(31)
    m = 16
    q4 = _crand(rng, m // 4, m // 4)
    Qc = O.prolong(O.prolong(q4))  # constant on 4 x 4 blocks
    zk, Rk = _crand(rng, m, m), _crand(rng, m, m)
    u = O.rpie_regulariser(Qc, 0.1)
    for L in (2, 3):
        assert _rel(O.magps_mgopt(zk, Qc, Rk, u, L), O.magps(zk, Qc, Rk, u, L)) < 1e-12
    Q = _crand(rng, m, m)
    u = O.rpie_regulariser(Q, 0.1)
    QH, Wz, WR, Wu = O.coarse_weights(Q)
    zH, RH, uH = O.restrict(Wz * zk), O.restrict(WR * Rk), Wu * O.restrict(u)
    grad_h = np.conj(Q) * (Q * zk - Rk)
    grad_H = np.conj(QH) * (QH * zH - RH)
    vH = grad_H - O.restrict(grad_h)
    # stationarity of 1/2|QH y - RH|^2 - Re<vH, y> + 1/2 uH |y - zH|^2
    yH = (np.conj(QH) * RH + vH + uH * zH) / (np.abs(QH) ** 2 + uH)
    zt = zk + O.prolong(yH - zH)
    # stationarity of 1/2|Q x - R|^2 + 1/2 u |x - zt|^2
    x = (np.conj(Q) * Rk + u * zt) / (np.abs(Q) ** 2 + u)
    assert _rel(O.magps_mgopt(zk, Q, Rk, u, 2), x) < 1e-12
    assert _rel(O.magps_mgopt(zk, Q, Rk, u, 2), O.magps(zk, Q, Rk, u, 2)) > 1e-6
    for L in (2, 3, 4):
        gs, us, ws = [np.conj(Q) * (Rk - Q * zk)], [u], [u + np.abs(Q) ** 2]
        Ql = Q
        for lvl in range(L - 1):
            _, _, _, Wl = O.coarse_weights(Ql)
            gs.append(O.restrict(gs[-1]))
            us.append(Wl * O.restrict(us[-1]))
            ws.append(Wl * O.restrict(ws[-1]))
            Ql = O.restrict(Ql)
        e = gs[-1] / ws[-1]
        for lvl in range(L - 2, -1, -1):
            e = (gs[lvl] + us[lvl] * O.prolong(e)) / ws[lvl]
        assert _rel(O.magps_mgopt(zk, Q, Rk, u, L) - zk, e) < 1e-11


def check_phase_rule_variant(O):
    """Eq. (specification) across visits: with no exact zero in the spectrum
    the rule changes nothing; a window whose object patch is exactly zero has
    a zero spectrum, so its first visit uses theta = 0 and every later visit
    the phases of the visit before (here: of a visit with a nonzero patch)."""
    z_true, Q, pos, d = _small_problem(O, seed=32)
    u = O.rpie_regulariser(Q, 0.1)
    rng = np.random.default_rng(32)
    z = z_true + 0.2 * _crand(rng, *z_true.shape)
    batch = list(range(len(pos)))
    ph = {}
    a = O.minibatch_step_variant(z, Q, pos, d, u, 2, batch, phases=ph)
    assert _rel(a, O.minibatch_step(z, Q, pos, d, u, 2, batch)) < 1e-14
    m = Q.shape[0]
    k = 3
    zk = O.extract(z, pos[k], m)
    R1, th1 = O.revised_exit_wave_recycled(zk, Q, d[k], None)
    zero = np.zeros_like(zk)
    R2, th2 = O.revised_exit_wave_recycled(zero, Q, d[k], th1)
    assert np.array_equal(th2, th1)
    assert _rel(R2, O.ifft2(np.sqrt(d[k]) * np.exp(1j * np.angle(O.fft2(Q * zk))))) < 1e-12
    R0, th0 = O.revised_exit_wave_recycled(zero, Q, d[k], None)
    assert np.all(th0 == 0) and _rel(R0, O.ifft2(np.sqrt(d[k]))) < 1e-14


# ----------------------------------------------------------- metrics
def check_stop_metric_closed_form(O):
    """Stopping criterion of Section 5, (1/(N m)) sum_k ||grad Phi_k(z_k)||_2,
    on data whose revised exit wave is known in closed form: with
    d_k = s_k^2 |F(Q . z_k)|^2 (s_k > 0) the projection keeps every phase and
    scales every modulus by s_k, so R_k = s_k Q . z_k and
    grad Phi_k = (1 - s_k) |Q|^2 . z_k; no transform is needed to state the
    expected value.  (a) One window, constant probe c and constant patch a:
    the metric is |1 - s| |c|^2 |a| (the m of the norm cancels the 1/m);
    (b) three windows with different s_k fix the 1/N average."""
    m = 8
    c, a, s = 0.6 - 0.3j, 1.3 + 0.4j, 1.75
    Q = np.full((m, m), c)
    z = np.full((m, m), a)
    d = (s * np.abs(O.fft2(Q * z))) ** 2
    pos = np.array([(0, 0)])
    val = O.stop_metric(z, Q, pos, d[None])
    assert abs(val - abs(1 - s) * abs(c) ** 2 * abs(a)) < 1e-12 * abs(c) ** 2 * abs(a), val
    rng = np.random.default_rng(33)
    n = 20
    z = _crand(rng, n, n)
    yy, xx = np.meshgrid(np.arange(m) - 3.5, np.arange(m) - 3.5, indexing="ij")
    Q = np.exp(-(xx ** 2 + yy ** 2) / 18.0) * np.exp(0.2j * xx)
    pos = np.array([(0, 0), (5, 9), (12, 3)])
    sk = np.array([0.5, 1.25, 3.0])
    d = np.stack([(sk[i] * np.abs(O.fft2(Q * O.extract(z, p, m)))) ** 2 for i, p in enumerate(pos)])
    expect = sum(abs(1 - sk[i]) * np.linalg.norm(np.abs(Q) ** 2 * z[r:r + m, cc:cc + m])
                 for i, (r, cc) in enumerate(pos)) / (len(pos) * m)
    val = O.stop_metric(z, Q, pos, d)
    assert abs(val - expect) < 1e-10 * expect, (val, expect)


def check_nrmse_definition(O):
    """NRMSE(a, b) = min_phi ||e^{i phi} a - b||_M / ||b||_M with b the
    reference: a = 2b gives 1 and b against 2b gives 1/2 (the reference's
    norm divides); a global phase alone gives 0; a real perturbation delta of
    a positive real b on the mask gives ||delta||_M / ||b||_M whatever lies
    off the mask; and the closed-form phase matches a brute-force search."""
    rng = np.random.default_rng(34)
    b = _crand(rng, 6, 7)
    assert abs(O.nrmse(2 * b, b) - 1.0) < 1e-14
    assert abs(O.nrmse(b, 2 * b) - 0.5) < 1e-14
    assert O.nrmse(np.exp(0.7j) * b, b) < 1e-14
    br = 0.5 + rng.random((10, 10))
    mask = rng.random((10, 10)) < 0.5
    delta = 0.01 * rng.standard_normal((10, 10)) * mask
    a = np.exp(-1.1j) * (br + delta)
    a[~mask] = 1e3 * _crand(rng, int((~mask).sum()))
    expect = np.linalg.norm(delta[mask]) / np.linalg.norm(br[mask])
    assert abs(O.nrmse(a, br, mask) - expect) < 1e-12 * expect
    a, b = _crand(rng, 5, 5), _crand(rng, 5, 5)
    phis = np.linspace(0.0, 2 * np.pi, 200001)
    brute = min(np.linalg.norm(np.exp(1j * p) * a - b) for p in phis[::100])
    p0 = phis[::100][int(np.argmin([np.linalg.norm(np.exp(1j * p) * a - b) for p in phis[::100]]))]
    fine = np.linspace(p0 - 0.01, p0 + 0.01, 20001)
    brute = min(brute, min(np.linalg.norm(np.exp(1j * p) * a - b) for p in fine)) / np.linalg.norm(b)
    assert abs(O.nrmse(a, b) - brute) < 1e-9, (O.nrmse(a, b), brute)


def check_regulariser_definition(O):
    """The rPIE regulariser u = alpha (max|Q|^2 - |Q|^2): nonnegative, zero
    exactly where |Q| is largest, linear in alpha and of degree two in Q for
    a probe of any scale (the workloads normalise max|Q| to 1, which would
    hide a missing maximum)."""
    rng = np.random.default_rng(21)
    Q = 3.0 * _crand(rng, 8, 8)
    a2 = np.abs(Q) ** 2
    u = O.rpie_regulariser(Q, 0.2)
    assert np.all(u >= -1e-12 * a2.max())
    assert abs(u.flat[int(np.argmax(a2))]) <= 1e-12 * a2.max()
    assert _rel(O.rpie_regulariser(2.0 * Q, 0.2), 4.0 * u) < 1e-12
    assert _rel(O.rpie_regulariser(Q, 0.6), 3.0 * u) < 1e-12


def _idft2_brute(x):
    """Inverse DFT by its defining double sum, (1/m^2) sum X exp(+2 pi i ...)."""
    m = x.shape[0]
    k = np.arange(m)
    w = np.exp(2j * np.pi * np.outer(k, k) / m)
    return w @ x @ w / (m * m)


def check_zero_spectrum_phase(O):
    """Definition REW with theta(0) = 0: for a window whose exit wave is zero
    every spectrum entry is exactly 0, so the revised exit wave is the inverse
    DFT of sqrt(d_k) itself (brute-force inverse DFT here)."""
    rng = np.random.default_rng(22)
    m = 8
    Q = _crand(rng, m, m)
    d = 4.0 * rng.random((m, m))
    R = O.revised_exit_wave(np.zeros((m, m), dtype=np.complex128), Q, d)
    assert _rel(R, _idft2_brute(np.sqrt(d))) < 1e-12


def check_disjoint_windows_decouple(O):
    """Windows that do not overlap do not interact in a minibatch (the weights
    cancel pixel by pixel), so a sweep over disjoint windows gives each window
    exactly its own MAGPS step, for any minibatch size: the sweep's last,
    short minibatch is applied like the others."""
    rng = np.random.default_rng(23)
    m, nw = 8, 5
    z_true = (0.8 + 0.2 * rng.random((m, nw * m))) * np.exp(1j * (rng.random((m, nw * m)) - 0.5))
    c = (m - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
    Q = np.exp(-(xx ** 2 + yy ** 2) / (2 * (m / 3.0) ** 2)) * np.exp(0.3j * (xx ** 2 + yy ** 2) / m)
    pos = np.array([(0, k * m) for k in range(nw)], dtype=np.int64)
    d = O.forward_intensities(z_true, Q, pos)
    z = np.ones(z_true.shape, dtype=np.complex128)
    u = O.rpie_regulariser(Q, 0.1)
    for B in (1, 2, 3, 5):
        out = O.sweep(z, Q, pos, d, u, 2, rng.permutation(nw), B)
        for k in range(nw):
            zk = z[:, k * m:(k + 1) * m]
            ref = O.magps(zk, Q, O.revised_exit_wave(zk, Q, d[k]), u, 2)
            assert _rel(out[:, k * m:(k + 1) * m], ref) < 1e-12, (B, k)


def check_dead_bins_stay_finite(O):
    """A probe with a dead 2 x 2 bin (so dead bins on every coarser level
    above it): every level weight and every MAGPS output stays finite.  What
    a dead bin's weight is, is a reading (the division rule); that it is
    finite is what any rule must give."""
    z_true, Q, pos, d = _small_problem(O, seed=24)
    Q = Q.copy()
    Q[2:4, 2:4] = 0.0
    d = O.forward_intensities(z_true, Q, pos)
    u = O.rpie_regulariser(Q, 0.1)
    Ql = Q
    for _ in range(3):
        QH, Wz, WR, Wu = O.coarse_weights(Ql)
        for a in (QH, Wz, WR, Wu):
            assert np.all(np.isfinite(a))
        Ql = QH
    rng = np.random.default_rng(24)
    z = z_true + 0.2 * _crand(rng, *z_true.shape)
    m = Q.shape[0]
    for k in (0, 3):
        zk = O.extract(z, pos[k], m)
        Rk = O.revised_exit_wave(zk, Q, d[k])
        for L in (2, 3, 4):
            assert np.all(np.isfinite(O.magps(zk, Q, Rk, u, L))), L
    assert np.all(np.isfinite(O.minibatch_step(z, Q, pos, d, u, 4, list(range(len(pos))))))


def check_metric_helpers(O):
    """The illuminated mask is the set of pixels whose summed probe intensity
    sum_k P_k^T |Q|^2 reaches `rel` of its maximum, computed here pixel by
    pixel from the windows that cover each pixel; the magnitude error of
    Section 5, || |z| - |z*| ||, ignores every pixel's phase and is ||z*|| for
    z = 2 z*."""
    rng = np.random.default_rng(25)
    m, n = 6, 20
    Q = _crand(rng, m, m)
    pos = [(0, 0), (3, 5), (10, 2), (14, 14), (2, 11)]
    for rel in (1e-3, 0.3, 0.7):
        cov = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                for r, c in pos:
                    if r <= i < r + m and c <= j < c + m:
                        cov[i, j] += abs(Q[i - r, j - c]) ** 2
        assert np.array_equal(O.illuminated_mask(Q, pos, (n, n), rel), cov >= rel * cov.max())
    zt = _crand(rng, n, n)
    assert O.magnitude_error(zt * np.exp(1j * rng.random((n, n)) * 6.0), zt) < 1e-12 * np.linalg.norm(zt)
    assert abs(O.magnitude_error(2 * zt, zt) - np.linalg.norm(zt)) < 1e-12 * np.linalg.norm(zt)


ALL_CHECKS = [
    check_dft_defining_sum, check_dft_parseval_inverse, check_dft_closed_forms,
    check_scan_adjoint, check_transfer_operators, check_objective_forms,
    check_gradient_fd, check_majorization, check_full_batch_monotone,
    check_minibatch_one_level_is_argmin, check_sublinear_bound,
    check_weight_properties, check_coarse_step_closed_form,
    check_coarse_prox_is_argmin, check_auto_regularisation,
    check_consistency_bounds, check_residual_form, check_special_cases,
    check_probe_step, check_recovery, check_mgopt_variant, check_phase_rule_variant,
    check_stop_metric_closed_form, check_nrmse_definition, check_regulariser_definition,
    check_zero_spectrum_phase, check_disjoint_windows_decouple, check_dead_bins_stay_finite,
    check_metric_helpers,
]
