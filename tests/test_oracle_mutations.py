"""Plant plausible mistakes in copies of the oracle and confirm that the pin
checks notice each one (CPU only; the real oracle is never modified)."""
import importlib.util
import os

import numpy as np
import pytest

from tests import pins

ORACLE_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "oracle", "magpie_oracle.py")


def fresh_oracle():
    spec = importlib.util.spec_from_file_location("oracle_copy", ORACLE_FILE)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def m_restrict_sum(O):
    O.restrict = lambda a: a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2]


def m_prolong_scaled(O):
    orig = O.prolong
    O.prolong = lambda b: 0.25 * orig(b)


def m_fft_sign(O):
    O.fft2 = lambda x: np.fft.ifft2(x) * x.shape[0] * x.shape[1]
    O.ifft2 = lambda x: np.fft.fft2(x) / (x.shape[0] * x.shape[1])


def m_fft_unnormalised_inverse(O):
    O.ifft2 = lambda x: np.fft.ifft2(x) * x.shape[0] * x.shape[1]


def m_no_sqrt(O):
    def rew(zk, Q, dk, prev_phase=None):
        psi = O.fft2(Q * zk)
        return O.ifft2(dk * np.exp(1j * np.angle(psi)))
    O.revised_exit_wave = rew


def m_gradient_no_conj(O):
    O.gradient_k = lambda zk, Q, dk: Q * (Q * zk - O.revised_exit_wave(zk, Q, dk))


def m_wr_no_conj(O):
    def cw(Q):
        a2 = np.abs(Q) ** 2
        QH = O.restrict(Q)
        S = O.restrict(a2)
        Wz = O.safe_div(a2, O.prolong(S))
        WR = O.prolong(QH) * O.safe_div(Wz, np.conj(Q))
        Wu = O.safe_div(np.abs(QH) ** 2, S)
        return QH, Wz, WR, Wu
    O.coarse_weights = cw


def m_wz_unnormalised(O):
    orig = O.coarse_weights

    def cw(Q):
        QH, Wz, WR, Wu = orig(Q)
        return QH, np.abs(Q) ** 2, WR, Wu
    O.coarse_weights = cw


def m_uh_unweighted(O):
    def magps(zk, Q, Rk, u, levels):
        if levels == 1:
            return O.proximal_step(zk, Q, Rk, u)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(WR * Rk)
        eH = magps(zH, QH, RH, O.restrict(u), levels - 1) - zH
        return O.proximal_step(zk + O.prolong(eH), Q, Rk, u)
    O.magps = magps


def m_post_smooth_from_z(O):
    def magps(zk, Q, Rk, u, levels):
        if levels == 1:
            return O.proximal_step(zk, Q, Rk, u)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(WR * Rk)
        eH = magps(zH, QH, RH, Wu * O.restrict(u), levels - 1) - zH
        return O.proximal_step(zk, Q, Rk, u) + O.prolong(eH)
    O.magps = magps


def m_minibatch_count_average(O):
    def step(z, Q, positions, d, u, levels, batch):
        m = Q.shape[0]
        num = np.zeros(z.shape, dtype=np.complex128)
        den = np.zeros(z.shape)
        for k in batch:
            r, c = positions[k]
            zk = z[r:r + m, c:c + m]
            Rk = O.revised_exit_wave(zk, Q, d[k])
            num[r:r + m, c:c + m] += O.magps(zk, Q, Rk, u, levels) - zk
            den[r:r + m, c:c + m] += 1.0
        out = np.array(z, dtype=np.complex128)
        lit = den > 0
        out[lit] += num[lit] / den[lit]
        return out
    O.minibatch_step = step


def m_regulariser_amplitude(O):
    O.rpie_regulariser = lambda Q, alpha: alpha * (np.abs(Q).max() - np.abs(Q))


def m_extract_transposed(O):
    O.extract = lambda z, pos, m: z[int(pos[1]):int(pos[1]) + m, int(pos[0]):int(pos[0]) + m].copy()


def m_objective_no_half(O):
    orig = O.objective_k
    O.objective_k = lambda zk, Q, dk: 2.0 * orig(zk, Q, dk)


def m_mgopt_shift_sign(O):
    orig = O.magps_mgopt

    def mg(zk, Q, Rk, u, levels, shift=None):
        return orig(zk, Q, Rk, u, levels, None if shift is None else -shift)
    O.magps_mgopt = mg


def m_mgopt_weighted_restriction(O):
    def mg(zk, Q, Rk, u, levels, shift=None):
        if shift is None:
            shift = np.zeros_like(zk)

        def step(z):
            return z + O.safe_div(np.conj(Q) * (Rk - Q * z) + shift, u + np.abs(Q) ** 2)
        if levels == 1:
            return step(zk)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH, RH, uH = O.restrict(Wz * zk), O.restrict(WR * Rk), Wu * O.restrict(u)
        g = np.conj(Q) * (Rk - Q * zk) + shift
        sH = Wu * O.restrict(g) - np.conj(QH) * (RH - QH * zH)
        return step(zk + O.prolong(mg(zH, QH, RH, uH, levels - 1, sH) - zH))
    O.magps_mgopt = mg


def m_phase_rule_forgets(O):
    def rec(zk, Q, dk, prev_theta):
        psi = O.fft2(O.exit_wave(zk, Q))
        theta = np.angle(psi)
        return O.ifft2(np.sqrt(dk) * np.exp(1j * theta)), theta
    O.revised_exit_wave_recycled = rec


def m_stop_metric_extra_inv_m(O):
    orig = O.stop_metric
    O.stop_metric = lambda z, Q, positions, d: orig(z, Q, positions, d) / Q.shape[0]


def m_stop_metric_squared_norms(O):
    def stop(z, Q, positions, d):
        m = Q.shape[0]
        tot = sum(np.linalg.norm(O.gradient_k(O.extract(z, p, m), Q, dk)) ** 2 for p, dk in zip(positions, d))
        return float(tot) / (len(positions) * m)
    O.stop_metric = stop


def m_stop_metric_sum_not_mean(O):
    orig = O.stop_metric
    O.stop_metric = lambda z, Q, positions, d: orig(z, Q, positions, d) * len(positions)


def m_nrmse_swapped(O):
    orig = O.nrmse
    O.nrmse = lambda a, b, mask=None: orig(b, a, mask)


def m_nrmse_no_phase(O):
    def nr(a, b, mask=None):
        a = np.asarray(a, dtype=np.complex128)
        b = np.asarray(b, dtype=np.complex128)
        if mask is not None:
            a, b = a[mask], b[mask]
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    O.nrmse = nr


def m_nrmse_conjugate_phase(O):
    def nr(a, b, mask=None):
        a = np.asarray(a, dtype=np.complex128)
        b = np.asarray(b, dtype=np.complex128)
        if mask is not None:
            a, b = a[mask], b[mask]
        ip = np.vdot(a, b)
        ph = np.conj(ip) / abs(ip) if abs(ip) > 0 else 1.0
        return float(np.linalg.norm(ph * a - b) / np.linalg.norm(b))
    O.nrmse = nr


def m_probe_step_sign(O):
    orig = O.probe_step

    def ps(z, Q, positions, d, beta, batch):
        return 2 * np.asarray(Q, dtype=np.complex128) - orig(z, Q, positions, d, beta, batch)
    O.probe_step = ps


def m_probe_regulariser_of_probe(O):
    def ps(z, Q, positions, d, beta, batch):
        m = Q.shape[0]
        num = np.zeros(Q.shape, dtype=np.complex128)
        den = np.zeros(Q.shape, dtype=np.float64)
        q2 = np.abs(Q) ** 2
        for k in batch:
            zk = O.extract(z, positions[k], m)
            Rk = O.revised_exit_wave(zk, Q, d[k])
            a2 = np.abs(zk) ** 2
            num += np.conj(zk) * (Rk - Q * zk)
            den += beta * (q2.max() - q2) + a2  # the probe's own intensity in place of the window's
        out = np.array(Q, dtype=np.complex128, copy=True)
        lit = den > 0
        out[lit] += num[lit] / den[lit]
        return out
    O.probe_step = ps


def m_theta_zero_is_pi(O):
    def rew(zk, Q, dk, prev_phase=None):
        psi = O.fft2(O.exit_wave(zk, Q))
        theta = np.angle(psi)
        zero = psi == 0
        theta[zero] = np.pi if prev_phase is None else prev_phase[zero]
        return O.ifft2(np.sqrt(dk) * np.exp(1j * theta))
    O.revised_exit_wave = rew


def m_proximal_without_u(O):
    O.proximal_step = lambda zk, Q, Rk, u: zk + O.safe_div(np.conj(Q), np.abs(Q) ** 2) * (Rk - Q * zk)


def m_forward_amplitude(O):
    O.forward_intensities = lambda z, Q, positions: np.stack(
        [np.abs(O.fft2(O.exit_wave(O.extract(z, p, Q.shape[0]), Q))) for p in positions])


def m_sweep_drops_short_minibatch(O):
    def sw(z, Q, positions, d, u, levels, order, minibatch):
        n = len(order) - len(order) % minibatch
        for s in range(0, n, minibatch):
            z = O.minibatch_step(z, Q, positions, d, u, levels, order[s:s + minibatch])
        return z
    O.sweep = sw


def m_minibatch_sequential(O):
    def mb(z, Q, positions, d, u, levels, batch):
        z = np.array(z, dtype=np.complex128, copy=True)
        m = Q.shape[0]
        for k in batch:
            r, c = positions[k]
            zk = z[r:r + m, c:c + m]
            Rk = O.revised_exit_wave(zk, Q, d[k])
            z[r:r + m, c:c + m] = O.magps(zk, Q, Rk, u, levels)
        return z
    O.minibatch_step = mb


def m_minibatch_unweighted(O):
    def mb(z, Q, positions, d, u, levels, batch):
        z = np.asarray(z, dtype=np.complex128)
        m = Q.shape[0]
        num = np.zeros(z.shape, dtype=np.complex128)
        den = np.zeros(z.shape, dtype=np.float64)
        for k in batch:
            r, c = positions[k]
            zk = z[r:r + m, c:c + m]
            Rk = O.revised_exit_wave(zk, Q, d[k])
            num[r:r + m, c:c + m] += O.magps(zk, Q, Rk, u, levels) - zk
            den[r:r + m, c:c + m] += 1.0
        out = z.copy()
        lit = den > 0
        out[lit] += num[lit] / den[lit]
        return out
    O.minibatch_step = mb


def m_regulariser_no_max(O):
    O.rpie_regulariser = lambda Q, alpha: alpha * (1.0 - np.abs(Q) ** 2)


def m_safe_div_unguarded(O):
    O.safe_div = lambda num, den: np.asarray(num) / np.asarray(den)


def m_gradient_scaled_twice(O):
    orig = O.gradient_k
    O.gradient_k = lambda zk, Q, dk: 2.0 * orig(zk, Q, dk)


def m_amplitude_form_unscaled(O):
    orig = O.objective_amplitude
    O.objective_amplitude = lambda z, Q, positions, d: orig(z, Q, positions, d) * Q.shape[0] ** 2


def m_magps_no_post_smoothing(O):
    orig_magps = O.magps

    def magps(zk, Q, Rk, u, levels):
        if levels == 1:
            return O.proximal_step(zk, Q, Rk, u)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(WR * Rk)
        uH = Wu * O.restrict(u)
        eH = magps(zH, QH, RH, uH, levels - 1) - zH
        return zk + O.prolong(eH)
    O.magps = magps


def m_coarse_r_unweighted(O):
    def magps(zk, Q, Rk, u, levels):
        if levels == 1:
            return O.proximal_step(zk, Q, Rk, u)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(Wz * zk)
        RH = O.restrict(Rk)
        uH = Wu * O.restrict(u)
        eH = magps(zH, QH, RH, uH, levels - 1) - zH
        return O.proximal_step(zk + O.prolong(eH), Q, Rk, u)
    O.magps = magps


def m_coarse_z_unweighted(O):
    def magps(zk, Q, Rk, u, levels):
        if levels == 1:
            return O.proximal_step(zk, Q, Rk, u)
        QH, Wz, WR, Wu = O.coarse_weights(Q)
        zH = O.restrict(zk)
        RH = O.restrict(WR * Rk)
        uH = Wu * O.restrict(u)
        eH = magps(zH, QH, RH, uH, levels - 1) - zH
        return O.proximal_step(zk + O.prolong(eH), Q, Rk, u)
    O.magps = magps


def m_sequential_reversed(O):
    orig = O.magpie_sequential
    O.magpie_sequential = lambda z, Q, positions, d, u, levels, order: orig(z, Q, positions, d, u, levels,
                                                                            list(order)[::-1])


def m_probe_ignores_beta(O):
    orig = O.probe_step
    O.probe_step = lambda z, Q, positions, d, beta, batch: orig(z, Q, positions, d, 0.0, batch)


def m_surrogate_at_new_point(O):
    def sur(z, zj, Q, positions, d):
        m = Q.shape[0]
        tot = 0.0
        for p, dk in zip(positions, d):
            Rk = O.revised_exit_wave(O.extract(z, p, m), Q, dk)  # R at z instead of z^(j)
            tot += 0.5 * float(np.sum(np.abs(O.exit_wave(O.extract(z, p, m), Q) - Rk) ** 2))
        return tot
    O.surrogate = sur


def m_extract_adjoint_shifted(O):
    def ea(patch, pos, shape):
        out = np.zeros(shape, dtype=np.complex128)
        r, c = pos
        m = patch.shape[0]
        r = min(r + 1, shape[0] - m)
        out[r:r + m, c:c + m] = patch
        return out
    O.extract_adjoint = ea


def m_wu_not_squared(O):
    orig = O.coarse_weights

    def cw(Q):
        QH, Wz, WR, Wu = orig(Q)
        return QH, Wz, WR, O.safe_div(np.abs(QH), O.restrict(np.abs(Q) ** 2))
    O.coarse_weights = cw


def m_mask_relative_to_sum(O):
    def im(Q, positions, shape, rel=1e-3):
        m = Q.shape[0]
        cov = np.zeros(shape)
        for r, c in positions:
            cov[r:r + m, c:c + m] += np.abs(Q) ** 2
        return cov >= rel * cov.sum()
    O.illuminated_mask = im


def m_mask_amplitude_coverage(O):
    def im(Q, positions, shape, rel=1e-3):
        m = Q.shape[0]
        cov = np.zeros(shape)
        for r, c in positions:
            cov[r:r + m, c:c + m] += np.abs(Q)
        return cov >= rel * cov.max()
    O.illuminated_mask = im


def m_magnitude_error_complex(O):
    O.magnitude_error = lambda z, z_true: float(np.linalg.norm(z - z_true))


def m_objective_skips_last_window(O):
    orig = O.objective
    O.objective = lambda z, Q, positions, d: orig(z, Q, positions[:-1], d[:-1])


def m_recycled_phase_not_stored(O):
    def rr(zk, Q, dk, prev_theta):
        psi = O.fft2(O.exit_wave(zk, Q))
        theta = np.angle(psi)
        zero = psi == 0
        theta[zero] = 0.0
        return O.ifft2(np.sqrt(dk) * np.exp(1j * theta)), theta
    O.revised_exit_wave_recycled = rr


MUTATIONS = [m_restrict_sum, m_prolong_scaled, m_fft_sign, m_fft_unnormalised_inverse,
             m_no_sqrt, m_gradient_no_conj, m_wr_no_conj, m_wz_unnormalised,
             m_uh_unweighted, m_post_smooth_from_z, m_minibatch_count_average,
             m_regulariser_amplitude, m_extract_transposed, m_objective_no_half,
             m_mgopt_shift_sign, m_mgopt_weighted_restriction, m_phase_rule_forgets,
             m_stop_metric_extra_inv_m, m_stop_metric_squared_norms, m_stop_metric_sum_not_mean,
             m_nrmse_swapped, m_nrmse_no_phase, m_nrmse_conjugate_phase,
             m_probe_step_sign, m_probe_regulariser_of_probe, m_theta_zero_is_pi, m_proximal_without_u,
             m_forward_amplitude, m_sweep_drops_short_minibatch, m_minibatch_sequential, m_minibatch_unweighted,
             m_regulariser_no_max, m_safe_div_unguarded,
             m_gradient_scaled_twice, m_amplitude_form_unscaled, m_magps_no_post_smoothing, m_coarse_r_unweighted,
             m_coarse_z_unweighted, m_sequential_reversed, m_probe_ignores_beta, m_surrogate_at_new_point,
             m_extract_adjoint_shifted, m_wu_not_squared,
             m_mask_relative_to_sum, m_mask_amplitude_coverage, m_magnitude_error_complex,
             m_objective_skips_last_window, m_recycled_phase_not_stored]

FAST_CHECKS = [c for c in pins.ALL_CHECKS if c is not pins.check_recovery]


@pytest.mark.parametrize("mutate", MUTATIONS, ids=lambda f: f.__name__[2:])
def test_planted_mistake_is_caught(mutate):
    O = fresh_oracle()
    mutate(O)
    failed = []
    for check in FAST_CHECKS:
        try:
            with np.errstate(all="ignore"):
                check(O)
        except (AssertionError, ValueError, IndexError, ZeroDivisionError, FloatingPointError):
            failed.append(check.__name__)
    assert failed, f"no pin caught {mutate.__name__}"
