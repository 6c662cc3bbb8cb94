"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins catch each one: a dropped term, a wrong sign, a wrong index, a
transposed operand, a wrong constant, and in Algorithm 3's control flow a
wrong comparison, a missing latch, an off-by-one or mis-counted iteration."""
import numpy as np
import pytest

import pins
from oracle import model as m
from oracle import solvers as s


def _bad_gradient_half(H, U, W, V, alpha, K, Nr, d):
    # linear term without its factor 2
    C = H.shape[0]
    G = np.zeros_like(V)
    for k in range(C):
        F = m.F_matrix(H, U, W, alpha, k, K, Nr)
        for i in range(K):
            r = k * K + i
            cols = slice(i * d, (i + 1) * d)
            G[k][:, cols] = F @ V[k][:, cols] - alpha[r] * m.link(H, r, k, Nr).conj().T @ U[r] @ W[r]
    return G


def _bad_F_transpose(H, U, W, alpha, k, K, Nr):
    # H^T instead of H^H
    C, _, Nt = H.shape
    F = np.zeros((Nt, Nt), dtype=complex)
    for r in range(C * K):
        Hrk = m.link(H, r, k, Nr)
        F = F + 2.0 * alpha[r] * Hrk.T @ U[r] @ W[r] @ U[r].conj().T @ Hrk
    return F


def _bad_F_own_cell(H, U, W, alpha, k, K, Nr):
    # link to the user's own BS instead of BS k (wrong index)
    C, _, Nt = H.shape
    F = np.zeros((Nt, Nt), dtype=complex)
    for r in range(C * K):
        Hrk = m.link(H, r, r // K, Nr)
        F = F + 2.0 * alpha[r] * Hrk.conj().T @ U[r] @ W[r] @ U[r].conj().T @ Hrk
    return F


_orig_mse = m.mse_matrix


def _bad_mse_no_noise(H, U, V, sigma2, r, K, Nr, d):
    return _orig_mse(H, U, V, np.zeros_like(sigma2), r, K, Nr, d)


_orig_cov = m.receive_covariance


def _bad_cov_sign(H, V, sigma2, r, K, Nr, d):
    # noise entered with the wrong sign
    return _orig_cov(H, V, sigma2, r, K, Nr, d) - 2 * sigma2[r] * np.eye(Nr)


def _bad_weight_no_inverse(H, U, V, K, Nr, d):
    C = H.shape[0]
    return [np.eye(d) - U[r].conj().T @ m.link(H, r, r // K, Nr) @ m.prec(V, r, K, d)
            for r in range(C * K)]


def _bad_project_power(Vk, Pk):
    p = float(np.sum(np.abs(Vk) ** 2))
    return Vk.copy() if p <= Pk else Vk * (Pk / p)


def _bad_omega(t):
    return max((t - 1.0) / (t + 2.0), 0.0)


_orig_rate = m.rate


def _bad_rate_intracell_only(H, V, sigma2, r, K, Nr, d):
    # interference from other cells dropped
    C = H.shape[0]
    k = r // K
    Hs = H.copy()
    for j in range(C):
        if j != k:
            Hs[j, r * Nr:(r + 1) * Nr] = 0.0
    return _orig_rate(Hs, V, sigma2, r, K, Nr, d)


def _bad_spectral_half(H, U, W, alpha, k, K, Nr):
    F = m.F_matrix(H, U, W, alpha, k, K, Nr)
    return 2.0 / float(np.linalg.eigvalsh(0.5 * (F + F.conj().T))[-1])


# ---- Algorithm 3's control flow (oracle.solvers decisions)
def _bad_stage_strict(stage, t, rho, rho_prev, opt):
    # "> eps1" instead of "<= eps1"
    if stage != 1:
        return stage
    if opt.switch_iter >= 1:
        return 2 if t >= opt.switch_iter else 1
    return 2 if (rho_prev is not None and m.relative_change(rho, rho_prev) > opt.eps1) else 1


def _bad_stage_at_t2(stage, t, rho, rho_prev, opt):
    # switches at the first test whatever the WSR change
    if stage != 1:
        return stage
    if opt.switch_iter >= 1:
        return 2 if t >= opt.switch_iter else 1
    return 2 if rho_prev is not None else 1


def _bad_stage_no_latch(stage, t, rho, rho_prev, opt):
    # re-tests every iteration: back to W = I when the change grows again
    if opt.switch_iter >= 1:
        return 2 if t >= opt.switch_iter else 1
    return 2 if (rho_prev is not None and m.relative_change(rho, rho_prev) <= opt.eps1) else 1


def _bad_stage_one_late(stage, t, rho, rho_prev, opt):
    # the test is not trusted until t = 3
    if stage != 1:
        return stage
    if opt.switch_iter >= 1:
        return 2 if t >= opt.switch_iter else 1
    return 2 if (t >= 3 and rho_prev is not None and m.relative_change(rho, rho_prev) <= opt.eps1) else 1


def _bad_spectral_global_t(stage_iter, t, opt):
    # Tc counted on the global iteration counter
    return opt.step_rule == 1 or (opt.step_rule == 0 and t <= opt.Tc)


def _bad_freeze_global_t(stage_iter, t, opt):
    return opt.step_rule == 0 and t == opt.Tc


def _bad_spectral_short(stage_iter, t, opt):
    # one spectral iteration too few
    return opt.step_rule == 1 or (opt.step_rule == 0 and stage_iter < opt.Tc)


def _bad_freeze_early(stage_iter, t, opt):
    # gamma_c taken from the stage's second iteration
    return opt.step_rule == 0 and stage_iter == opt.Tc - 1


def _bad_tolerance_any_stage(rho, rho_prev, last_stage, eps2):
    # stops on a small change even before any stage-II iteration
    return rho_prev is not None and m.relative_change(rho, rho_prev) <= eps2


def _bad_mmmse_switch_first(hist, eps1):
    # the MMMSE baseline skips its W = I stage
    return True


_orig_wpc = s.wmmse_precoder_cell


def _bad_wpc_lower_end(H, U, W, alpha, P, k, K, Nr, d, tol=1e-4, max_bisect=100, exact=False):
    # eq. (12) at a multiplier 10 % below the bisection's (infeasible power)
    V, lam = _orig_wpc(H, U, W, alpha, P, k, K, Nr, d, tol, max_bisect, exact)
    if lam <= 0:
        return V, lam
    C, _, Nt = H.shape
    A = np.zeros((Nt, Nt), dtype=complex)
    B = np.zeros((Nt, K * d), dtype=complex)
    for r in range(C * K):
        Hrk = m.link(H, r, k, Nr)
        A = A + alpha[r] * Hrk.conj().T @ U[r] @ W[r] @ U[r].conj().T @ Hrk
    for i in range(K):
        r = k * K + i
        B[:, i * d:(i + 1) * d] = alpha[r] * m.link(H, r, k, Nr).conj().T @ U[r] @ W[r]
    lam2 = 0.9 * lam
    return np.linalg.solve(A + lam2 * np.eye(Nt), B), lam2


def _bad_wpc_no_alpha(H, U, W, alpha, P, k, K, Nr, d, tol=1e-4, max_bisect=100, exact=False):
    # the priority weights dropped from eq. (12)
    return _orig_wpc(H, U, W, np.ones_like(alpha), P, k, K, Nr, d, tol, max_bisect, exact)


MUTANTS = [
    ("gradient", _bad_gradient_half, [pins.pin_gradient_fd]),
    ("F_matrix", _bad_F_transpose, [pins.pin_gradient_fd]),
    ("F_matrix", _bad_F_own_cell, [pins.pin_gradient_fd]),
    ("mse_matrix", _bad_mse_no_noise, [pins.pin_wsr_equivalence]),
    ("receive_covariance", _bad_cov_sign, [pins.pin_wsr_equivalence, pins.pin_U_minimizer]),
    ("mse_weight", _bad_weight_no_inverse, [pins.pin_wsr_equivalence]),
    ("project", _bad_project_power, [pins.pin_projection]),
    ("extrapolation_weight", _bad_omega, [pins.pin_omega_and_defaults]),
    ("rate", _bad_rate_intracell_only, [pins.pin_rate_scalar_sinr]),
    ("spectral_step", _bad_spectral_half, [pins.pin_spectral_step_factor]),
    ("next_stage", _bad_stage_strict, [pins.pin_stage_switch_rule]),
    ("next_stage", _bad_stage_at_t2, [pins.pin_stage_switch_rule, pins.pin_tolerance_stop]),
    ("next_stage", _bad_stage_no_latch, [pins.pin_stage_switch_rule]),
    ("next_stage", _bad_stage_one_late, [pins.pin_stage_switch_rule]),
    ("spectral_step_used", _bad_spectral_global_t, [pins.pin_step_size_schedule]),
    ("freezes_gamma_c", _bad_freeze_global_t, [pins.pin_step_size_schedule]),
    ("spectral_step_used", _bad_spectral_short, [pins.pin_step_size_schedule]),
    ("freezes_gamma_c", _bad_freeze_early, [pins.pin_step_size_schedule]),
    ("tolerance_reached", _bad_tolerance_any_stage, [pins.pin_tolerance_stop]),
    ("mmmse_switch", _bad_mmmse_switch_first, [pins.pin_mmmse_first_stage]),
    ("wmmse_precoder_cell", _bad_wpc_lower_end, [pins.pin_V_minimizer, pins.pin_bisection_slackness]),
    ("wmmse_precoder_cell", _bad_wpc_no_alpha, [pins.pin_V_minimizer]),
]


@pytest.mark.parametrize("name,bad,catchers", MUTANTS,
                         ids=[f"{n}:{b.__name__}" for n, b, _ in MUTANTS])
def test_pin_catches_planted_mistake(monkeypatch, name, bad, catchers):
    monkeypatch.setattr(m if hasattr(m, name) else s, name, bad)
    caught = 0
    for pin in catchers:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError):
            caught += 1
    assert caught == len(catchers), f"{name} mutant {bad.__name__} not caught"
