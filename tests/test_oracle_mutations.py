"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins catch each one: a dropped term, a wrong sign, a wrong index, a
transposed operand, a wrong constant."""
import numpy as np
import pytest

import pins
from oracle import model as m


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
]


@pytest.mark.parametrize("name,bad,catchers", MUTANTS,
                         ids=[f"{n}:{b.__name__}" for n, b, _ in MUTANTS])
def test_pin_catches_planted_mistake(monkeypatch, name, bad, catchers):
    monkeypatch.setattr(m, name, bad)
    caught = 0
    for pin in catchers:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError):
            caught += 1
    assert caught == len(catchers), f"{name} mutant {bad.__name__} not caught"
