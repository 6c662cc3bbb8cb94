"""FP64 oracle, part 1: the system model and the WMMSE reformulation.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
CPU restatement of the paper's equations in float64/complex128.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the GPU library never calls it and shares no code with it.

Notation follows the paper (arXiv 2510.20507) with the build's letters:
C cells (paper K), K users per cell (paper I), Nt BS antennas (paper M),
Nr receive antennas (paper N), d streams.  User r = k*K + i is user i_k.

Layouts (see ``workloads``):
  H (C, C*K*Nr, Nt)   H[j, r*Nr:(r+1)*Nr] = H_{r j}
  V (C, Nt, K*d)      V[k][:, i*d:(i+1)*d] = V_{i_k}
  U list of (Nr, d), W list of (d, d), one per user r.

Every function cites the passage of the paper it restates.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------- indexing
def dims(H: np.ndarray, V: np.ndarray):
    C, rows, Nt = H.shape
    Kd = V.shape[2]
    return C, rows, Nt, Kd


def cell_of(r: int, K: int) -> int:
    return r // K


def link(H: np.ndarray, r: int, j: int, Nr: int) -> np.ndarray:
    """H_{r j}: channel from BS j to user r (N_r x N_t), system model Sec. II."""
    return H[j, r * Nr:(r + 1) * Nr, :]


def prec(V: np.ndarray, r: int, K: int, d: int) -> np.ndarray:
    """V_{i_k} for r = k*K + i (N_t x d)."""
    k, i = divmod(r, K)
    return V[k][:, i * d:(i + 1) * d]


def users(C: int, K: int):
    return range(C * K)


# ------------------------------------------------------------ rate and WSR
def rate(H, V, sigma2, r, K, Nr, d) -> float:
    """Achievable rate R_{i_k} in nats, written exactly as defined below
    problem (1) (Sec. II): log det(I + H_kk V V^H H_kk^H (interference +
    sigma^2 I)^{-1}), interference summed over every other stream (l, j)."""
    C = H.shape[0]
    k = cell_of(r, K)
    Hrk = link(H, r, k, Nr)
    Vr = prec(V, r, K, d)
    interf = sigma2[r] * np.eye(Nr, dtype=complex)
    for rr in users(C, K):
        if rr == r:
            continue
        j = cell_of(rr, K)
        Hrj = link(H, r, j, Nr)
        Vl = prec(V, rr, K, d)
        interf = interf + Hrj @ Vl @ Vl.conj().T @ Hrj.conj().T
    S = Hrk @ Vr @ Vr.conj().T @ Hrk.conj().T
    M = np.eye(Nr) + S @ np.linalg.inv(interf)
    # det M = det(interference + S) / det(interference) is real and positive
    _, logabsdet = np.linalg.slogdet(M)
    return float(logabsdet)


def rates(H, V, sigma2, K, Nr, d) -> np.ndarray:
    C = H.shape[0]
    return np.array([rate(H, V, sigma2, r, K, Nr, d) for r in users(C, K)])


def wsr(H, V, sigma2, alpha, K, Nr, d) -> float:
    """Weighted sum rate, objective of problem (1), in nats."""
    return float(np.dot(alpha, rates(H, V, sigma2, K, Nr, d)))


def wsr_bits(H, V, sigma2, alpha, K, Nr, d) -> float:
    """WSR in bits per channel use (the unit of Sec. VII's figures)."""
    return wsr(H, V, sigma2, alpha, K, Nr, d) / np.log(2.0)


# --------------------------------------------------------- MSE and objective
def mse_matrix(H, U, V, sigma2, r, K, Nr, d) -> np.ndarray:
    """E_{i_k} of eq. (7), term by term: own-stream error, interference
    from every other stream (l, j) != (i, k), and noise."""
    C = H.shape[0]
    k = cell_of(r, K)
    Ur = U[r]
    A = np.eye(d) - Ur.conj().T @ link(H, r, k, Nr) @ prec(V, r, K, d)
    E = A @ A.conj().T
    for rr in users(C, K):
        if rr == r:
            continue
        j = cell_of(rr, K)
        B = Ur.conj().T @ link(H, r, j, Nr) @ prec(V, rr, K, d)
        E = E + B @ B.conj().T
    return E + sigma2[r] * (Ur.conj().T @ Ur)


def objective(H, U, W, V, sigma2, alpha, K, Nr, d) -> float:
    """f(U, W, V) = sum alpha (Tr(W E) - log det W), objective of problem (8)."""
    C = H.shape[0]
    total = 0.0
    for r in users(C, K):
        E = mse_matrix(H, U, V, sigma2, r, K, Nr, d)
        sign, logdetW = np.linalg.slogdet(W[r])
        total += alpha[r] * (np.trace(W[r] @ E).real - logdetW)
    return float(total)


def sum_mse(H, U, V, sigma2, alpha, K, Nr, d) -> float:
    """Weighted sum-MSE, objective of problem (6)."""
    C = H.shape[0]
    return float(sum(alpha[r] * np.trace(mse_matrix(H, U, V, sigma2, r, K, Nr, d)).real
                     for r in users(C, K)))


# -------------------------------------------------- block-coordinate updates
def receive_covariance(H, V, sigma2, r, K, Nr, d) -> np.ndarray:
    """sum_{j,l} H_{r j} V_{l j} V_{l j}^H H_{r j}^H + sigma^2 I, the matrix
    inverted in eq. (9)."""
    C = H.shape[0]
    T = sigma2[r] * np.eye(Nr, dtype=complex)
    for rr in users(C, K):
        j = cell_of(rr, K)
        Hrj = link(H, r, j, Nr)
        Vl = prec(V, rr, K, d)
        T = T + Hrj @ Vl @ Vl.conj().T @ Hrj.conj().T
    return T


def mmse_receiver(H, V, sigma2, K, Nr, d, cov_hook=None):
    """U update, eq. (9): U_{i_k} = T^{-1} H_{i_k k} V_{i_k} (eq. (9) writes
    H_{i_k}; the direct link H_{i_k k} is meant).  ``cov_hook``, if given,
    is applied to each T before the solve (the FP32-sensitivity study of
    ``oracle.sensitivity`` rounds T there; no solver path sets it)."""
    C = H.shape[0]
    out = []
    for r in users(C, K):
        T = receive_covariance(H, V, sigma2, r, K, Nr, d)
        if cov_hook is not None:
            T = cov_hook(T)
        k = cell_of(r, K)
        out.append(np.linalg.solve(T, link(H, r, k, Nr) @ prec(V, r, K, d)))
    return out


def mse_weight(H, U, V, K, Nr, d):
    """W update, eq. (10): W = (I - U^H H_kk V)^{-1}.  The inverse is
    Hermitian in exact arithmetic; its Hermitian part is returned."""
    C = H.shape[0]
    out = []
    for r in users(C, K):
        k = cell_of(r, K)
        E = np.eye(d) - U[r].conj().T @ link(H, r, k, Nr) @ prec(V, r, K, d)
        Wr = np.linalg.inv(E)
        out.append(0.5 * (Wr + Wr.conj().T))
    return out


def identity_weights(C, K, d):
    """W = I, the stage-I weight of the mixed scheme (problem (19))."""
    return [np.eye(d, dtype=complex) for _ in users(C, K)]


def F_matrix(H, U, W, alpha, k, K, Nr) -> np.ndarray:
    """F_k = sum_{(l,j)} 2 alpha H_{l_j k}^H U W U^H H_{l_j k}: the matrix
    multiplying V in the gradient (14) and inside the norm of eq. (16)."""
    C, _, Nt = H.shape
    F = np.zeros((Nt, Nt), dtype=complex)
    for r in users(C, K):
        Hrk = link(H, r, k, Nr)
        F = F + 2.0 * alpha[r] * Hrk.conj().T @ U[r] @ W[r] @ U[r].conj().T @ Hrk
    return F


def gradient(H, U, W, V, alpha, K, Nr, d) -> np.ndarray:
    """Gradient of f in V, eq. (14): F_k V_{i_k} - 2 alpha H_{i_k k}^H U W,
    with F_k formed explicitly."""
    C = H.shape[0]
    G = np.zeros_like(V)
    for k in range(C):
        F = F_matrix(H, U, W, alpha, k, K, Nr)
        for i in range(K):
            r = k * K + i
            cols = slice(i * d, (i + 1) * d)
            G[k][:, cols] = (F @ V[k][:, cols]
                             - 2.0 * alpha[r] * link(H, r, k, Nr).conj().T @ U[r] @ W[r])
    return G


def project(Vk: np.ndarray, Pk: float) -> np.ndarray:
    """Projection onto the k-th sum-power constraint, eq. (15)."""
    power = float(np.sum(np.abs(Vk) ** 2))
    if power <= Pk:
        return Vk.copy()
    return Vk * np.sqrt(Pk / power)


def spectral_step(H, U, W, alpha, k, K, Nr) -> float:
    """gamma = 1 / ||F_k||_2, first branch of eq. (16); F_k is Hermitian
    PSD so its spectral norm is its largest eigenvalue."""
    F = F_matrix(H, U, W, alpha, k, K, Nr)
    lam = float(np.linalg.eigvalsh(0.5 * (F + F.conj().T))[-1])
    return 1.0 / lam


def extrapolation_weight(t: int) -> float:
    """omega^t = max((t - 2)/(t + 1), 0), eq. (18)."""
    return max((t - 2.0) / (t + 1.0), 0.0)


def relative_change(new: float, old: float) -> float:
    """|R^t - R^{t-1}| / R^{t-1}, the test of Algorithms 2 and 3 (the paper
    divides by R^{t-1}; WSR is positive here)."""
    return abs(new - old) / abs(old)
