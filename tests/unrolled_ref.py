"""Reference gradients for the unrolled A-MMMSE: the unrolled iteration of
Algorithm 3 restated with plain torch float64 CPU ops (eqs. (9), (10),
(13)-(18), with F_k formed explicitly as in eq. (14)), differentiated by
torch autograd.  Test infrastructure; pinned to the oracle's
ammmse_unrolled in tests/test_unrolled.py."""
import math

import torch


def unrolled_wsr_torch(H, sigma2, alpha, P, V0, gammas, K, Nr, d, switch_iter, extrapolate=True):
    """Single cell.  H: (K Nr, Nt) complex128, sigma2 / alpha: (K,) float64,
    P: float, V0: (Nt, K d) complex128, gammas: (T,) float64.  Returns
    WSR(V^T) in bits."""
    dt = H.dtype
    Nt = H.shape[1]
    V, Vp = V0, V0
    T = gammas.shape[0]
    eyeN = torch.eye(Nr, dtype=dt)
    eyed = torch.eye(d, dtype=dt)
    for t in range(1, T + 1):
        omega = max((t - 2.0) / (t + 1.0), 0.0) if extrapolate else 0.0
        Vh = V + omega * (V - Vp) if t >= 2 else V
        stage2 = switch_iter >= 1 and t >= switch_iter
        F = torch.zeros(Nt, Nt, dtype=dt)
        B = []
        for r in range(K):
            Hr = H[r * Nr:(r + 1) * Nr]
            Tr = sigma2[r] * eyeN + Hr @ V @ V.conj().T @ Hr.conj().T
            Vr = V[:, r * d:(r + 1) * d]
            Ur = torch.linalg.solve(Tr, Hr @ Vr)                         # eq. (9)
            if stage2:
                Wr = torch.linalg.inv(eyed - Ur.conj().T @ Hr @ Vr)     # eq. (10)
                Wr = 0.5 * (Wr + Wr.conj().T)
            else:
                Wr = eyed
            F = F + 2.0 * alpha[r] * Hr.conj().T @ Ur @ Wr @ Ur.conj().T @ Hr
            B.append(2.0 * alpha[r] * Hr.conj().T @ Ur @ Wr)
        G = F @ Vh - torch.cat(B, dim=1)                                  # eq. (14)
        Vt = Vh - gammas[t - 1] * G                                       # eq. (13)
        power = (Vt.abs() ** 2).sum()
        Vn = Vt * torch.sqrt(P / power) if power.item() > P else Vt      # eq. (15)
        Vp, V = V, Vn
    total = torch.zeros((), dtype=torch.float64)
    for r in range(K):
        Hr = H[r * Nr:(r + 1) * Nr]
        Tr = sigma2[r] * eyeN + Hr @ V @ V.conj().T @ Hr.conj().T
        Vr = V[:, r * d:(r + 1) * d]
        Sr = Hr @ Vr @ Vr.conj().T @ Hr.conj().T
        total = total + alpha[r] * (torch.linalg.slogdet(Tr)[1] - torch.linalg.slogdet(Tr - Sr)[1])
    return total / math.log(2.0)
