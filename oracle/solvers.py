"""FP64 oracle, part 2: Algorithm 2 (WMMSE) and Algorithm 3 (A-MMMSE).

TEST INFRASTRUCTURE ONLY (see ``oracle.model``).  The steps run in the order
the paper lists them, one user and one cell at a time, with the readings of
the paper's silent or ambiguous points passed in as options:

  u_at_extrapolated  U^t is computed at V^{t-1} (False, default) or at the
                     extrapolated point (True).
  switch_iter        -1: the stage switch of Algorithm 3 fires at the first
                     t >= 2 whose relative WSR change is <= eps1 and stays on;
                     s >= 1: stage II from iteration s on (1 gives A-WMMSE).
  step_rule          0: gamma = 1/||F_k||_2 for the first Tc iterations of
                     each stage, then the last such value is kept (gamma_c);
                     1: 1/||F_k||_2 at every iteration; 2: gamma_c fixed.
  gamma_c            a positive value overrides the frozen gamma_c.
  extrapolate        False gives the "(w/o extrap.)" variants (omega = 0).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import model as m


@dataclasses.dataclass
class Options:
    eps1: float = 0.1          # Sec. VII-A: all MMMSE methods use eps1 = 0.1
    eps2: float = 1e-3         # Sec. VII-D: eps2 = 0.001
    Tc: int = 3                # Sec. V-A: Tc = 3
    gamma_c: float = 0.0
    extrapolate: bool = True
    switch_iter: int = -1
    step_rule: int = 0
    u_at_extrapolated: bool = False


@dataclasses.dataclass
class IterRecord:
    t: int
    omega: float
    rho: float                 # R^t = WSR(V^{t-1}) in nats (reading: Alg. 3 tests it)
    stage: int                 # 1 (W = I) or 2 (W from eq. (10)) in this iteration
    gamma: np.ndarray          # step size per cell used in this iteration
    V: np.ndarray              # V^t after the projected step


@dataclasses.dataclass
class SolveResult:
    V: np.ndarray              # final iterate
    Vprev: np.ndarray          # the iterate before it
    history: List[IterRecord]
    iters: int
    converged: bool
    gamma_c: np.ndarray
    stage: int
    stage_iter: int
    rho_prev: float


def initial_precoder(G0: np.ndarray, P: np.ndarray) -> np.ndarray:
    """V^0: the CN(0,1) draws projected onto each cell's power ball
    (Sec. VII-A setup, eq. (15))."""
    return np.stack([m.project(G0[k], P[k]) for k in range(G0.shape[0])])


@dataclasses.dataclass
class AState:
    """Resumable state of Algorithm 3 between iterations."""
    V: np.ndarray              # V^{t-1}
    Vprev: np.ndarray          # V^{t-2}
    t: int = 1
    stage: int = 1
    stage_iter: int = 0
    rho_prev: Optional[float] = None
    gamma_c: Optional[np.ndarray] = None


# ---- the control flow of Algorithm 3, one decision per function (the
#      planted-mistake tests replace them one at a time)
def next_stage(stage: int, t: int, rho: float, rho_prev: Optional[float], opt: Options) -> int:
    """The stage (1: W = I, 2: W from eq. (10)) of iteration t.  Algorithm 3
    leaves stage I once the relative WSR change is at most eps1; the test
    needs R^{t-1}, so it cannot fire at t = 1.  Once in stage II the scheme
    stays there (reading: the switch latches).  switch_iter >= 1 forces the
    switch at that iteration instead."""
    if stage != 1:
        return stage
    if opt.switch_iter >= 1:
        return 2 if t >= opt.switch_iter else 1
    go = rho_prev is not None and m.relative_change(rho, rho_prev) <= opt.eps1
    return 2 if go else 1


def spectral_step_used(stage_iter: int, t: int, opt: Options) -> bool:
    """Whether eq. (16) takes gamma = 1/||F_k||_2 in iteration t, the
    stage_iter-th iteration of the current stage (step_rule 0: the stage's
    first Tc iterations, the per-stage reading of eq. (16); 1: always;
    2: never).  The global counter t does not enter the per-stage reading."""
    return opt.step_rule == 1 or (opt.step_rule == 0 and stage_iter <= opt.Tc)


def freezes_gamma_c(stage_iter: int, t: int, opt: Options) -> bool:
    """Whether the spectral step of this iteration becomes gamma_c, the
    constant step of eq. (16) for the rest of the stage (step_rule 0: the
    step of the stage's Tc-th iteration)."""
    return opt.step_rule == 0 and stage_iter == opt.Tc


def tolerance_reached(rho: float, rho_prev: Optional[float], last_stage: int, eps2: float) -> bool:
    """The stopping test of Algorithm 3: the relative WSR change is at most
    eps2, checked only after an iteration of the second (weighted) stage."""
    return last_stage == 2 and rho_prev is not None and m.relative_change(rho, rho_prev) <= eps2


def ammmse_iteration(H, sigma2, alpha, P, K, Nr, d, st: AState, opt: Options,
                     cov_hook=None, step_hook=None) -> IterRecord:
    """One pass of the repeat-loop of Algorithm 3, advancing ``st`` in place.

    ``cov_hook`` / ``step_hook`` perturb the receive covariance of eq. (9)
    and the spectral step of eq. (16) for ``oracle.sensitivity``; every
    solver path leaves them unset."""
    C = H.shape[0]
    t = st.t
    # omega^t, eq. (18); extrapolated point, eq. (17)
    omega = m.extrapolation_weight(t) if opt.extrapolate else 0.0
    Vhat = st.V + omega * (st.V - st.Vprev) if t >= 2 else st.V.copy()
    # U^t by eq. (9)
    U = m.mmse_receiver(H, Vhat if opt.u_at_extrapolated else st.V, sigma2, K, Nr, d, cov_hook=cov_hook)
    # R^t: WSR of the current iterate V^{t-1}
    rho = m.wsr(H, st.V, sigma2, alpha, K, Nr, d)
    # stage test of Algorithm 3 (latched)
    stage = next_stage(st.stage, t, rho, st.rho_prev, opt)
    if stage != st.stage:
        st.stage = stage
        st.stage_iter = 0
    if st.stage == 2:
        W = m.mse_weight(H, U, st.V, K, Nr, d)             # eq. (10)
    else:
        W = m.identity_weights(C, K, d)                     # W = I
    st.stage_iter += 1
    # gamma^t by eq. (16)
    if st.gamma_c is None:
        st.gamma_c = np.zeros(C)
    gamma = np.zeros(C)
    for k in range(C):
        if spectral_step_used(st.stage_iter, t, opt):
            gamma[k] = m.spectral_step(H, U, W, alpha, k, K, Nr)
            if step_hook is not None:
                gamma[k] = step_hook(gamma[k])
            if freezes_gamma_c(st.stage_iter, t, opt):
                st.gamma_c[k] = gamma[k]
        else:
            gamma[k] = opt.gamma_c if opt.gamma_c > 0 else st.gamma_c[k]
    # V^t by eq. (13) with the gradient (14) at the extrapolated point and eq. (15)
    G = m.gradient(H, U, W, Vhat, alpha, K, Nr, d)
    Vnew = np.stack([m.project(Vhat[k] - gamma[k] * G[k], P[k]) for k in range(C)])
    rec = IterRecord(t=t, omega=omega, rho=rho, stage=st.stage, gamma=gamma, V=Vnew)
    st.Vprev = st.V
    st.V = Vnew
    st.rho_prev = rho
    st.t = t + 1
    return rec


def ammmse(H, sigma2, alpha, P, K, Nr, d, V0, iters: int,
           opt: Optional[Options] = None, tolerance_stop: bool = False,
           state: Optional[AState] = None) -> SolveResult:
    """Algorithm 3 (A-MMMSE) from V^0 for ``iters`` iterations.

    With ``tolerance_stop`` the loop ends once an iteration that followed a
    stage-II iteration sees a relative WSR change <= eps2; the iterate tested
    is then the result.
    """
    opt = opt or Options()
    st = state or AState(V=V0.copy(), Vprev=V0.copy())
    hist: List[IterRecord] = []
    converged = False
    for _ in range(iters):
        if tolerance_stop and hist:
            rho = m.wsr(H, st.V, sigma2, alpha, K, Nr, d)
            if tolerance_reached(rho, st.rho_prev, hist[-1].stage, opt.eps2):
                converged = True
                break
        hist.append(ammmse_iteration(H, sigma2, alpha, P, K, Nr, d, st, opt))
    return SolveResult(V=st.V, Vprev=st.Vprev, history=hist, iters=len(hist),
                       converged=converged, gamma_c=st.gamma_c, stage=st.stage,
                       stage_iter=st.stage_iter, rho_prev=st.rho_prev)


# ------------------------------------------------------------------ WMMSE
def wmmse_precoder_cell(H, U, W, alpha, P, k, K, Nr, d, tol: float = 1e-4,
                        max_bisect: int = 100, exact: bool = False):
    """V update of eq. (12) for cell k with lambda_k >= 0 from bisection.

    A_k = sum alpha H^H U W U^H H and B_k = [alpha H_{i_k k}^H U W]_i.  With the
    eigen-decomposition A_k = Q diag(l) Q^H the cell power at multiplier lam
    is p(lam) = sum_m phi_m/(l_m + lam)^2, phi = row norms of Q^H B.  lam = 0
    when A_k is nonsingular and p(0) <= P_k; otherwise bisect on
    [0, ||B||_F / sqrt(P_k)] (p(lam) <= ||B||_F^2/lam^2 bounds the top end).
    Stops when the interval is narrower than ``tol`` (absolute, the setting
    of Sec. VII-A) or after ``max_bisect`` halvings, and returns the upper end
    so the power constraint holds.  ``exact`` uses a relative width of 1e-14.
    """
    C, _, Nt = H.shape
    A = np.zeros((Nt, Nt), dtype=complex)
    for r in m.users(C, K):
        Hrk = m.link(H, r, k, Nr)
        A = A + alpha[r] * Hrk.conj().T @ U[r] @ W[r] @ U[r].conj().T @ Hrk
    A = 0.5 * (A + A.conj().T)
    B = np.zeros((Nt, K * d), dtype=complex)
    for i in range(K):
        r = k * K + i
        B[:, i * d:(i + 1) * d] = alpha[r] * m.link(H, r, k, Nr).conj().T @ U[r] @ W[r]
    lam_e, Q = np.linalg.eigh(A)
    lam_e = np.maximum(lam_e, 0.0)
    phi = np.sum(np.abs(Q.conj().T @ B) ** 2, axis=1)

    def power(mu):
        return float(np.sum(phi / (lam_e + mu) ** 2))

    def solve(mu):
        return Q @ ((Q.conj().T @ B) / (lam_e + mu)[:, None])

    scale = max(float(lam_e[-1]), 1.0)
    if lam_e[0] > 1e-12 * scale and power(0.0) <= P[k]:
        return solve(0.0), 0.0
    lo, hi = 0.0, float(np.linalg.norm(B)) / np.sqrt(P[k])
    for _ in range(max_bisect if not exact else 400):
        width = hi - lo
        if (not exact and width < tol) or (exact and width <= 1e-14 * hi):
            break
        mid = 0.5 * (lo + hi)
        if power(mid) > P[k]:
            lo = mid
        else:
            hi = mid
    return solve(hi), hi


@dataclasses.dataclass
class WState:
    V: np.ndarray
    rho_prev: Optional[float] = None


def mmmse_switch(hist, eps1: float) -> bool:
    """Whether the MMMSE baseline leaves its W = I stage: the relative
    change of the last two WSR values (hist holds WSR(V^0), WSR(V^1), ...)
    is at most eps1; it needs two values, so the first iteration is always
    an MMSE one."""
    return len(hist) >= 2 and m.relative_change(hist[-1], hist[-2]) <= eps1


def wmmse(H, sigma2, alpha, P, K, Nr, d, V0, iters: int, tol: float = 1e-4,
          max_bisect: int = 100, exact: bool = False, eps: Optional[float] = None,
          mmse_first_stage: bool = False, eps1: float = 0.1):
    """Algorithm 2 (WMMSE): U by eq. (9), W by eq. (10), V by eq. (12).

    ``eps`` enables the relative-WSR stopping test.  ``mmse_first_stage``
    gives the MMMSE baseline: W = I (so eq. (12) becomes eq. (20)) until the
    relative WSR change first drops to eps1.  Returns (V, list of WSR(V^t)
    in nats for t = 0..iters, iterations run).
    """
    C = H.shape[0]
    V = V0.copy()
    hist = [m.wsr(H, V, sigma2, alpha, K, Nr, d)]
    stage = 1 if mmse_first_stage else 2
    it = 0
    for it in range(1, iters + 1):
        U = m.mmse_receiver(H, V, sigma2, K, Nr, d)
        if stage == 1 and mmmse_switch(hist, eps1):
            stage = 2
        W = m.mse_weight(H, U, V, K, Nr, d) if stage == 2 else m.identity_weights(C, K, d)
        V = np.stack([wmmse_precoder_cell(H, U, W, alpha, P, k, K, Nr, d, tol,
                                          max_bisect, exact)[0] for k in range(C)])
        hist.append(m.wsr(H, V, sigma2, alpha, K, Nr, d))
        if eps is not None and m.relative_change(hist[-1], hist[-2]) <= eps:
            break
    return V, hist, it


# --------------------------------------------------- unrolled A-MMMSE
def ammmse_unrolled(H, sigma2, alpha, P, K, Nr, d, V0, gammas, switch_iter: int,
                    extrapolate: bool = True):
    """T = len(gammas) iterations of Algorithm 3 with the step of iteration
    t fixed to gammas[t-1] (the same for every cell) and the stage schedule
    fixed: stage I before iteration switch_iter, stage II from it on (the
    unrolled network of the differentiable variant; every other step as in
    ammmse_iteration); switch_iter < 1 keeps stage I throughout.  Returns
    (V^T, WSR(V^T) in bits)."""
    st = AState(V=V0.copy(), Vprev=V0.copy())
    sw = switch_iter if switch_iter >= 1 else len(gammas) + 1
    for g in gammas:
        opt = Options(step_rule=2, gamma_c=float(g), switch_iter=sw, extrapolate=extrapolate)
        ammmse_iteration(H, sigma2, alpha, P, K, Nr, d, st, opt)
    return st.V, m.wsr_bits(H, st.V, sigma2, alpha, K, Nr, d)
