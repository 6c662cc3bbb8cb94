"""Checks that pin the FP64 oracle to the paper and to the mathematics.

Each check raises AssertionError on failure.  They are written against
``oracle.model`` / ``oracle.solvers`` attributes looked up at call time, so
``test_oracle_mutations`` can plant a mistake in the oracle and show that some
check here catches it.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as wl
from oracle import closed_forms as cf
from oracle import model as m
from oracle import solvers as s


def _inst(seed, C, K, Nt, Nr, d, **kw):
    return wl.random_small(np.random.default_rng(seed), C, K, Nt, Nr, d, **kw)


def _V0(inst):
    return s.initial_precoder(inst.G0, inst.P)


def _args(inst):
    return inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d


# ---------------------------------------------------------------- rates
def pin_rate_scalar_sinr(seed=11):
    """Nr = d = 1: the rate is log(1 + SINR) with scalar powers (Sec. II)."""
    inst = _inst(seed, 2, 3, 4, 1, 1)
    V = _V0(inst)
    C, K = inst.C, inst.K
    for r in range(C * K):
        k = r // K
        h = lambda j: inst.H[j, r, :]                 # noqa: E731
        v = lambda rr: V[rr // K][:, rr % K]          # noqa: E731
        sig = abs(h(k) @ v(r)) ** 2
        intf = sum(abs(h(rr // K) @ v(rr)) ** 2 for rr in range(C * K) if rr != r)
        want = math.log(1.0 + sig / (intf + inst.sigma2[r]))
        got = m.rate(inst.H, V, inst.sigma2, r, K, 1, 1)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (r, got, want)


def pin_rate_det_ratio(seed=12):
    """R = log det(T) - log det(T - S), T the full receive covariance and S
    the own-signal term: the same rate through det(A+B)/det(B)."""
    inst = _inst(seed, 2, 2, 5, 2, 2)
    V = _V0(inst)
    C, K, Nr, d = inst.C, inst.K, inst.Nr, inst.d
    for r in range(C * K):
        T = inst.sigma2[r] * np.eye(Nr, dtype=complex)
        for rr in range(C * K):
            Z = inst.H[rr // K, r * Nr:(r + 1) * Nr] @ V[rr // K][:, (rr % K) * d:(rr % K + 1) * d]
            T += Z @ Z.conj().T
            if rr == r:
                S = Z @ Z.conj().T
        want = np.linalg.slogdet(T)[1] - np.linalg.slogdet(T - S)[1]
        got = m.rate(inst.H, V, inst.sigma2, r, K, Nr, d)
        assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (r, got, want)


def pin_wsr_equivalence(seed=13):
    """At U = MMSE(V) and W = E^{-1}: f(U, W, V) = sum alpha d - WSR(V)
    (the WMMSE / WSR equivalence the paper relies on, Sec. IV)."""
    for C, K, Nt, Nr, d in [(1, 3, 4, 2, 2), (2, 2, 5, 3, 2), (3, 2, 4, 2, 1)]:
        inst = _inst(seed + C, C, K, Nt, Nr, d)
        V = _V0(inst)
        U = m.mmse_receiver(inst.H, V, inst.sigma2, K, Nr, d)
        W = m.mse_weight(inst.H, U, V, K, Nr, d)
        f = m.objective(inst.H, U, W, V, inst.sigma2, inst.alpha, K, Nr, d)
        R = m.wsr(inst.H, V, inst.sigma2, inst.alpha, K, Nr, d)
        want = float(np.sum(inst.alpha)) * d - R
        assert abs(f - want) <= 1e-10 * max(1.0, abs(want)), (f, want)


# ------------------------------------------------------- closed-form optima
def pin_single_user_capacity(n_seeds=8, iters=1500):
    """C = K = 1: WMMSE (exact bisection) and A-MMMSE both reach the
    water-filling capacity over the d largest singular values."""
    for seed in range(n_seeds):
        inst = _inst(100 + seed, 1, 1, 8, 2, 2, P=10.0)
        inst.P[:] = 10.0
        inst.sigma2[:] = 1.0
        inst.alpha[:] = 1.0
        cap = cf.single_user_capacity(inst.H[0], 10.0, 1.0, 2)
        V0 = _V0(inst)
        Vw, hist, _ = s.wmmse(*_args(inst), V0, 200, exact=True)
        assert abs(hist[-1] - cap) <= 1e-6 * cap, ("wmmse", seed, hist[-1], cap)
        res = s.ammmse(*_args(inst), V0, iters)
        R = m.wsr(inst.H, res.V, inst.sigma2, inst.alpha, 1, 2, 2)
        assert abs(R - cap) <= 1e-6 * cap, ("ammmse", seed, R, cap)


def pin_miso_mrt(seed=21, iters=1000):
    """Nr = d = 1, one user: the optimum is maximum-ratio transmission with
    rate log(1 + P ||h||^2 / sigma2)."""
    inst = _inst(seed, 1, 1, 6, 1, 1)
    want = cf.miso_mrt_rate(inst.H[0, 0], inst.P[0], inst.sigma2[0])
    res = s.ammmse(*_args(inst), _V0(inst), iters)
    R = m.rate(inst.H, res.V, inst.sigma2, 0, 1, 1, 1)
    assert abs(R - want) <= 1e-8 * want, (R, want)


def pin_orthogonal_users(seed=22, iters=3000):
    """Users on disjoint antenna subsets (no interference), alpha = 1: the
    optimum is water-filling over the union of all users' singular values."""
    rng = np.random.default_rng(seed)
    inst = wl.rayleigh_instance(rng, 1, 2, 4, 2, 2, P=10.0)
    inst.H[0, 0:2, 2:4] = 0.0
    inst.H[0, 2:4, 0:2] = 0.0
    gains = np.concatenate([np.linalg.svd(inst.H[0, 2 * r:2 * r + 2], compute_uv=False) ** 2
                            for r in range(2)])
    want = cf.capacity_nats(gains, 10.0, 1.0)
    V0 = _V0(inst)
    _, hist, _ = s.wmmse(*_args(inst), V0, 400, exact=True)
    assert abs(hist[-1] - want) <= 1e-6 * want, ("wmmse", hist[-1], want)
    res = s.ammmse(*_args(inst), V0, iters)
    R = m.wsr(inst.H, res.V, inst.sigma2, inst.alpha, 2, 2, 2)
    assert abs(R - want) <= 1e-5 * want, ("ammmse", R, want)


# ---------------------------------------------------- block minimisers
def _objective_at(inst, U, W, V):
    return m.objective(inst.H, U, W, V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


def _random_pd(rng, d):
    A = wl.cn01(rng, (d, d))
    return A @ A.conj().T + 0.5 * np.eye(d)


def pin_U_minimizer(seed=31):
    """eq. (9) is the exact minimiser of f over U for any PD W: perturbing U
    never lowers f, and the directional derivatives vanish."""
    rng = np.random.default_rng(seed)
    for C, K, Nt, Nr, d in [(1, 2, 3, 2, 1), (1, 2, 3, 2, 2), (2, 2, 3, 2, 2)]:
        inst = _inst(seed + Nt + d + C, C, K, Nt, Nr, d)
        V = _V0(inst)
        U = m.mmse_receiver(inst.H, V, inst.sigma2, K, Nr, d)
        W = [_random_pd(rng, d) for _ in range(C * K)]
        f0 = _objective_at(inst, U, W, V)
        for _ in range(50):
            D = [wl.cn01(rng, (Nr, d)) for _ in range(C * K)]
            for eps in (1e-2, 1e-4):
                Up = [u + eps * dd for u, dd in zip(U, D)]
                assert _objective_at(inst, Up, W, V) >= f0 - 1e-12 * abs(f0)
            h = 1e-6
            fp = _objective_at(inst, [u + h * dd for u, dd in zip(U, D)], W, V)
            fm = _objective_at(inst, [u - h * dd for u, dd in zip(U, D)], W, V)
            assert abs(fp - fm) / (2 * h) <= 1e-6 * max(1.0, abs(f0))


def pin_W_minimizer(seed=32):
    """eq. (10) is the exact minimiser of f over PD W: Hermitian
    perturbations never lower f."""
    rng = np.random.default_rng(seed)
    inst = _inst(seed, 2, 2, 4, 2, 2)
    V = _V0(inst)
    U = m.mmse_receiver(inst.H, V, inst.sigma2, 2, 2, 2)
    W = m.mse_weight(inst.H, U, V, 2, 2, 2)
    f0 = _objective_at(inst, U, W, V)
    for _ in range(50):
        D = []
        for _ in range(4):
            A = wl.cn01(rng, (2, 2))
            D.append(A + A.conj().T)
        for eps in (1e-2, 1e-4):
            Wp = [w + eps * dd for w, dd in zip(W, D)]
            if all(np.linalg.eigvalsh(w)[0] > 0 for w in Wp):
                assert _objective_at(inst, U, Wp, V) >= f0 - 1e-12 * abs(f0)
    # also a random (non-optimal) U: W = E^{-1} still minimises
    U2 = [u + 0.3 * wl.cn01(rng, u.shape) for u in U]
    E = [m.mse_matrix(inst.H, U2, V, inst.sigma2, r, 2, 2, 2) for r in range(4)]
    W2 = [np.linalg.inv(e) for e in E]
    f2 = _objective_at(inst, U2, W2, V)
    for _ in range(20):
        D = []
        for _ in range(4):
            A = wl.cn01(rng, (2, 2))
            D.append(A + A.conj().T)
        Wp = [w + 1e-3 * dd for w, dd in zip(W2, D)]
        if all(np.linalg.eigvalsh(w)[0] > 0 for w in Wp):
            assert _objective_at(inst, U2, Wp, V) >= f2 - 1e-12 * abs(f2)


def pin_gradient_fd(seed=41):
    """eq. (14) against central finite differences of f over the real and
    imaginary parts (inner product of Def. 1): Df[D] = Re <grad, D>."""
    rng = np.random.default_rng(seed)
    for C, K, Nt, Nr, d in [(1, 2, 3, 2, 2), (2, 2, 4, 2, 1), (3, 1, 3, 2, 2)]:
        inst = _inst(seed + C + K, C, K, Nt, Nr, d)
        V = _V0(inst)
        U = [wl.cn01(rng, (Nr, d)) for _ in range(C * K)]
        W = [_random_pd(rng, d) for _ in range(C * K)]
        G = m.gradient(inst.H, U, W, V, inst.alpha, K, Nr, d)
        for _ in range(6):
            D = wl.cn01(rng, V.shape)
            h = 1e-5
            fd = (_objective_at(inst, U, W, V + h * D) - _objective_at(inst, U, W, V - h * D)) / (2 * h)
            an = float(np.sum((G.conj() * D).real))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (C, fd, an)


def pin_projection(seed=51):
    """eq. (15): identity inside the ball, radial scaling onto its surface
    outside, idempotent."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        V = wl.cn01(rng, (6, 4)) * rng.uniform(0.1, 3.0)
        P = rng.uniform(0.5, 20.0)
        Vp = m.project(V, P)
        pw = float(np.sum(np.abs(V) ** 2))
        pp = float(np.sum(np.abs(Vp) ** 2))
        if pw > P:
            assert abs(pp - P) <= 1e-12 * P
            # radial: Vp is a positive multiple of V
            c = np.vdot(V, Vp).real / pw
            assert np.allclose(Vp, c * V, rtol=0, atol=1e-12) and c > 0
        else:
            assert np.array_equal(Vp, V)
        assert np.allclose(m.project(Vp, P), Vp, rtol=0, atol=1e-13)


# ------------------------------------------------------------ monotonicity
def pin_wmmse_monotone(seed=61, iters=25):
    """BCM on every block (Algorithm 2 with exact bisection) never lowers
    the WSR (Sec. IV)."""
    for C, K, Nt, Nr, d in [(1, 4, 8, 2, 2), (2, 2, 4, 2, 2)]:
        inst = _inst(seed + C, C, K, Nt, Nr, d)
        _, hist, _ = s.wmmse(*_args(inst), _V0(inst), iters, exact=True)
        for a, b in zip(hist, hist[1:]):
            assert b >= a - 1e-9 * abs(a), (a, b)


def pin_ammmse_descent_chain(seed=62, iters=25):
    """Theorem 1 with omega = 0 and gamma = 1/||F_k||_2 at every iteration in
    stage II: f(Z_v^{t-1}) >= f(Z_u^t) >= f(Z_w^t) >= f(Z_v^t), hence the
    WSR never decreases."""
    opt = s.Options(extrapolate=False, step_rule=1, switch_iter=1)
    for C, K, Nt, Nr, d in [(1, 4, 8, 2, 2), (2, 2, 4, 2, 2)]:
        inst = _inst(seed + C, C, K, Nt, Nr, d)
        H, sg, al, P, K_, Nr_, d_ = _args(inst)
        st = s.AState(V=_V0(inst), Vprev=_V0(inst))
        U = m.mmse_receiver(H, st.V, sg, K, Nr, d)
        W = m.mse_weight(H, U, st.V, K, Nr, d)
        f_prev = m.objective(H, U, W, st.V, sg, al, K, Nr, d)
        wsr_prev = m.wsr(H, st.V, sg, al, K, Nr, d)
        for _ in range(iters):
            Vold = st.V
            s.ammmse_iteration(H, sg, al, P, K, Nr, d, st, opt)
            # the iteration used U^t, W^t at Vold; V^t is st.V
            U = m.mmse_receiver(H, Vold, sg, K, Nr, d)
            fu = m.objective(H, U, W, Vold, sg, al, K, Nr, d)
            W = m.mse_weight(H, U, Vold, K, Nr, d)
            fw = m.objective(H, U, W, Vold, sg, al, K, Nr, d)
            fv = m.objective(H, U, W, st.V, sg, al, K, Nr, d)
            tol = 1e-10 * max(1.0, abs(f_prev))
            assert f_prev >= fu - tol and fu >= fw - tol and fw >= fv - tol, (f_prev, fu, fw, fv)
            f_prev = fv
            R = m.wsr(H, st.V, sg, al, K, Nr, d)
            assert R >= wsr_prev - 1e-9 * abs(wsr_prev)
            wsr_prev = R


# ------------------------------------------------------------- lemma bounds
def pin_lemma_bounds(seed=71, iters=15):
    """Lemma 1 (lambda_min(E) bound), Lemma 2 (||U||_F^2 <= d/sigma^2 and
    lambda_max(W) bound) and Lemma 3 (||F_k||_2 <= 2 alpha_max (C K) kappa /
    sigma^2_min, kappa over every link) along an A-MMMSE run."""
    for C, K, Nt, Nr, d in [(1, 4, 8, 2, 2), (2, 3, 4, 2, 2)]:
        inst = _inst(seed + C, C, K, Nt, Nr, d)
        H, sg, al, P, K_, Nr_, d_ = _args(inst)
        kap_direct = max(np.linalg.norm(m.link(H, r, r // K, Nr), 2) ** 2 for r in range(C * K))
        kap_all = max(np.linalg.norm(m.link(H, r, j, Nr), 2) ** 2
                      for r in range(C * K) for j in range(C))
        Pmax = float(np.max(P))
        st = s.AState(V=_V0(inst), Vprev=_V0(inst))
        for _ in range(iters):
            U = m.mmse_receiver(H, st.V, sg, K, Nr, d)
            W = m.mse_weight(H, U, st.V, K, Nr, d)
            for r in range(C * K):
                E = m.mse_matrix(H, U, st.V, sg, r, K, Nr, d)
                lo = sg[r] / (Pmax * kap_direct + sg[r])
                assert np.linalg.eigvalsh(E)[0] >= lo * (1 - 1e-12)
                assert np.sum(np.abs(U[r]) ** 2) <= d / sg[r] * (1 + 1e-12)
                assert np.linalg.eigvalsh(W[r])[-1] <= (Pmax * kap_direct + sg[r]) / sg[r] * (1 + 1e-12)
            for k in range(C):
                F = m.F_matrix(H, U, W, al, k, K, Nr)
                bound = 2 * np.max(al) * C * K * kap_all / np.min(sg)
                assert np.linalg.eigvalsh(F)[-1] <= bound * (1 + 1e-12)
            s.ammmse_iteration(H, sg, al, P, K, Nr, d, st, s.Options())


# ----------------------------------------------------------------- bisection
def pin_bisection_slackness(seed=81):
    """eq. (12) with exact bisection: lambda > 0 implies the cell's power
    budget is met with equality (complementary slackness); lambda = 0
    implies it is met."""
    for C, K, Nt, Nr, d, P in [(1, 4, 8, 2, 2, 10.0), (1, 4, 6, 2, 2, 1e4), (2, 2, 4, 2, 1, 5.0)]:
        inst = _inst(seed + Nt, C, K, Nt, Nr, d, P=P)
        V = _V0(inst)
        U = m.mmse_receiver(inst.H, V, inst.sigma2, K, Nr, d)
        W = m.mse_weight(inst.H, U, V, K, Nr, d)
        for k in range(C):
            Vk, lam = s.wmmse_precoder_cell(inst.H, U, W, inst.alpha, inst.P, k, K, Nr, d, exact=True)
            pw = float(np.sum(np.abs(Vk) ** 2))
            if lam > 0:
                assert abs(pw - inst.P[k]) <= 1e-9 * inst.P[k], (pw, inst.P[k])
            else:
                assert pw <= inst.P[k] * (1 + 1e-12)


# --------------------------------------------------------------- invariances
def pin_scale_invariance(seed=91, iters=20):
    """(c H, c^2 sigma^2) gives the same iterates and WSR: the whole method
    sees H only through H V V^H H^H / sigma^2."""
    inst = _inst(seed, 2, 2, 4, 2, 2)
    V0 = _V0(inst)
    a = s.ammmse(*_args(inst), V0, iters)
    c = 1e-5
    b = s.ammmse(c * inst.H, c * c * inst.sigma2, inst.alpha, inst.P, 2, 2, 2, V0, iters)
    assert np.allclose(a.V, b.V, rtol=0, atol=1e-8 * np.max(np.abs(a.V)))
    for ha, hb in zip(a.history, b.history):
        assert abs(ha.rho - hb.rho) <= 1e-9 * abs(ha.rho)


def pin_unitary_invariance(seed=92, iters=20):
    """H_j -> H_j Q_j and V0_j -> Q_j^H V0_j (Q_j unitary) gives V_j -> Q_j^H V_j
    with the same WSR; relabelling users permutes the outputs."""
    inst = _inst(seed, 2, 2, 4, 2, 2)
    V0 = _V0(inst)
    rng = np.random.default_rng(seed)
    Q = [np.linalg.qr(wl.cn01(rng, (4, 4)))[0] for _ in range(2)]
    H2 = np.stack([inst.H[j] @ Q[j] for j in range(2)])
    V02 = np.stack([Q[j].conj().T @ V0[j] for j in range(2)])
    a = s.ammmse(*_args(inst), V0, iters)
    b = s.ammmse(H2, inst.sigma2, inst.alpha, inst.P, 2, 2, 2, V02, iters)
    for j in range(2):
        assert np.allclose(b.V[j], Q[j].conj().T @ a.V[j], rtol=0, atol=1e-9)
    # swap the two users of cell 0 (and of every H block's rows)
    perm = [1, 0, 2, 3]
    Nr, d = 2, 2
    rows = np.concatenate([np.arange(p * Nr, (p + 1) * Nr) for p in perm])
    H3 = inst.H[:, rows, :]
    V03 = V0.copy()
    V03[0] = V0[0][:, np.r_[2:4, 0:2]]
    c = s.ammmse(H3, inst.sigma2[perm], inst.alpha[perm], inst.P, 2, 2, 2, V03, iters)
    assert np.allclose(c.V[0], a.V[0][:, np.r_[2:4, 0:2]], rtol=0, atol=1e-9)
    assert np.allclose(c.V[1], a.V[1], rtol=0, atol=1e-9)


def pin_omega_and_defaults():
    """omega^t of eq. (18) and the hyper-parameters printed in the paper,
    read from tests/golden/paper_constants.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    vals = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=")
            num, _, den = v.strip().partition("/")
            vals[k.strip()] = float(num) / float(den) if den else float(num)
    opt = s.Options()
    assert opt.Tc == vals["Tc"] and opt.eps1 == vals["eps1"] and opt.eps2 == vals["eps2"]
    for t in range(1, 9):
        assert abs(m.extrapolation_weight(t) - vals[f"omega_{t}"]) <= 1e-15


def pin_spectral_step_factor(seed=93):
    """eq. (16): gamma = 1/||F_k||_2.  F_k = A^H A with A stacking
    sqrt(2 alpha) W^{1/2} U^H H_{r k} over every user r, so ||F_k||_2 is the
    squared largest singular value of A (a different matrix and routine)."""
    rng = np.random.default_rng(seed)
    for C, K, Nt, Nr, d in [(1, 3, 5, 2, 2), (2, 2, 4, 2, 1)]:
        inst = _inst(seed + C, C, K, Nt, Nr, d)
        U = [wl.cn01(rng, (Nr, d)) for _ in range(C * K)]
        W = [_random_pd(rng, d) for _ in range(C * K)]
        for k in range(C):
            blocks = []
            for r in range(C * K):
                ev, Q = np.linalg.eigh(W[r])
                Wh = Q @ np.diag(np.sqrt(ev)) @ Q.conj().T
                blocks.append(np.sqrt(2 * inst.alpha[r]) * Wh @ U[r].conj().T @ m.link(inst.H, r, k, Nr))
            smax = np.linalg.svd(np.vstack(blocks), compute_uv=False)[0]
            g = m.spectral_step(inst.H, U, W, inst.alpha, k, K, Nr)
            assert abs(g * smax ** 2 - 1.0) <= 1e-12, (g, smax)


ALL_PINS = [pin_spectral_step_factor, pin_rate_scalar_sinr, pin_rate_det_ratio, pin_wsr_equivalence,
            pin_single_user_capacity, pin_miso_mrt, pin_orthogonal_users,
            pin_U_minimizer, pin_W_minimizer, pin_gradient_fd, pin_projection,
            pin_wmmse_monotone, pin_ammmse_descent_chain, pin_lemma_bounds,
            pin_bisection_slackness, pin_scale_invariance, pin_unitary_invariance,
            pin_omega_and_defaults]


def pin_wmmse_ammmse_agree(n=100, iters=200):
    """WMMSE and A-MMMSE reach almost the same WSR (Sec. VII-C): on the
    tiny single-cell workload the mean final WSR agrees within 1e-3
    relative, and WMMSE with exact bisection ends at a stationary point
    (projected-gradient residual below 1e-5 on each instance)."""
    A, W = [], []
    for inst in wl.tiny_fp64(n):
        V0 = _V0(inst)
        a = s.ammmse(*_args(inst), V0, iters)
        A.append(m.wsr(inst.H, a.V, inst.sigma2, inst.alpha, 4, 2, 2))
        _, hist, _ = s.wmmse(*_args(inst), V0, iters)
        W.append(hist[-1])
    A, W = np.array(A), np.array(W)
    gap = abs(A.mean() - W.mean()) / W.mean()
    assert gap <= 1e-3, gap
    for inst in wl.tiny_fp64(4):
        V, _, _ = s.wmmse(*_args(inst), _V0(inst), 300, exact=True)
        U = m.mmse_receiver(inst.H, V, inst.sigma2, 4, 2, 2)
        Wt = m.mse_weight(inst.H, U, V, 4, 2, 2)
        G = m.gradient(inst.H, U, Wt, V, inst.alpha, 4, 2, 2)
        g = m.spectral_step(inst.H, U, Wt, inst.alpha, 0, 4, 2)
        res = np.linalg.norm(V[0] - m.project(V[0] - g * G[0], inst.P[0])) / np.linalg.norm(V[0])
        assert res <= 1e-5, res


# ------------------------------------------------- Algorithm 3 control flow
def _stage1_wsr_sequence(inst, iters):
    """WSR(V^t), t = 0..iters, of a run held in stage I (W = I throughout),
    from the rate definition: R^t of iteration t is entry t - 1."""
    H, sg, al, P, K, Nr, d = _args(inst)
    V0 = _V0(inst)
    pure = s.ammmse(*_args(inst), V0, iters, s.Options(switch_iter=10 ** 9))
    return pure, [m.wsr(H, V, sg, al, K, Nr, d) for V in [V0] + [h.V for h in pure.history]]


def pin_stage_switch_rule(seed=507, iters=14):
    """Stage test of Algorithm 3: the scheme leaves stage I at the first
    iteration t >= 2 whose relative WSR change |R^t - R^{t-1}| / R^{t-1} is at
    most eps1 (R^t = WSR(V^{t-1})), and stays in stage II afterwards.  Checked
    against WSR values computed from the iterates of a run held in stage I,
    and against a run whose switch is forced at that iteration (identical
    iterates).  On this instance the paper's eps1 = 0.1 switches at t = 6 and
    the first stage-II iterate then raises the WSR by about 13 %, more than
    eps1, so a switch that is re-tested every iteration would fall back."""
    inst = _inst(seed, 1, 3, 4, 2, 2)
    V0 = _V0(inst)
    pure, R = _stage1_wsr_sequence(inst, iters)
    for eps1, want in ((0.1, 6), (0.2, 5), (1e9, 2), (0.0, None)):
        first = next((t for t in range(2, iters + 1) if abs(R[t - 1] - R[t - 2]) <= eps1 * abs(R[t - 2])), None)
        assert first == want, (eps1, first, want)  # this instance's trajectory, read off by hand
        run = s.ammmse(*_args(inst), V0, iters, s.Options(eps1=eps1))
        stages = [h.stage for h in run.history]
        if want is None:
            assert stages == [1] * iters, (eps1, stages)
            forced = pure
        else:
            assert stages == [1] * (want - 1) + [2] * (iters - want + 1), (eps1, stages)
            forced = s.ammmse(*_args(inst), V0, iters, s.Options(switch_iter=want))
        for a, b in zip(run.history, forced.history):
            assert np.array_equal(a.V, b.V), eps1
    # the latch has something to hold here: a stage-II change beyond eps1 = 0.1
    run = s.ammmse(*_args(inst), V0, iters, s.Options())
    rho = [h.rho for h in run.history]
    assert max(abs(b - a) / a for a, b in zip(rho[5:], rho[6:])) > 0.1


def pin_step_size_schedule(seed=507, iters=14):
    """eq. (16) with the per-stage reading: gamma = 1/||F_k||_2 in the first
    Tc = 3 iterations of each stage, then the last of those values (gamma_c)
    until the stage ends.  With the switch forced at t = 6 the schedule is
    spectral at t = 1, 2, 3 and 6, 7, 8, frozen at gamma^3 for t = 4, 5 and at
    gamma^8 from t = 9 on.  The spectral values are recomputed from each
    iteration's U (eq. (9) at V^{t-1}) and W; the recorded steps are then
    shown to be the ones the iterates took, by replaying them through the
    fixed-step unrolled form."""
    inst = _inst(seed, 1, 3, 4, 2, 2)
    H, sg, al, P, K, Nr, d = _args(inst)
    V0 = _V0(inst)
    run = s.ammmse(*_args(inst), V0, iters, s.Options(switch_iter=6))
    kinds = "sssffsssffffff"
    freeze_src = {4: 3, 5: 3, 9: 8, 10: 8, 11: 8, 12: 8, 13: 8, 14: 8}
    Vs = [V0] + [h.V for h in run.history]
    for t, h in enumerate(run.history, 1):
        assert h.stage == (2 if t >= 6 else 1)
        if kinds[t - 1] == "s":
            U = m.mmse_receiver(H, Vs[t - 1], sg, K, Nr, d)
            W = m.mse_weight(H, U, Vs[t - 1], K, Nr, d) if h.stage == 2 else m.identity_weights(1, K, d)
            want = m.spectral_step(H, U, W, al, 0, K, Nr)
        else:
            want = run.history[freeze_src[t] - 1].gamma[0]
        assert abs(h.gamma[0] - want) <= 1e-12 * want, (t, h.gamma[0], want)
    # stage II's frozen step differs from stage I's (W = E^{-1} changes ||F||)
    assert abs(run.history[8].gamma[0] - run.history[3].gamma[0]) > 1e-3 * run.history[3].gamma[0]
    Vu, _ = s.ammmse_unrolled(*_args(inst), V0, [h.gamma[0] for h in run.history], switch_iter=6)
    assert np.allclose(Vu, run.V, rtol=0, atol=1e-12)


def pin_tolerance_stop(seed=507, iters=60):
    """The stopping test of Algorithm 3: the solve ends at the start of the
    first iteration t that follows a stage-II iteration and sees
    |R^t - R^{t-1}| <= eps2 R^{t-1}; the result is V^{t-1}.  With eps1 = 0.01
    (a late switch, at t = 10) and eps2 = 0.05 the stage-I changes drop below
    eps2 from t = 8 on, where no stop may happen yet."""
    inst = _inst(seed, 1, 3, 4, 2, 2)
    H, sg, al, P, K, Nr, d = _args(inst)
    V0 = _V0(inst)
    opt = s.Options(eps1=0.01, eps2=0.05)
    full = s.ammmse(*_args(inst), V0, iters, opt)
    Vs = [V0] + [h.V for h in full.history]
    R = [m.wsr(H, V, sg, al, K, Nr, d) for V in Vs]
    stages = [h.stage for h in full.history]
    assert stages.index(2) + 1 == 10
    assert abs(R[7] - R[6]) <= 0.05 * R[6]                # t = 8, still stage I: no stop
    want = next(t for t in range(2, iters + 1)
                if stages[t - 2] == 2 and abs(R[t - 1] - R[t - 2]) <= 0.05 * abs(R[t - 2]))
    tol = s.ammmse(*_args(inst), V0, iters, opt, tolerance_stop=True)
    assert tol.converged and tol.iters == want - 1, (tol.iters, want)
    assert np.array_equal(tol.V, Vs[want - 1])
    # not converged within a budget that ends before that iteration
    short = s.ammmse(*_args(inst), V0, want - 2, opt, tolerance_stop=True)
    assert not short.converged and short.iters == want - 2


def _feasible_perturbations(rng, V, P, n):
    for _ in range(n):
        D = wl.cn01(rng, V.shape)
        for eps in (1e-2, 1e-4):
            yield np.stack([m.project(V[k] + eps * D[k], P[k]) for k in range(V.shape[0])])


def pin_V_minimizer(seed=94):
    """eq. (12) (and eq. (20), its W = I case) with exact bisection gives the
    minimiser of f(U, W, .) over the per-cell power balls: f separates over
    the cells' precoders, so no feasible perturbation of any cell's block
    lowers f, whether the power constraint is active (lambda > 0) or not."""
    rng = np.random.default_rng(seed)
    seen_active = seen_inactive = False
    for C, K, Nt, Nr, d, P, W_identity in [(1, 3, 5, 2, 2, 10.0, False), (2, 2, 4, 2, 1, 5.0, False),
                                           (1, 3, 5, 2, 2, 10.0, True), (1, 3, 4, 2, 2, 1e4, False)]:
        inst = _inst(seed + C + K + Nt, C, K, Nt, Nr, d, P=P)
        V = _V0(inst)
        U = m.mmse_receiver(inst.H, V, inst.sigma2, K, Nr, d)
        W = m.identity_weights(C, K, d) if W_identity else m.mse_weight(inst.H, U, V, K, Nr, d)
        res = [s.wmmse_precoder_cell(inst.H, U, W, inst.alpha, inst.P, k, K, Nr, d, exact=True) for k in range(C)]
        Vs = np.stack([r[0] for r in res])
        seen_active |= any(r[1] > 0 for r in res)
        seen_inactive |= any(r[1] == 0 for r in res)
        for k in range(C):  # feasible: an infeasible point could undercut every feasible one
            assert float(np.sum(np.abs(Vs[k]) ** 2)) <= inst.P[k] * (1 + 1e-9), (C, K, k)
        f0 = _objective_at(inst, U, W, Vs)
        for Vp in _feasible_perturbations(rng, Vs, inst.P, 30):
            assert _objective_at(inst, U, W, Vp) >= f0 - 1e-10 * max(1.0, abs(f0)), (C, K, W_identity)
    assert seen_active and seen_inactive


def pin_mmmse_first_stage(seed=95, iters=8):
    """The MMMSE baseline (Algorithm 2 with the mixed warm start): in stage
    I it is block-coordinate minimisation of the weighted sum-MSE (6) over
    U (eq. (9)) and V (eq. (20)), so the sum-MSE at (U(V^t), V^t) never
    increases; with eps1 huge the switch comes at the first test (iteration
    2), after which the iterates are those of WMMSE started from MMMSE's
    first iterate."""
    inst = _inst(seed, 1, 3, 6, 2, 2)
    H, sg, al, P, K, Nr, d = _args(inst)
    V0 = _V0(inst)
    prev = None
    for t in range(1, iters + 1):
        Vt, _, _ = s.wmmse(*_args(inst), V0, t, exact=True, mmse_first_stage=True, eps1=0.0)
        U = m.mmse_receiver(H, Vt, sg, K, Nr, d)
        f = m.sum_mse(H, U, Vt, sg, al, K, Nr, d)
        if prev is not None:
            assert f <= prev + 1e-10 * abs(prev), (t, f, prev)
        prev = f
    V1, _, _ = s.wmmse(*_args(inst), V0, 1, exact=True, mmse_first_stage=True, eps1=1e9)
    Va, ha, _ = s.wmmse(*_args(inst), V0, iters, exact=True, mmse_first_stage=True, eps1=1e9)
    Vb, hb, _ = s.wmmse(*_args(inst), V1, iters - 1, exact=True)
    assert np.allclose(Va, Vb, rtol=0, atol=1e-12)
    assert np.allclose(ha[1:], hb, rtol=1e-13, atol=0)
    # the first MMSE iterate differs from a WMMSE step (the stage-I update is a different one)
    Vw, _, _ = s.wmmse(*_args(inst), V0, 1, exact=True)
    assert np.linalg.norm(V1 - Vw) > 1e-6 * np.linalg.norm(Vw)


ALL_PINS += [pin_stage_switch_rule, pin_step_size_schedule, pin_tolerance_stop, pin_V_minimizer,
             pin_mmmse_first_stage]
