"""FP64 oracle, part 4: how much perturbations of the size of FP32
arithmetic move a solve's final WSR.

TEST INFRASTRUCTURE ONLY (see ``oracle.model``).  A final WSR of Algorithm 3
after a fixed number of iterations is a property of a trajectory; at high
SNR some trajectories amplify rounding, and the oracle itself, perturbed at
the FP32 level, then ends far from its unperturbed run.  ``fp32_spread``
measures that, so a free-running FP32 solve can be judged against what
arithmetic with FP32-level error per step can reproduce at all.  The
perturbations enter through the explicit hooks of
``solvers.ammmse_iteration`` and of ``perturbed_wsr_bits``; no module state
is changed.
"""
from __future__ import annotations

import numpy as np

from . import model as m
from . import solvers as s

# Relative size of the random per-iteration perturbation of the iterate in
# the spread ensemble: the per-step error of the GPU iteration measured by
# the teacher-forced tests on the timed and seven-cell workloads (1e-7 to
# 1e-6 relative; the bound those tests enforce is 1e-5).
STEP_NOISE = 5e-7
N_NOISE = 8


def _round_c64(T):
    return T.astype(np.complex64).astype(np.complex128)


def perturbed_wsr_bits(inst, iters, cov32=False, v32=False, step_rel=0.0, opt=None, v_noise=0.0, seed=0):
    """Final WSR (bits) of Algorithm 3 (options ``opt``, default the
    paper's) from the projected V^0, with the receive covariance of eq. (9)
    rounded to complex64 (cov32), the iterate rounded to complex64 after
    every iteration (v32), the spectral step of eq. (16) scaled by
    1 + step_rel, and the iterate multiplied after every iteration by
    1 + v_noise * xi, xi complex standard normal per entry drawn from a PCG64
    generator seeded with ``seed``.  With no perturbation this is the plain
    oracle solve."""
    cov_hook = _round_c64 if cov32 else None
    step_hook = (lambda g: g * (1.0 + step_rel)) if step_rel else None
    opt = opt or s.Options()
    rng = np.random.default_rng(seed) if v_noise else None
    V0 = s.initial_precoder(inst.G0, inst.P)
    st = s.AState(V=V0.copy(), Vprev=V0.copy())
    for _ in range(iters):
        s.ammmse_iteration(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, st, opt,
                           cov_hook=cov_hook, step_hook=step_hook)
        if v32:
            st.V = _round_c64(st.V)
        if v_noise:
            xi = (rng.standard_normal(st.V.shape) + 1j * rng.standard_normal(st.V.shape)) / np.sqrt(2.0)
            st.V = st.V * (1.0 + v_noise * xi)
    return m.wsr_bits(inst.H, st.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


# the perturbations fp32_spread applies, keyword arguments of perturbed_wsr_bits:
# first the per-step noise of the measured size, then the FP32 roundings
VARIANTS = tuple(dict(v_noise=STEP_NOISE, seed=k + 1) for k in range(N_NOISE)) + (
    dict(cov32=True), dict(v32=True), dict(step_rel=-5e-7), dict(cov32=True, v32=True, step_rel=5e-7))


def fp32_wsr_samples(inst, iters, opt=None):
    """The final WSR (bits) under each perturbation of VARIANTS."""
    return [perturbed_wsr_bits(inst, iters, opt=opt, **v) for v in VARIANTS]


def fp32_spread(inst, iters, reference=None, opt=None, stop_at=None):
    """Largest relative change of the final WSR (Algorithm 3, ``iters``
    iterations, options ``opt``) over the perturbations of VARIANTS: eight
    runs whose iterate takes random relative errors of STEP_NOISE after every
    iteration (the per-step error of the FP32 GPU iteration), the N_r x N_r
    receive covariance of eq. (9) stored in complex64, the iterate stored in
    complex64, the spectral step of eq. (16) off by -5e-7 relative, and the
    last two with a +5e-7 step error together.  ``reference``: the
    unperturbed final WSR in bits, if already known.  ``stop_at``: stop as
    soon as the spread reaches this value (the result is then a lower bound
    that already reaches it)."""
    ref = perturbed_wsr_bits(inst, iters, opt=opt) if reference is None else reference
    spread = 0.0
    for v in VARIANTS:
        spread = max(spread, abs(perturbed_wsr_bits(inst, iters, opt=opt, **v) - ref) / ref)
        if stop_at is not None and spread >= stop_at:
            break
    return spread
