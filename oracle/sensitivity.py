"""FP64 oracle, part 4: how much FP32-sized perturbations of its own
arithmetic move a solve's final WSR.

TEST INFRASTRUCTURE ONLY (see ``oracle.model``).  A final WSR of Algorithm 3
after a fixed number of iterations is a property of a trajectory; at high
SNR some trajectories amplify rounding, and the oracle itself, perturbed at
the FP32 level, then ends far from its unperturbed run.  ``fp32_spread``
measures that, so a free-running FP32 solve can be judged against what FP32
arithmetic can reproduce at all.  The perturbations enter through the
explicit hooks of ``solvers.ammmse_iteration``; no module state is changed.
"""
from __future__ import annotations

import numpy as np

from . import model as m
from . import solvers as s


def _round_c64(T):
    return T.astype(np.complex64).astype(np.complex128)


def perturbed_wsr_bits(inst, iters, cov32=False, v32=False, step_rel=0.0, opt=None):
    """Final WSR (bits) of Algorithm 3 (options ``opt``, default the
    paper's) from the projected V^0, with the receive covariance of eq. (9)
    rounded to complex64 (cov32), the iterate rounded to complex64 after
    every iteration (v32) and the spectral step of eq. (16) scaled by
    1 + step_rel.  With no perturbation this is the plain oracle solve."""
    cov_hook = _round_c64 if cov32 else None
    step_hook = (lambda g: g * (1.0 + step_rel)) if step_rel else None
    opt = opt or s.Options()
    V0 = s.initial_precoder(inst.G0, inst.P)
    st = s.AState(V=V0.copy(), Vprev=V0.copy())
    for _ in range(iters):
        s.ammmse_iteration(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, st, opt,
                           cov_hook=cov_hook, step_hook=step_hook)
        if v32:
            st.V = _round_c64(st.V)
    return m.wsr_bits(inst.H, st.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


# the perturbations fp32_spread applies: (cov32, v32, step_rel)
VARIANTS = ((True, False, 0.0), (False, True, 0.0), (False, False, -5e-7), (True, True, 5e-7))


def fp32_wsr_samples(inst, iters, opt=None):
    """The final WSR (bits) under each perturbation of VARIANTS."""
    return [perturbed_wsr_bits(inst, iters, *v, opt=opt) for v in VARIANTS]


def fp32_spread(inst, iters, reference=None, opt=None):
    """Largest relative change of the final WSR (Algorithm 3, default
    options, ``iters`` iterations) under four FP32-sized perturbations: the
    N_r x N_r receive covariance of eq. (9) stored in complex64; the iterate V
    stored in complex64 after every iteration; the spectral step of eq. (16)
    off by -5e-7 relative (the accuracy of an FP32 Lanczos estimate); and the
    first two with a +5e-7 step error together.  Single perturbations can
    cancel by chance on a sensitive instance, hence the maximum.
    ``reference``: the unperturbed final WSR in bits, if already known;
    ``opt``: the options of the solve (e.g. a forced switch iteration)."""
    ref = perturbed_wsr_bits(inst, iters, opt=opt) if reference is None else reference
    return max(abs(w - ref) / ref for w in fp32_wsr_samples(inst, iters, opt=opt))
