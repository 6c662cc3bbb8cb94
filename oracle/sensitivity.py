"""FP64 oracle, part 4: how much FP32-sized perturbations of its own
arithmetic move a solve's final WSR.

TEST INFRASTRUCTURE ONLY (see ``oracle.model``).  A final WSR of Algorithm 3
after a fixed number of iterations is a property of a trajectory; at high
SNR some trajectories amplify rounding, and the oracle itself, perturbed at
the FP32 level, then ends far from its unperturbed run.  ``fp32_spread``
measures that, so a free-running FP32 solve can be judged against what FP32
arithmetic can reproduce at all.
"""
from __future__ import annotations

import numpy as np

from . import model as m
from . import solvers as s


def _perturbed_wsr_bits(inst, iters, cov32, v32, step_rel):
    exact_cov, exact_step = m.receive_covariance, m.spectral_step
    if cov32:
        m.receive_covariance = lambda *a: exact_cov(*a).astype(np.complex64).astype(np.complex128)
    if step_rel:
        m.spectral_step = lambda *a: exact_step(*a) * (1.0 + step_rel)
    try:
        V0 = s.initial_precoder(inst.G0, inst.P)
        st = s.AState(V=V0.copy(), Vprev=V0.copy())
        for _ in range(iters):
            s.ammmse_iteration(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, st, s.Options())
            if v32:
                st.V = st.V.astype(np.complex64).astype(np.complex128)
        return m.wsr_bits(inst.H, st.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)
    finally:
        m.receive_covariance, m.spectral_step = exact_cov, exact_step


def fp32_spread(inst, iters, reference=None):
    """Largest relative change of the final WSR (Algorithm 3, default
    options, ``iters`` iterations) under four FP32-sized perturbations: the
    N_r x N_r receive covariance of eq. (9) stored in complex64; the iterate V
    stored in complex64 after every iteration; the spectral step of eq. (16)
    off by -5e-7 relative (the accuracy of an FP32 Lanczos estimate); and the
    first two with a +5e-7 step error together.  Single perturbations can
    cancel by chance on a sensitive instance, hence the maximum.
    ``reference``: the unperturbed final WSR in bits, if already known."""
    if reference is None:
        V0 = s.initial_precoder(inst.G0, inst.P)
        ref = m.wsr_bits(inst.H, s.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0,
                                          iters).V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)
    else:
        ref = reference
    variants = [(True, False, 0.0), (False, True, 0.0), (False, False, -5e-7), (True, True, 5e-7)]
    return max(abs(_perturbed_wsr_bits(inst, iters, *v) - ref) / ref for v in variants)
