"""The rule free-running GPU solves are judged by (oracle.parity) and the
FP32-sensitivity measure it uses (oracle.sensitivity), on the CPU."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as wl
from oracle import model as m
from oracle import parity as op
from oracle import sensitivity as sens
from oracle import solvers as s


def _inst(seed, C, K, Nt, Nr, d):
    return wl.random_small(np.random.default_rng(seed), C, K, Nt, Nr, d)


def _solve_bits(inst, iters, **opt):
    V0 = s.initial_precoder(inst.G0, inst.P)
    r = s.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, iters, s.Options(**opt))
    return m.wsr_bits(inst.H, r.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


def test_unambiguous_instance_has_one_reference():
    inst = _inst(507, 1, 3, 4, 2, 2)
    ref = op.reference_solves(inst, 14)
    assert ref.switch == [6] and ref.margin > op.SWITCH_MARGIN
    assert ref.wsr == [_solve_bits(inst, 14)]


def test_ambiguous_switch_gets_each_admissible_trajectory():
    """eps1 set 5e-5 above the relative change of the stage test at t = 6
    (a decision within the margin): switching at 6 and, the test going the
    other way, at 7 (the next test, unambiguously below eps1) are both
    admissible; each reference is the forced-switch solve."""
    inst = _inst(507, 1, 3, 4, 2, 2)
    V0 = s.initial_precoder(inst.G0, inst.P)
    r = s.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, 14,
                 s.Options(switch_iter=10 ** 9))
    c6 = m.relative_change(r.history[5].rho, r.history[4].rho)
    opt = s.Options(eps1=c6 + 5e-5)
    ref = op.reference_solves(inst, 14, opt)
    assert ref.switch == [6, 7] and ref.margin < op.SWITCH_MARGIN
    assert ref.wsr[0] == _solve_bits(inst, 14, eps1=c6 + 5e-5)
    assert ref.wsr[1] == _solve_bits(inst, 14, eps1=c6 + 5e-5, switch_iter=7)
    assert abs(ref.wsr[0] - ref.wsr[1]) > 1e-6 * ref.wsr[0]  # genuinely different trajectories
    # a result on the second trajectory is judged against it
    v = op.judge(ref.wsr[1] * (1 + 2e-4), ref, inst, 14, opt)
    assert v.ok and v.which == 1 and abs(v.gap - 2e-4) < 1e-9


def test_judge_rule():
    ref = op.Reference([10.0], [5], 1.0)
    assert op.judge(10.0 * (1 + 9e-4), ref).ok
    v = op.judge(10.0 * (1 - 3e-3), ref, spread=1e-3)       # 3x the spread: FP32-sensitive
    assert v.ok and v.sensitive and v.signed < 0
    v = op.judge(10.0 * (1 + 5e-3), ref, spread=1e-3)       # 5x the spread: fails
    assert not v.ok and not v.sensitive
    v = op.judge(10.0 * (1 + 2e-3), ref, spread=1e-9)       # beyond tol with no spread to speak of
    assert not v.ok
    assert not op.judge(math.nan, ref).ok


def test_judge_tries_every_admissible_trajectory():
    """Two admissible switch trajectories: the result lies nearest the calm
    one (spread 1e-4) but 1.6e-2 from the chaotic one (spread 1.5e-2), the
    trajectory it took; it passes against the latter.  With both spreads
    small it fails, and the verdict describes the nearest trajectory."""
    ref = op.Reference([324.1, 328.2], [8, 9], 9e-5)
    got = 324.1 * (1 + 1.6e-2)
    v = op.judge(got, ref, spreads=[1.5e-2, 1e-4])
    assert v.ok and v.sensitive and v.which == 0 and abs(v.gap - 1.6e-2) < 1e-12
    v = op.judge(got, ref, spreads=[1e-3, 1e-4])
    assert not v.ok and v.which == 1 and abs(v.signed - (got - 328.2) / 328.2) < 1e-12


def test_perturbed_solve_without_perturbation_is_the_oracle():
    inst = wl.tiny_fp64(1)[0]
    assert sens.perturbed_wsr_bits(inst, 12) == _solve_bits(inst, 12)
    assert sens.perturbed_wsr_bits(inst, 12, opt=s.Options(switch_iter=3)) == _solve_bits(inst, 12, switch_iter=3)


def test_each_perturbation_acts_and_spread_is_their_maximum():
    """Every perturbation changes the result (it is applied), by small
    amounts on this well-conditioned 10 dB instance; the spread is the
    largest of those changes; the noise runs differ by seed; an early stop
    returns a value that reaches the requested level."""
    inst = wl.tiny_fp64(1)[0]
    ref = _solve_bits(inst, 12)
    w = sens.fp32_wsr_samples(inst, 12)
    rel = [abs(x - ref) / ref for x in w]
    assert len(w) == len(sens.VARIANTS) == 12
    assert all(0 < r < 1e-5 for r in rel), rel
    assert len(set(w[:sens.N_NOISE])) == sens.N_NOISE
    assert sens.fp32_spread(inst, 12) == max(rel)
    assert sens.fp32_spread(inst, 12, reference=ref) == max(rel)
    early = sens.fp32_spread(inst, 12, reference=ref, stop_at=rel[0] / 2)
    assert early == rel[0]


def test_noise_perturbation_has_the_stated_size():
    """One iteration with the per-step noise: the iterate moves by
    STEP_NOISE relative (Frobenius, to within sampling error)."""
    inst = wl.tiny_fp64(1)[0]
    V0 = s.initial_precoder(inst.G0, inst.P)
    st = s.AState(V=V0.copy(), Vprev=V0.copy())
    s.ammmse_iteration(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, st, s.Options())
    rng = np.random.default_rng(1)
    xi = (rng.standard_normal(st.V.shape) + 1j * rng.standard_normal(st.V.shape)) / np.sqrt(2.0)
    Vn = st.V * (1.0 + sens.STEP_NOISE * xi)
    relchg = np.linalg.norm(Vn - st.V) / np.linalg.norm(st.V)
    assert 0.5 * sens.STEP_NOISE < relchg < 2.0 * sens.STEP_NOISE


def test_covariance_rounding_hook_rounds_to_complex64():
    T = wl.cn01(np.random.default_rng(3), (3, 3))
    R = sens._round_c64(T)
    assert np.array_equal(R, T.astype(np.complex64).astype(np.complex128))
    assert 0 < np.max(np.abs(R - T) / np.abs(T)) <= 2.0 ** -24 * 1.01


@pytest.mark.slow
def test_spread_separates_the_regimes():
    """At 0 dB FP32-sized perturbations move the 50-iteration result of the
    timed workload by less than 1e-7; on a 25 dB instance by more than 1e-3."""
    lo = wl.single_cell_64(first=100, count=1)[0]
    hi = wl.single_cell_64(first=5488, count=1)[0]
    assert sens.fp32_spread(lo, 50) < 1e-7
    assert sens.fp32_spread(hi, 50) > 1e-3
