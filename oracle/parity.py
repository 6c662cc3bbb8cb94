"""FP64 oracle, part 5: the reference results a free-running GPU solve is
judged against, and the rule that judges it.

TEST INFRASTRUCTURE ONLY (see ``oracle.model``): used by ``tests/`` and by
the CPU-baseline leg of ``bench.py``.

The target is a final WSR within GAP_TOL = 1e-3 (relative) of the FP64
oracle after the same number of iterations.  Two things make a single
oracle number the wrong reference for some instances:

* The stage switch of Algorithm 3 is a threshold test on the relative WSR
  change.  Where that change lies within SWITCH_MARGIN of eps1 the decision
  is fixed by rounding, and each decision gives a different, equally valid
  trajectory.  Such an instance gets one reference per admissible switch
  iteration (``reference_solves``), each the oracle's solve with that switch
  forced, and the GPU result is compared with the nearest.
* At high SNR some trajectories amplify rounding: the oracle itself, with
  perturbations of the size of the FP32 iteration's per-step error, moves by
  ``spread`` (``oracle.sensitivity.fp32_spread``).  An instance beyond
  GAP_TOL passes as FP32-sensitive only if its gap is at most SPREAD_FACTOR
  times that spread; otherwise it fails.  (The spread is computed only as
  far as the verdict needs: it stops once it reaches gap / SPREAD_FACTOR.)
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

from . import model as m
from . import solvers as s
from .sensitivity import fp32_spread

GAP_TOL = 1e-3
SWITCH_MARGIN = 1e-4
SPREAD_FACTOR = 4.0


@dataclasses.dataclass
class Reference:
    wsr: List[float]                 # final WSR (bits) per admissible trajectory; [0] = the oracle's own
    switch: List[Optional[int]]      # its switch iteration (None: stage I throughout)
    margin: float                    # closest |relative change - eps1| over the decisions taken


def _solve_bits(inst, iters, opt):
    V0 = s.initial_precoder(inst.G0, inst.P)
    r = s.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, iters, opt)
    return r, m.wsr_bits(inst.H, r.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


def _switch_of(r):
    return next((h.t for h in r.history if h.stage == 2), None)


def reference_solves(inst, iters, opt: Optional[s.Options] = None) -> Reference:
    """The oracle's solve (Algorithm 3, options ``opt``, default the paper's)
    and, where a stage decision came within SWITCH_MARGIN of eps1, the solves
    with the switch forced at each other admissible iteration: every stage-I
    test t up to the first unambiguous switch whose relative change is within
    the margin may go either way, and a switch at such a t (all earlier
    ambiguous tests going the other way) is one more admissible trajectory."""
    opt = opt or s.Options()
    r, w = _solve_bits(inst, iters, opt)
    sw = _switch_of(r)
    if opt.switch_iter >= 1:
        return Reference([w], [sw], math.inf)
    rho = [h.rho for h in r.history]
    # relative changes of the stage-I tests the oracle ran (t = 2 .. switch)
    last = sw if sw is not None else len(rho)
    chg = {t: m.relative_change(rho[t - 1], rho[t - 2]) for t in range(2, last + 1)}
    margin = min((abs(c - opt.eps1) for c in chg.values()), default=math.inf)
    if margin >= SWITCH_MARGIN:
        return Reference([w], [sw], margin)
    # the ambiguous tests need the stage-I trajectory past the oracle's switch
    pure = s.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d,
                    s.initial_precoder(inst.G0, inst.P), iters, dataclasses.replace(opt, switch_iter=10 ** 9))
    prho = [h.rho for h in pure.history]
    cands = []
    for t in range(2, iters + 1):
        c = m.relative_change(prho[t - 1], prho[t - 2])
        if abs(c - opt.eps1) < SWITCH_MARGIN:
            cands.append(t)
        elif c <= opt.eps1:
            cands.append(t)
            break
    else:
        cands.append(None)  # every test may go the "stay" way: stage I throughout
    ref = Reference([w], [sw], margin)
    for t in cands:
        if t == sw:
            continue
        o = dataclasses.replace(opt, switch_iter=10 ** 9 if t is None else t)
        ref.wsr.append(_solve_bits(inst, iters, o)[1])
        ref.switch.append(t)
    return ref


@dataclasses.dataclass
class Verdict:
    gap: float                       # relative gap to the nearest admissible reference
    signed: float                    # (gpu - reference) / reference for that reference
    which: int                       # index into Reference.wsr
    spread: Optional[float] = None   # fp32_spread of that reference (computed only beyond GAP_TOL)
    ok: bool = True
    sensitive: bool = False          # beyond GAP_TOL but within SPREAD_FACTOR * spread


def nearest(gpu_wsr: float, ref: Reference):
    gaps = [abs(gpu_wsr - w) / abs(w) for w in ref.wsr]
    k = min(range(len(gaps)), key=gaps.__getitem__)
    return k, gaps[k], (gpu_wsr - ref.wsr[k]) / abs(ref.wsr[k])


def judge(gpu_wsr: float, ref: Reference, inst=None, iters: int = 0, opt: Optional[s.Options] = None,
          spread: Optional[float] = None, spreads: Optional[List[float]] = None) -> Verdict:
    """Judge one GPU result against its references, each admissible
    trajectory in turn from the nearest: within GAP_TOL of one it passes;
    beyond, that trajectory's FP32 spread (``spreads[k]``, else ``spread``,
    else computed from ``inst``) decides: gap <= SPREAD_FACTOR * spread
    passes as FP32-sensitive.  A run follows one trajectory, and the
    nearest in WSR need not be the one it took (a chaotic trajectory can
    end beside a calm one), so every trajectory is tried before the result
    fails; the verdict then describes the nearest.  A non-finite GPU result
    fails."""
    if not math.isfinite(gpu_wsr):
        return Verdict(math.inf, math.inf, 0, None, ok=False)
    gaps = [abs(gpu_wsr - w) / abs(w) for w in ref.wsr]
    order = sorted(range(len(gaps)), key=gaps.__getitem__)
    first = None
    for k in order:
        v = Verdict(gaps[k], (gpu_wsr - ref.wsr[k]) / abs(ref.wsr[k]), k)
        if v.gap <= GAP_TOL:
            return v
        if spreads is not None:
            sp = spreads[k]
        elif spread is not None:
            sp = spread
        else:
            o = opt or s.Options()
            if ref.switch[k] is not None or k > 0:
                o = dataclasses.replace(o, switch_iter=10 ** 9 if ref.switch[k] is None else ref.switch[k])
            sp = fp32_spread(inst, iters, reference=ref.wsr[k], opt=o, stop_at=v.gap / SPREAD_FACTOR)
        v.spread = sp
        v.sensitive = v.gap <= SPREAD_FACTOR * sp
        v.ok = v.sensitive
        if v.ok:
            return v
        if first is None:
            first = v
    return first
