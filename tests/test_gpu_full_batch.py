"""Every instance of the timed workload against the FP64 oracle.

The target is a final WSR within 1e-3 relative of the oracle.  This solves
the whole single-cell P sweep (7 x 1024 instances, Nt=64, K=16, Nr=4, d=4,
50 iterations) on the GPU in the launch configuration bench.py times, for
the plain FP32 path and the
BF16X6 tensor-core path, and re-solves all 7168 instances with the oracle
on a spawn-started process pool over the host cores (about two minutes on
16 cores).  Instances whose oracle trajectory takes the stage decision
within 1e-4 of eps1 are reported separately (the decision is then not
determined by either side's rounding).

Per step the GPU matches the oracle to about 1e-7, but at 20-30 dB some
50-iteration trajectories (about 1 %) are sensitive to rounding: storing
only the N_r x N_r receive covariance in FP32 moves the oracle's own final
WSR by more than 1e-3 on such instances (test_oracle_rounding_sensitivity).
So the bar here is: every instance within 1e-3 unless FP32-sized
perturbations move the oracle's own result by more than 1e-5 there
(gpu_util.oracle_fp32_spread; elsewhere they move it by 1e-7 or less), at
least 98 % of instances within 1e-3, the mean WSR of each P value within
3e-4 of the oracle's, and no instance beyond 5e-2.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ITERS = 50


def _spread_one(b):
    import workloads as wl
    from gpu_util import oracle_fp32_spread, round_inputs
    return oracle_fp32_spread(round_inputs(wl.single_cell_64(first=b, count=1))[0], ITERS)


def _pool():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(os.cpu_count() or 1)


def _oracle_chunk(args):
    first, count = args
    import workloads as wl
    from oracle import model as om
    from oracle import solvers as osv
    out = []
    for inst in wl.single_cell_64(first=first, count=count):
        inst.H = inst.H.astype(np.complex64).astype(np.complex128)
        inst.G0 = inst.G0.astype(np.complex64).astype(np.complex128)
        inst.alpha = inst.alpha.astype(np.float32).astype(np.float64)
        inst.sigma2 = inst.sigma2.astype(np.float32).astype(np.float64)
        inst.P = inst.P.astype(np.float32).astype(np.float64)
        V0 = osv.initial_precoder(inst.G0, inst.P)
        r = osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, ITERS)
        margin = np.inf
        for a, b in zip(r.history, r.history[1:]):
            if a.stage == 1:
                margin = min(margin, abs(abs(b.rho - a.rho) / abs(a.rho) - 0.1))
        out.append((om.wsr_bits(inst.H, r.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d), margin))
    return out


@pytest.fixture(scope="module")
def oracle_all():
    cores = os.cpu_count() or 1
    chunk = 7168 // (4 * cores) + 1
    jobs = [(f, min(chunk, 7168 - f)) for f in range(0, 7168, chunk)]
    with _pool() as pool:
        res = pool.map(_oracle_chunk, jobs)
    flat = [x for r in res for x in r]
    return np.array([w for w, _ in flat]), np.array([m for _, m in flat])


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_every_instance_within_gap(prec, oracle_all):
    import __graft_entry__ as ge
    ge.build()
    import workloads as wl
    from gpu_util import SENSITIVE, GpuRun
    want, margin = oracle_all
    g = GpuRun(wl.single_cell_64(), precision=prec)
    g.warmstart()
    g.step(ITERS)
    got = g.wsr()
    g.close()
    gap = np.abs(got - want) / want
    decided = margin >= 1e-4
    bad = np.where(decided & (gap > 1e-3))[0]
    print(f"{prec}: max gap {gap[decided].max():.2e}, p99 {np.percentile(gap[decided], 99):.2e}, "
          f"median {np.median(gap):.2e}, instances over 1e-3: {len(bad)} "
          f"(near-threshold stage decisions excluded: {int((~decided).sum())})")
    for b in bad[:10]:
        print(f"  instance {b}: P={10 * np.log10(wl.single_cell_64(first=b, count=1)[0].P[0]):.0f} dB "
              f"gpu {got[b]:.6f} oracle {want[b]:.6f} gap {gap[b]:.2e}")
    means = []
    for q in range(7):
        sl = slice(q * 1024, (q + 1) * 1024)
        means.append((got[sl].mean() - want[sl].mean()) / want[sl].mean())
    print(f"{prec}: per-P mean WSR gap " + " ".join(f"{x:+.1e}" for x in means))
    with _pool() as pool:
        spread = np.array(pool.map(_spread_one, [int(b) for b in bad]))
    for b, sp in zip(bad, spread):
        print(f"  instance {b}: gap {gap[b]:.2e}, oracle spread under FP32-sized perturbation {sp:.2e}")
    assert np.all(spread > SENSITIVE), [(int(b), sp) for b, sp in zip(bad, spread) if sp <= SENSITIVE]
    assert np.mean(gap[decided] <= 1e-3) >= 0.98
    assert max(abs(x) for x in means) <= 3e-4
    assert gap.max() <= 5e-2
