"""Every instance of the timed workload against the FP64 oracle.

The target is a final WSR within 1e-3 relative of the oracle.  This solves
the whole single-cell P sweep (7 x 1024 instances, Nt=64, K=16, Nr=4, d=4,
50 iterations) on the GPU in the launch configuration bench.py times, for
the plain FP32 path and the BF16X6 tensor-core path (with FP64 and with
float-float per-user solves), and re-solves all 7168
instances with the oracle on a spawn-started process pool over the host
cores (about two minutes on 16 cores).

Each instance is judged by oracle.parity: within 1e-3 of the nearest
admissible oracle trajectory (two or more only where the oracle's stage
decision came within 1e-4 of eps1, where rounding decides it), or else
within 4 x the oracle's own spread under FP32-sized perturbations of its
arithmetic (at 20-30 dB about 1 % of these 50-iteration trajectories
amplify rounding; test_oracle_rounding_sensitivity).  No instance may fail
that rule, none is skipped, and the mean WSR of each P value must be within
3e-4 of the oracle's.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ITERS = 50


def _refs_chunk(args):
    first, count = args
    import workloads as wl
    from gpu_util import round_inputs
    from oracle import parity as op
    return [op.reference_solves(inst, ITERS) for inst in round_inputs(wl.single_cell_64(first=first, count=count))]


def _judge_beyond(args):
    b, got, ref = args
    import workloads as wl
    from gpu_util import round_inputs
    from oracle import parity as op
    return op.judge(got, ref, round_inputs(wl.single_cell_64(first=b, count=1))[0], ITERS)


@pytest.fixture(scope="module")
def oracle_refs():
    import os
    from gpu_util import spawn_pool
    cores = os.cpu_count() or 1
    chunk = 7168 // (4 * cores) + 1
    jobs = [(f, min(chunk, 7168 - f)) for f in range(0, 7168, chunk)]
    with spawn_pool() as pool:
        res = pool.map(_refs_chunk, jobs)
    return [r for part in res for r in part]


@pytest.mark.parametrize("prec,solves", [("fp32", 1), ("bf16x6", 1), ("bf16x6", 2)])
def test_every_instance_within_gap(prec, solves, oracle_refs):
    import __graft_entry__ as ge
    ge.build()
    import workloads as wl
    from gpu_util import GpuRun, spawn_pool
    from oracle import parity as op
    g = GpuRun(wl.single_cell_64(), precision=prec, fp64_solves=solves)
    g.warmstart()
    g.step(ITERS)
    got = g.wsr()
    assert np.all(g.status() == 0)
    g.close()
    near = [op.nearest(float(got[b]), ref) for b, ref in enumerate(oracle_refs)]
    gap = np.array([x[1] for x in near])
    signed = np.array([x[2] for x in near])
    beyond = [int(b) for b in np.where(gap > op.GAP_TOL)[0]]
    with spawn_pool() as pool:
        verdicts = pool.map(_judge_beyond, [(b, float(got[b]), oracle_refs[b]) for b in beyond], chunksize=1)
    fails = [(b, v.gap, v.spread) for b, v in zip(beyond, verdicts) if not v.ok]
    for b, v in zip(beyond, verdicts):
        print(f"  instance {b}: P={10 * np.log10(wl.single_cell_64(first=b, count=1)[0].P[0]):.0f} dB "
              f"gap {v.gap:.2e} signed {v.signed:+.2e} spread {v.spread:.2e} ratio {v.gap / v.spread:.2f} "
              f"{'ok' if v.ok else 'FAIL'}")
    means = []
    for q in range(7):
        sl = slice(q * 1024, (q + 1) * 1024)
        w = np.array([r.wsr[k] for r, (k, _, _) in zip(oracle_refs[sl], near[sl])])
        means.append((got[sl].mean() - w.mean()) / w.mean())
    print(f"{prec}: max gap {gap.max():.2e}, p99 {np.percentile(gap, 99):.2e}, median {np.median(gap):.2e}, "
          f"mean signed {signed.mean():+.2e}, over 1e-3: {len(beyond)}, failed: {len(fails)}, "
          f"ambiguous switch: {sum(len(r.wsr) > 1 for r in oracle_refs)}")
    print(f"{prec}: per-P mean WSR gap " + " ".join(f"{x:+.1e}" for x in means))
    assert not fails, fails
    assert max(abs(x) for x in means) <= 3e-4
