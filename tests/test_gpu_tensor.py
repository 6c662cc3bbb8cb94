"""Tensor-core (tcgen05) GEMM path against the FP64 oracle.

BF16X6 splits each FP32 operand into three bf16 terms (24 significant bits)
and accumulates the six products down to 2^-16 x 2^-8 in FP32: FP32-level
accuracy, held to the FP32 path's 1e-5 teacher-forced bound.  BF16X3 (hi +
lo, three products) carries a GEMM error of order 2^-16 (about 1.5e-5): its
teacher-forced bound is 2e-4.  Plain BF16 (8 significant bits): 2e-2.
Free-running solves of BF16X6 and BF16X3 must end within the 1e-3 WSR gap
(gpu_util.check_free_running: unless the instance is FP32-sensitive).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import solvers as osv

from gpu_util import GpuRun, check_free_running, rel, round_inputs

pytestmark = pytest.mark.gpu

TC_SHAPES = [
    (1, 4, 8, 2, 2),     # tiny workload shape
    (1, 16, 64, 4, 4),   # the timed workload shape (one full M = 128 tile each way)
    (1, 16, 64, 2, 2),   # unrolled workload shape
    (1, 5, 33, 4, 3),    # padded K (2Nt = 66 -> 80) and N (15 -> 16)
    (1, 7, 40, 4, 4),
    (1, 1, 5, 1, 1),
]
STEP_TOL = {"bf16x6": 1e-5, "bf16x3": 2e-4, "bf16": 2e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def small_batch(shape, n, seed):
    rng = np.random.default_rng(seed)
    return round_inputs([wl.random_small(rng, *shape) for _ in range(n)])


def _oracle_states(inst, iters, opt):
    V0 = osv.initial_precoder(inst.G0, inst.P)
    st = osv.AState(V=V0.copy(), Vprev=V0.copy())
    before, after, recs = [], [], []
    for _ in range(iters):
        before.append(osv.AState(V=st.V.copy(), Vprev=st.Vprev.copy(), t=st.t, stage=st.stage,
                                 stage_iter=st.stage_iter, rho_prev=st.rho_prev,
                                 gamma_c=None if st.gamma_c is None else st.gamma_c.copy()))
        recs.append(osv.ammmse_iteration(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d,
                                         st, opt))
        after.append(st.V.copy())
    return before, after, recs


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tc_teacher_forced_step(shape, prec):
    n, iters = 4, 10
    insts = small_batch(shape, n, 5000 + sum(shape))
    opt = osv.Options()
    runs = [_oracle_states(inst, iters, opt) for inst in insts]
    g = GpuRun(insts, precision=prec)
    worst = 0.0
    for t in range(iters):
        g.set_state_from_oracle([r[0][t] for r in runs])
        g.step(1)
        Vs = g.V()
        for b in range(n):
            if t > 0 and runs[b][0][t].stage == 1:
                relchg = abs(runs[b][2][t].rho - runs[b][2][t - 1].rho) / abs(runs[b][2][t - 1].rho)
                if abs(relchg - opt.eps1) < 1e-3:
                    continue
            e = rel(Vs[b], runs[b][1][t])
            worst = max(worst, e)
            assert e <= STEP_TOL[prec], (shape, prec, b, t + 1, e)
    print(f"{prec} {shape}: teacher-forced worst rel V err {worst:.2e}")
    g.close()


@pytest.mark.parametrize("shape", [(1, 16, 64, 4, 4), (1, 16, 64, 2, 2), (1, 5, 33, 4, 3)])
def test_tc_teacher_forced_step_fp32_solves(shape):
    """BF16X6 GEMMs with the per-user solves in FP32 (fp64_solves = 0; the
    extrapolation then overlaps the solves on the warps without a user):
    one step from the oracle's state within 1e-5, 10 iterations."""
    n, iters = 4, 10
    insts = small_batch(shape, n, 8500 + sum(shape))
    opt = osv.Options()
    runs = [_oracle_states(inst, iters, opt) for inst in insts]
    g = GpuRun(insts, precision="bf16x6", fp64_solves=0)
    worst = 0.0
    for t in range(iters):
        g.set_state_from_oracle([r[0][t] for r in runs])
        g.step(1)
        Vs = g.V()
        for b in range(n):
            if t > 0 and runs[b][0][t].stage == 1:
                relchg = abs(runs[b][2][t].rho - runs[b][2][t - 1].rho) / abs(runs[b][2][t - 1].rho)
                if abs(relchg - opt.eps1) < 1e-3:
                    continue
            e = rel(Vs[b], runs[b][1][t])
            worst = max(worst, e)
            assert e <= STEP_TOL["bf16x6"], (shape, b, t + 1, e)
    print(f"bf16x6 fp32 solves {shape}: teacher-forced worst rel V err {worst:.2e}")
    g.close()


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3"])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tc_free_running(shape, prec):
    n, iters = 8, 30
    insts = small_batch(shape, n, 6000 + sum(shape))
    g = GpuRun(insts, precision=prec)
    g.warmstart()
    g.step(iters)
    got = g.wsr()
    assert np.all(g.status() == 0)
    check_free_running(got, insts, iters, f"{prec} {shape}")
    g.close()


@pytest.mark.parametrize("prec", ["bf16x6"])
def test_tc_matches_plain_path_on_timed_workload_sample(prec):
    """512 instances of the timed workload (all seven P values), 50
    iterations: the tensor-core path against the FP32 path and against the
    oracle on a sample (BF16X6, the accuracy-matched split)."""
    insts = []
    for q in range(7):
        insts += wl.single_cell_64(first=q * 1024, count=512 // 7 + 1)
    insts = insts[:512]
    a = GpuRun(insts, precision="fp32")
    a.warmstart()
    a.step(50)
    wa = a.wsr()
    b = GpuRun(insts, precision=prec)
    b.warmstart()
    b.step(50)
    wb = b.wsr()
    d = np.abs(wa - wb) / wa
    print(f"{prec} vs fp32 WSR: median {np.median(d):.2e}, max {d.max():.2e}")
    check_free_running(wb, insts, 50, f"{prec} sample", sample=[0, 100, 250, 400, 511])
    a.close()
    b.close()


def test_tc_checkpoint_resume_is_exact():
    insts = small_batch((1, 16, 64, 4, 4), 3, 91)
    a = GpuRun(insts, precision="bf16x6")
    a.warmstart()
    a.step(9)
    b = GpuRun(insts, precision="bf16x6")
    b.warmstart()
    b.step(4)
    st = b.get_state()
    c = GpuRun(insts, precision="bf16x6")
    c.s.set_state(**st)
    c.step(5)
    for x, y in zip(a.V(), c.V()):
        assert np.array_equal(x, y)
    for r in (a, b, c):
        r.close()
