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
from gpu_util import GpuRun, assert_step_bounds, check_free_running, round_inputs, teacher_forced

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
RHO_TOL = STEP_TOL  # R^t carries the relative error of the Z it is computed from
GAMMA_TOL = {"bf16x6": 1e-5, "bf16x3": 2e-4, "bf16": 2e-2}
FLIP = {"bf16x6": 1e-4, "bf16x3": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def small_batch(shape, n, seed):
    rng = np.random.default_rng(seed)
    return round_inputs([wl.random_small(rng, *shape) for _ in range(n)])


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tc_teacher_forced_step(shape, prec):
    """One iteration from the oracle's state, every t of a 10-iteration
    run: V (whole and per user block), R^t, stage and gamma_c, with the
    precision's bounds (R^t and gamma_c scale with the GEMM error)."""
    insts = small_batch(shape, 4, 5000 + sum(shape))
    worst = teacher_forced(insts, 10, gpu_opts=dict(precision=prec), flip_margin=FLIP[prec])
    assert_step_bounds(worst, f"{prec} {shape}", v_tol=STEP_TOL[prec], rho_tol=RHO_TOL[prec],
                       gamma_tol=GAMMA_TOL[prec])


@pytest.mark.parametrize("solves", [0, 2])
@pytest.mark.parametrize("shape", [(1, 16, 64, 4, 4), (1, 16, 64, 2, 2), (1, 5, 33, 4, 3), (1, 4, 8, 2, 2)])
def test_tc_teacher_forced_step_other_solves(shape, solves):
    """BF16X6 GEMMs with the per-user solves in FP32 (fp64_solves = 0; the
    extrapolation then overlaps the solves on the warps without a user) or
    in float-float (2): one step from the oracle's state within 1e-5, 10
    iterations."""
    insts = small_batch(shape, 4, 8500 + sum(shape))
    worst = teacher_forced(insts, 10, gpu_opts=dict(precision="bf16x6", fp64_solves=solves))
    assert_step_bounds(worst, f"bf16x6 solves {solves} {shape}")


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
