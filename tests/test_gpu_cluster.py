"""The multi-cell cluster kernel (one thread-block cluster per instance,
one block per cell, exchanges over distributed shared memory) against the
FP64 oracle and against the one-block-per-instance kernel.

Small multi-cell shapes are sent down the cluster path by a shared-memory
budget under which the whole channel no longer fits one block but one
cell's block does; the seven-cell layout takes it by default (its 1 MB
channel never fits one block).  Same bounds as the other per-step tests."""
import numpy as np
import pytest

import workloads as wl

from gpu_util import GpuRun, assert_step_bounds, check_free_running, rel, round_inputs, teacher_forced

pytestmark = pytest.mark.gpu

# (shape, shared-memory budget that forces the cluster path)
SMALL = [((3, 3, 40, 2, 2), 16384), ((2, 4, 57, 4, 3), 34816), ((4, 2, 24, 2, 1), 12288), ((7, 2, 16, 1, 1), 12288)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def small_batch(shape, n, seed):
    rng = np.random.default_rng(seed)
    return round_inputs([wl.random_small(rng, *shape) for _ in range(n)])


@pytest.mark.parametrize("shape,budget", SMALL)
def test_small_shapes_take_the_cluster_path(shape, budget):
    g = GpuRun(small_batch(shape, 2, 1), smem_budget=budget)
    assert g.s.path == "cluster"
    g.close()
    g = GpuRun(small_batch(shape, 2, 1), smem_budget=budget, cluster_cells=0)
    assert g.s.path == "block"
    g.close()


def test_seven_cell_layout_takes_the_cluster_path():
    g = GpuRun(round_inputs(wl.hex7(n=256, count=2)))
    assert g.s.path == "cluster"
    g.close()


@pytest.mark.parametrize("solves", [1, 2])
@pytest.mark.parametrize("shape,budget", SMALL)
def test_cluster_teacher_forced_step(shape, budget, solves):
    """Every iteration of a 12-iteration run from the oracle's state: V
    (whole and per user block), R^t, stage, stage counter, gamma_c."""
    insts = small_batch(shape, 4, 9100 + sum(shape))
    worst = teacher_forced(insts, 12, gpu_opts=dict(smem_budget=budget, fp64_solves=solves))
    assert_step_bounds(worst, f"cluster {shape} solves {solves}")


@pytest.mark.parametrize("shape,budget", SMALL)
def test_cluster_free_running(shape, budget):
    insts = small_batch(shape, 8, 9200 + sum(shape))
    g = GpuRun(insts, smem_budget=budget)
    assert g.s.path == "cluster"
    g.warmstart()
    g.step(30)
    got = g.wsr()
    assert np.all(g.status() == 0)
    g.close()
    check_free_running(got, insts, 30, f"cluster {shape}")


def test_cluster_matches_block_kernel_on_seven_cells():
    """The same seven-cell instances, 5 iterations, on the cluster kernel and
    on the one-block kernel that restages each cell's channel block: the
    same iterates to FP32 accuracy (the summation orders differ)."""
    insts = round_inputs(wl.hex7(n=256, count=12))
    out = []
    for cl in (1, 0):
        g = GpuRun(insts, cluster_cells=cl)
        assert g.s.path == ("cluster" if cl else "block")
        g.warmstart()
        g.step(5)
        out.append((g.V(), g.wsr()))
        g.close()
    for b in range(len(insts)):
        assert rel(out[0][0][b], out[1][0][b]) <= 1e-5, b
        assert abs(out[0][1][b] - out[1][1][b]) <= 1e-5 * abs(out[1][1][b]), b


def test_cluster_tolerance_mode_and_resume():
    """amm_solve's eps2 stop on the cluster path, and a bit-exact resume from
    amm_get_state."""
    import torch
    shape, budget = SMALL[0]
    insts = small_batch(shape, 4, 9300)
    a = GpuRun(insts, smem_budget=budget)
    a.warmstart()
    a.step(9)
    Va = a.V()
    b = GpuRun(insts, smem_budget=budget)
    b.warmstart()
    b.step(4)
    st = b.get_state()
    c = GpuRun(insts, smem_budget=budget)
    c.s.set_state(**st)
    c.step(5)
    for x, y in zip(Va, c.V()):
        assert np.array_equal(x, y)
    d = GpuRun(insts, smem_budget=budget)
    d.warmstart()
    iters = torch.zeros(len(insts), dtype=torch.int32, device="cuda:0")
    d.s.solve(300, iters)
    assert np.all(d.status() == 0) and np.all(iters.cpu().numpy() < 300)
    for r in (a, b, c, d):
        r.close()
