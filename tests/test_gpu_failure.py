"""Failure detection on the GPU without a fault: a wait budget of one SM
clock cycle makes every bounded device-side wait run out (the bulk-copy
mbarrier of the plain kernel, the tensor-core commit mbarrier), so each
instance must report AMM_ETIMEOUT through its status word and WSR NaN,
the call must return normally, and the device must stay usable for a
fresh context whose solves match the FP64 oracle."""
import numpy as np
import pytest
import torch

import workloads as wl

from gpu_util import GpuRun, oracle_run, oracle_wsr_bits

pytestmark = pytest.mark.gpu

AMM_ETIMEOUT = 5


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_wait_budget_exhausted_reports_timeout(prec):
    import __graft_entry__ as ge
    ge.build()
    insts = wl.single_cell_64(first=3000, count=16)
    g = GpuRun(insts, precision=prec, spin_budget=1)
    g.warmstart()
    g.step(3)
    st = g.status()
    w = g.wsr()
    g.close()
    print(f"{prec}: statuses {np.unique(st)}")
    assert np.all(st == AMM_ETIMEOUT), st
    assert np.all(np.isnan(w))
    # the device is still usable: a fresh context solves correctly
    ok = GpuRun(wl.single_cell_64(first=3000, count=4), precision=prec)
    ok.warmstart()
    ok.step(10)
    got = ok.wsr()
    assert np.all(ok.status() == 0)
    for b, inst in enumerate(ok.insts):
        want = oracle_wsr_bits(inst, oracle_run(inst, 10).V)
        assert abs(got[b] - want) <= 1e-4 * want
    ok.close()


@pytest.mark.parametrize("nth", [1, 3, 7])
def test_injected_allocation_failure_cleans_up(nth):
    """A device allocation that fails part-way through amm_create (injected
    on the host at the nth allocation) returns AMM_ENOMEM after freeing what
    it had allocated; the device is untouched and a context created next
    solves correctly."""
    import ctypes
    import paper_2510_20507_gb300 as pkg
    lib = pkg.load_library()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.amm_test_fail_alloc(nth)
    try:
        with pytest.raises(pkg.AmmError) as ei:
            pkg.Solver(64, (1, 16, 64, 4, 4))
    finally:
        lib.amm_test_fail_alloc(0)
    assert ei.value.status == pkg.AMM_ENOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)  # nothing of the failed context stays allocated
    insts = wl.tiny_fp64(3)
    g = GpuRun(insts)
    g.warmstart()
    g.step(5)
    assert np.all(np.isfinite(g.wsr())) and np.all(g.status() == 0)
    g.close()


def test_cluster_wait_budget_exhausted_reports_timeout():
    """The seven-cell cluster kernel with a one-cycle wait budget: the bulk
    copies and the cluster exchange rounds run out, every instance reports
    AMM_ETIMEOUT with WSR NaN, the launch returns, and a fresh context on
    the same layout solves."""
    import __graft_entry__ as ge
    ge.build()
    from gpu_util import round_inputs
    insts = round_inputs(wl.hex7(n=256, count=8))
    g = GpuRun(insts, spin_budget=1)
    assert g.s.path == "cluster"
    g.warmstart()
    g.step(3)
    st = g.status()
    w = g.wsr()
    g.close()
    assert np.all(st == AMM_ETIMEOUT), st
    assert np.all(np.isnan(w))
    ok = GpuRun(insts[:2])
    ok.warmstart()
    ok.step(4)
    assert np.all(ok.status() == 0) and np.all(np.isfinite(ok.wsr()))
    ok.close()
