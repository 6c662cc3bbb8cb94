"""Failure detection on the GPU without a fault: a wait budget of one SM
clock cycle makes every bounded device-side wait run out (the bulk-copy
mbarrier of the plain kernel, the tensor-core commit mbarrier), so each
instance must report AMM_ETIMEOUT through its status word and WSR NaN,
the call must return normally, and the device must stay usable for a
fresh context whose solves match the FP64 oracle."""
import numpy as np
import pytest

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
