"""amm_solve_noalloc, the entry point for callers that may not allocate
device memory while they run (for example a scheduler working inside a
per-slot deadline, where an allocation can stall the device), against the
regular entry points on the same inputs, on two calls in a row.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test when it gets here; it also passes on its own
in a fresh process.
"""
import numpy as np
import pytest

import workloads as wl

from gpu_util import GpuRun, round_inputs, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _regular(insts, iters):
    g = GpuRun(insts)
    g.warmstart()
    g.step(iters)
    wsr = g.wsr()
    V = g.V()
    g.close()
    return wsr, V


def _noalloc(insts, iters):
    import torch
    import paper_2510_20507_gb300 as pkg
    pk = wl.pack(insts)
    V_out = torch.empty(pk.G0.size, dtype=torch.complex64, device="cuda:0")
    wsr = torch.empty(len(insts), dtype=torch.float64, device="cuda:0")
    pkg.solve_noalloc(len(insts), pk.dims[0], to_dev(pk.H), to_dev(pk.alpha), to_dev(pk.sigma2), to_dev(pk.P),
                      to_dev(pk.G0), iters, V_out, wsr)
    torch.cuda.synchronize()
    return wsr.cpu().numpy(), wl.unpack_V(pk, V_out.cpu().numpy())


def test_noalloc_matches_regular_entry_points_on_two_calls():
    cases = [(wl.single_cell_64(first=3000, count=96), 20),   # Nt=64, K=16, Nr=4, d=4
             (wl.tiny_fp64(40), 15)]                           # Nt=8, K=4, Nr=2, d=2
    for insts, iters in cases:
        insts = round_inputs(insts)
        want_wsr, want_V = _regular(insts, iters)
        got_wsr, got_V = _noalloc(insts, iters)
        assert np.all(np.isfinite(got_wsr))
        assert np.allclose(got_wsr, want_wsr, rtol=1e-6, atol=0)
        for a, b in zip(got_V, want_V):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_noalloc_rejects_a_batch_beyond_its_array():
    import torch
    import paper_2510_20507_gb300 as pkg
    n = 2000  # 2000 instances of Nt=64, K=16 need ~130 MB of workspace
    z = torch.zeros(8, dtype=torch.float32, device="cuda:0")
    with pytest.raises(pkg.AmmError) as ei:
        pkg.solve_noalloc(n, (1, 16, 64, 4, 4), z, z, z, z, z, 10, z, z)
    assert ei.value.status == pkg.AMM_EINVAL
    assert "static array" in str(ei.value)
