"""Host-side pieces of bench.py: the source digest that gates the captured
ncu counters, and the oracle workers of the CPU-baseline legs."""
import numpy as np

import bench
import workloads as wl
from oracle import model as om
from oracle import solvers as osv


def test_kernel_digest_covers_existing_sources():
    dg = bench.kernel_digest()
    assert len(dg) == 16 and int(dg, 16) >= 0


def test_oracle_worker_on_named_workloads_matches_direct_oracle():
    for name, gen in (("uneven", lambda: wl.uneven(n=bench.UNEVEN_N, first=3, count=1)[0]),
                      ("sweep", lambda: wl.single_cell_64(bench.N_PER_P, first=3, count=1)[0])):
        (b, ref), = bench._oracle_worker((3, 1, 4, name))
        w, margin = ref.wsr[0], ref.margin
        inst = bench._round32(gen())
        V0 = osv.initial_precoder(inst.G0, inst.P)
        r = osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, 4)
        assert b == 3 and margin >= 0
        assert np.isclose(w, om.wsr_bits(inst.H, r.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d), rtol=0,
                          atol=0)


def test_gap_check_counts_every_instance():
    """bench.gap_check on fabricated GPU results: one within 1e-3, one off
    by 2e-2 on a well-conditioned instance (fails: its FP32 spread is tiny);
    nothing is skipped."""
    import multiprocessing.dummy as mpd
    res = bench._oracle_worker((3, 2, 4, "sweep"))
    got = {3: res[0][1].wsr[0] * (1 + 5e-4), 4: res[1][1].wsr[0] * (1 + 2e-2)}
    with mpd.Pool(2) as pool:
        par = bench.gap_check(pool, got, res, iters=4)
    assert par["checked"] == 2 and par["within_1e-3"] == 1 and par["over_1e-3"] == 1
    assert par["failed"] == 1 and not par["all_pass"]


def test_wmmse_worker_is_the_oracle_wmmse_on_rounded_inputs():
    """The WMMSE workload's CPU leg: the oracle's Algorithm 2 on instance b
    of the workload, inputs rounded as the GPU receives them, WSR in bits."""
    b, got = bench._wmmse_worker((3, 2))
    inst = bench._round32(wl.unrolled_64(n=bench.WMMSE_N, first=3, count=1)[0])
    V0 = osv.initial_precoder(inst.G0, inst.P)
    _, hist, _ = osv.wmmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, 2,
                           tol=1e-4, max_bisect=100)
    assert b == 3 and got == hist[-1] / np.log(2.0)
    assert bench._instances("wmmse", 3, 1)[0].dims == (1, 16, 64, 2, 2)
