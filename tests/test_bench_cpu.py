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
        (b, w, margin), = bench._oracle_worker((3, 1, 4, name))
        inst = bench._round32(gen())
        V0 = osv.initial_precoder(inst.G0, inst.P)
        r = osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, 4)
        assert b == 3 and margin >= 0
        assert np.isclose(w, om.wsr_bits(inst.H, r.V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d), rtol=0,
                          atol=0)
