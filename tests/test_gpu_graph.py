"""CUDA-graph replay of a whole solve (amm_graph_*) against the same calls
issued one by one, including a replay after the inputs were refilled."""
import numpy as np
import pytest
import torch

import workloads as wl

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_graph_replay_matches_direct_calls(prec):
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    a = wl.pack(wl.single_cell_64(first=5000, count=64))
    b = wl.pack(wl.single_cell_64(first=200, count=64))
    dims = a.dims[0]
    H, al, s2, P, G0 = (to_dev(a.H), to_dev(a.alpha), to_dev(a.sigma2), to_dev(a.P), to_dev(a.G0))
    stream = torch.cuda.Stream()

    def direct(pk):
        s = pkg.Solver(64, dims, stream=stream, precision=prec)
        out = torch.empty(64, dtype=torch.float64, device="cuda:0")
        ins = [to_dev(x) for x in (pk.H, pk.alpha, pk.sigma2, pk.P, pk.G0)]
        torch.cuda.synchronize()
        s.set_problem(*ins[:4])
        s.warmstart(ins[4])
        s.step(30)
        s.wsr(out)
        stream.synchronize()
        s.close()
        return out.cpu().numpy()

    want_a, want_b = direct(a), direct(b)
    s = pkg.Solver(64, dims, stream=stream, precision=prec)
    out = torch.empty(64, dtype=torch.float64, device="cuda:0")
    nxt = [to_dev(x) for x in (b.H, b.alpha, b.sigma2, b.P, b.G0)]
    torch.cuda.synchronize()
    g = s.capture(H, al, s2, P, G0, 30, out)
    n0 = s.launches
    g.launch()
    stream.synchronize()
    assert np.array_equal(out.cpu().numpy(), want_a)
    with torch.cuda.stream(stream):  # refill the inputs in place, stream-ordered, and replay
        for dst, src in zip((H, al, s2, P, G0), nxt):
            dst.copy_(src)
    g.launch()
    stream.synchronize()
    assert np.array_equal(out.cpu().numpy(), want_b)
    assert s.launches - n0 == 2 * 4  # normalise, warm start, iterate, WSR per replay
    g.close()
    s.close()
