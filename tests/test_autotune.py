"""Autotuner: candidate selection and the cache (CPU, with the timing and
the device name replaced), and on the GPU that every candidate of the FP32
class computes the same solve."""
import json

import numpy as np
import pytest

from paper_2510_20507_gb300 import autotune


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    cache = str(tmp_path / "tune.json")
    monkeypatch.setattr(autotune, "_device_name", lambda: "Fake GPU")
    fake = {("fp32", 0): 3.5, ("fp32", 1): 5.0, ("fp32", 2): 3.0, ("fp32", 3): 4.0, ("fp32", 4): 3.2,
            ("fp32", 5): 3.3, ("bf16x6", 0): 2.5}
    calls = []

    def fake_time(dims, ov, base=None, **kw):
        calls.append(ov)
        return fake[(ov["precision"], ov["gemm_tile"])]
    monkeypatch.setattr(autotune, "time_config", fake_time)
    e = autotune.tune((1, 16, 64, 4, 4), "fp32", base={"fp64_solves": 1}, cache=cache)
    assert e["overrides"] == {"precision": "bf16x6", "gemm_tile": 0} and len(calls) == 7
    table = json.load(open(cache))
    assert list(table) == ["Fake_GPU|1x16x64x4x4|fp32|fp64_solves=1"]
    calls.clear()
    assert autotune.tune((1, 16, 64, 4, 4), "fp32", base={"fp64_solves": 1}, cache=cache) == e
    assert calls == []  # served from the cache
    e2 = autotune.tune((1, 4, 8, 2, 2), "fp32", base={"fp64_solves": 1}, cache=cache)
    assert len(json.load(open(cache))) == 2 and e2["ms"] == 2.5
    with pytest.raises(KeyError):
        autotune.tune((1, 4, 8, 2, 2), "fp16", cache=cache)


@pytest.mark.gpu
def test_fp32_class_candidates_compute_the_same_solve():
    """The register tiles change which thread computes an entry (and so the
    order of the block reductions), not the arithmetic: three iterations
    agree to FP32 rounding on an uneven batch."""
    import __graft_entry__ as ge
    ge.build()
    import workloads as wl
    from gpu_util import GpuRun, rel
    insts = wl.uneven(n=64)
    res = {}
    for tile in (1, 2, 3, 4, 5):
        g = GpuRun(insts, gemm_tile=tile)
        g.warmstart()
        g.step(3)
        res[tile] = g.V()
        g.close()
    worst = max(rel(res[t][b], res[1][b]) for t in (2, 3, 4, 5) for b in range(len(insts)))
    print(f"gemm tiles: worst relative V difference after 3 iterations {worst:.2e}")
    assert worst <= 1e-5


@pytest.mark.gpu
def test_tune_on_the_gpu(tmp_path):
    import __graft_entry__ as ge
    ge.build()
    e = autotune.tune((1, 8, 32, 2, 2), "fp32", cache=str(tmp_path / "t.json"), n=304, iters=4)
    print("autotune (1, 8, 32, 2, 2):", e)
    assert e["overrides"] in autotune.CLASSES["fp32"] and e["ms"] > 0
    opts = autotune.tuned_opts((1, 8, 32, 2, 2), "fp32", cache=str(tmp_path / "t.json"))
    assert opts.gemm_tile == e["overrides"]["gemm_tile"]
