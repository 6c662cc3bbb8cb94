"""Autotuner for the solver's launch configuration.

For one instance shape (C, K, Nt, Nr, d) and an accuracy class it times
every configuration of the library that gives that accuracy on a seeded
synthetic batch of that shape, keeps the fastest, and caches the choice in
a JSON file keyed by GPU, shape and class.  Accuracy classes and their
candidates:

  "fp32"    FP32-level GEMMs: the FP32 FFMA path with each register tile of
            its block GEMMs (gemm_tile 1: 4x4, 2: 2x2, 3: 4x2, 4: 4x3,
            5: 2x5; 0: the library's own pick by shape), and the
            tensor-core path with the six-product bf16 split (BF16X6), which
            computes the same GEMMs to FP32 accuracy;
  "bf16x3"  the tensor-core path with the three-product split;
  "bf16"    the tensor-core path with plain bf16 operands.

Every candidate keeps the caller's other options (FP64 solves, step rule,
...).  The timing runs on the device with CUDA events around amm_step.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Tuple

import numpy as np

from .amm import Opts, Solver, default_opts

CLASSES = {
    "fp32": [dict(precision="fp32", gemm_tile=t) for t in (0, 1, 2, 3, 4, 5)] +
            [dict(precision="bf16x6", gemm_tile=0)],
    "bf16x3": [dict(precision="bf16x3", gemm_tile=0)],
    "bf16": [dict(precision="bf16", gemm_tile=0)],
}

DEFAULT_CACHE = os.environ.get("AMM_TUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "amm_autotune.json"))


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def _key(dims: Tuple[int, int, int, int, int], cls: str, extra: Dict) -> str:
    name = _device_name().replace(" ", "_")
    ex = ",".join(f"{k}={v}" for k, v in sorted(extra.items()))
    return f"{name}|{'x'.join(map(str, dims))}|{cls}|{ex}"


def _synthetic(dims, n, seed):
    """Seeded i.i.d. CN(0,1) channels and start points of one shape (sigma2 =
    1, alpha = 1, P = 100), in the C-ABI layouts."""
    C, K, Nt, Nr, d = dims
    g = np.random.default_rng(seed)

    def cn(*shape):
        return ((g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)
    return (cn(n * C * C * K * Nr * Nt), np.ones(n * C * K, np.float32), np.ones(n * C * K, np.float32),
            np.full(n * C, 100.0, np.float32), cn(n * C * Nt * K * d))


def time_config(dims, overrides: Dict, base: Optional[Dict] = None, n: int = 1216, iters: int = 10,
                reps: int = 3, seed: int = 7) -> float:
    """Milliseconds for amm_step(iters) on n instances (best of reps)."""
    import torch
    H, al, s2, P, V0 = (torch.from_numpy(x).to("cuda:0") for x in _synthetic(dims, n, seed))
    s = Solver(n, dims, **{**(base or {}), **overrides})
    s.set_problem(H, al, s2, P)
    best = float("inf")
    for _ in range(reps + 1):
        s.warmstart(V0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        s.step(iters)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    s.close()
    return best


def tune(dims, cls: str = "fp32", base: Optional[Dict] = None, cache: Optional[str] = DEFAULT_CACHE,
         n: int = 1216, iters: int = 10, refresh: bool = False) -> Dict:
    """The fastest configuration of class ``cls`` for shape ``dims``:
    {"overrides": {...}, "ms": ..., "timings": [...]} (from the cache unless
    ``refresh``).  ``base`` holds the caller's fixed options."""
    if cls not in CLASSES:
        raise KeyError(f"unknown accuracy class {cls}")
    base = dict(base or {})
    key = _key(tuple(dims), cls, base)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
    if not refresh and key in table:
        return table[key]
    timings = []
    for cand in CLASSES[cls]:
        timings.append({"overrides": cand, "ms": time_config(dims, cand, base, n=n, iters=iters)})
    best = min(timings, key=lambda r: r["ms"])
    entry = {"overrides": best["overrides"], "ms": best["ms"], "timings": timings}
    if cache:
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        table[key] = entry
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1)
        os.replace(tmp, cache)
    return entry


def tuned_opts(dims, cls: str = "fp32", base: Optional[Dict] = None, **kw) -> Opts:
    """Options for Solver(...) with the tuned configuration applied."""
    entry = tune(dims, cls, base, **kw)
    return default_opts(**{**(base or {}), **entry["overrides"]})
