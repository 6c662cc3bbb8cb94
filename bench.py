#!/usr/bin/env python3
"""Throughput of the batched A-MMMSE solver on GB300.

Workload (one "step"): the single-cell P-sweep batch -- Nt=64 BS antennas,
K=16 users, Nr=4 receive antennas, d=4 streams, i.i.d. CN(0,1) channels,
sigma^2=1, alpha~U(0.5,1.5), P = 0..30 dB in 5 dB steps x 1024 realizations
= 7168 instances -- solved end to end: initial projection, 50 iterations of
Algorithm 3 (two-stage warm start included) and the FP64 WSR evaluation.
Metric: instance-solves/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32]
    python bench.py --impl reference      # the FP64 CPU oracle on host cores

Under torchrun every rank solves its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "instance-solves/s at <=1e-3 WSR gap to FP64 oracle vs plain path; % roofline"
UNIT = "instance-solves/s"
ITERS = 50
N_PER_P = 1024
HEX7_N, HEX7_ITERS = 256, 50
UNEVEN_N, UNEVEN_ITERS = 4096, 30
WMMSE_N, WMMSE_ITERS = 1024, 10
SOLVES = {"fp64": 1, "ff": 2, "fp32": 0}
SOLVE_NAMES = {"fp64": "f64", "ff": "f32x2 (float-float, about 48-bit significands)", "fp32": "f32"}
WORKLOAD = "single-cell P sweep: Nt=64, K=16, Nr=4, d=4, iid CN(0,1), P=0..30 dB (7x1024 instances), 50 iterations"


def algorithmic_gemm_flops(C, K, Nt, Nr, d):
    """Flops of the two complex GEMMs of one iteration of one instance:
    Z = H V and G = H^H Y, each (C K Nr) x Nt x (K d) per cell, 8 real
    flops per complex multiply-add."""
    m, n = C * K * Nr, K * d
    return 2 * 8 * m * Nt * n * C


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per instance of
# the iteration kernels, from the ncu captures summarised in profiles/
# (tc_iterate_kernel: 4864 instances of the single-cell shape, 50 iterations;
# cluster_iterate_kernel: 160 seven-cell instances, 50 iterations; traffic
# grows with the instance count, so a full launch is this times its
# instances).  Valid only for the kernel sources the captures ran: see
# kernel_digest().  Kernels without an entry report null.
TRAFFIC = {"digest": "57f30d916a58a20f",
           "tc_iterate_kernel": (486.432256e6 + 283.902976e6) / 4864,
           "cluster_iterate_kernel": (186.953984e6 + 47.981568e6) / 160}
# pipe utilisation of the same captures (% of peak, ncu --set full), reported
# beside the roofline while the sources match the digest: which unit is busy
PIPES = {"tc_iterate_kernel": {"tensor_pct": 5.78, "fp64_pct": 0.34, "fma_pct": 19.09, "alu_pct": 23.19,
                               "dram_pct": 0.22, "issue_active_pct": 37.85},
         "cluster_iterate_kernel": {"tensor_pct": 0.0, "fp64_pct": 0.28, "fma_pct": 30.31, "alu_pct": 16.21,
                                    "dram_pct": 0.10, "issue_active_pct": 45.62}}


# the sources the iteration kernels and their launches are built from
DIGEST_SOURCES = ("amm_capi.cu", "amm_device.cuh", "amm_internal.cuh", "amm_solver.cu", "amm_tc.cu", "amm_tc.cuh",
                  "amm_cluster.cu", "amm_ff.cuh")


def kernel_digest():
    """First 16 hex digits of the sha256 over the iteration kernels' sources."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2510_20507_gb300", "csrc")
    h = hashlib.sha256()
    for f in DIGEST_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def rank_base_seed(rank):
    """Each rank solves its own disjoint set of instances (weak scaling)."""
    return 2 + 1000 * rank


def max_over_ranks(value, dist, device=None):
    """Max of a per-rank float over the process group (identity without one)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, per_rank_units, steps, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return world * per_rank_units * steps / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def fp32_peak_tflops(sm_mhz):
    """FP32 FFMA peak: 152 SMs x 128 FP32 lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle
def _round32(inst):
    """The inputs as the GPU receives them (complex64 / float32)."""
    import numpy as np
    inst.H = inst.H.astype(np.complex64).astype(np.complex128)
    inst.G0 = inst.G0.astype(np.complex64).astype(np.complex128)
    inst.alpha = inst.alpha.astype(np.float32).astype(np.float64)
    inst.sigma2 = inst.sigma2.astype(np.float32).astype(np.float64)
    inst.P = inst.P.astype(np.float32).astype(np.float64)
    return inst


def _instances(name, first, count):
    """Instances [first, first+count) of a named workload."""
    import workloads as wl
    if name == "hex7":
        return wl.hex7(n=HEX7_N, first=first, count=count)
    if name == "uneven":
        return wl.uneven(n=UNEVEN_N, first=first, count=count)
    if name == "wmmse":
        return wl.unrolled_64(n=WMMSE_N, first=first, count=count)
    return wl.single_cell_64(N_PER_P, first=first, count=count)


def _oracle_worker(args):
    """Oracle solves of instances [first, first+count) of a workload (the
    timed sweep unless a name is given): (index, oracle.parity.Reference:
    the final WSR in bits of the oracle's trajectory and, where a stage
    decision came within 1e-4 of eps1, of each other admissible one)."""
    first, count, iters = args[:3]
    name = args[3] if len(args) > 3 else "sweep"
    from oracle import parity as op
    return [(first + k, op.reference_solves(_round32(inst), iters))
            for k, inst in enumerate(_instances(name, first, count))]


def _judge_worker(args):
    """oracle.parity.judge of one GPU result beyond the 1e-3 gap (computes
    the oracle's FP32 spread for it)."""
    b, got, ref, iters = args[:4]
    name = args[4] if len(args) > 4 else "sweep"
    from oracle import parity as op
    return op.judge(got, ref, _round32(_instances(name, b, 1)[0]), iters)


def _wmmse_worker(args):
    """The oracle's plain WMMSE (Algorithm 2, bisection to width 1e-4, at
    most 100 halvings) on one instance of the WMMSE workload: (index, WSR in
    bits after the iterations)."""
    import math
    from oracle import solvers as osv
    b, iters = args
    inst = _round32(_instances("wmmse", b, 1)[0])
    V0 = osv.initial_precoder(inst.G0, inst.P)
    _, hist, _ = osv.wmmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, iters,
                           tol=1e-4, max_bisect=100)
    return b, hist[-1] / math.log(2.0)


def _oracle_serial(jobs):
    """Several oracle jobs one after the other in one worker (one core)."""
    return [x for j in jobs for x in _oracle_worker(j)]


def _pool_init(barrier):
    """Worker start-up: import what the oracle workers use, then wait until
    every worker has done so (a worker that starts later gives up waiting
    after a minute)."""
    import threading
    import numpy  # noqa: F401
    from oracle import parity  # noqa: F401
    import workloads  # noqa: F401
    try:
        barrier.wait(timeout=60)
    except threading.BrokenBarrierError:
        pass


def make_pool(cores):
    """A spawn pool of oracle workers (spawned before the first CUDA call),
    returned once every worker has finished its imports, so that no worker
    is still importing on a host core while the GPU is timed."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores + 1)
    pool = ctx.Pool(cores, initializer=_pool_init, initargs=(barrier,))
    try:
        barrier.wait(timeout=600)
    except Exception:
        pass
    return pool


def oracle_solve(pool, indices):
    """Oracle solves of the given workload instances over the pool; returns
    (results, seconds)."""
    jobs = [(b, 1, ITERS) for b in indices]
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, jobs, chunksize=max(1, len(jobs) // (8 * (os.cpu_count() or 1))))
    return [x for r in res for x in r], time.perf_counter() - t0


def oracle_throughput(pool, cores, n_instances, offset=0):
    """Solve n_instances of the workload with the oracle over the pool;
    returns (instance-solves/s, seconds, instances)."""
    total = 7 * N_PER_P
    res, dt = oracle_solve(pool, [(offset + k) % total for k in range(n_instances)])
    return len(res) / dt, dt, len(res)


def gap_check(pool, got, oracle_res, name="sweep", iters=None):
    """The WSR gap of the GPU's solves to the oracle's on the oracle's
    sample, every instance judged by oracle.parity: within 1e-3 of the
    nearest admissible oracle trajectory passes; beyond it, a gap of at most
    4 x the oracle's own spread under FP32-sized perturbations of its
    arithmetic passes as FP32-sensitive, anything more fails."""
    import numpy as np
    from oracle import parity as op
    near = [(b, ref) + op.nearest(float(got[b]), ref)[1:] for b, ref in oracle_res]
    gaps = np.array([g for _, _, g, _ in near])
    signed = np.array([sg for _, _, _, sg in near])
    beyond = [(b, ref) for b, ref, g, _ in near if g > op.GAP_TOL]
    verdicts = (pool.map(_judge_worker, [(b, float(got[b]), ref, iters or ITERS, name) for b, ref in beyond],
                         chunksize=1) if beyond else [])
    ratios = [v.gap / max(v.spread, 1e-300) for v in verdicts]
    failed = sum(not v.ok for v in verdicts)
    return {"rule": f"gap <= {op.GAP_TOL:g}, else gap <= {op.SPREAD_FACTOR:g} x the oracle's FP32 spread; "
                    f"stage decisions within {op.SWITCH_MARGIN:g} of eps1 compared with every admissible "
                    f"trajectory",
            "checked": len(near), "ambiguous_switch": sum(len(ref.wsr) > 1 for _, ref in oracle_res),
            "max_wsr_gap": float(gaps.max()) if len(gaps) else None,
            "p99_wsr_gap": float(np.percentile(gaps, 99)) if len(gaps) else None,
            "median_wsr_gap": float(np.median(gaps)) if len(gaps) else None,
            # mean of (GPU - oracle) / oracle: whether the sample leans to one side
            "mean_signed_wsr_gap": float(signed.mean()) if len(gaps) else None,
            "within_1e-3": int(np.sum(gaps <= op.GAP_TOL)),
            "over_1e-3": len(beyond), "over_1e-3_fp32_sensitive": len(verdicts) - failed, "failed": failed,
            "all_pass": failed == 0,
            "over_1e-3_max_gap_over_spread": float(max(ratios)) if ratios else None}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    pool = make_pool(cores)
    # warm-up (imports in the workers)
    oracle_throughput(pool, cores, cores)
    vals, n_total, t_total = [], 0, 0.0
    per_step = max(cores, 2 * cores)
    for s in range(args.warmup):
        oracle_throughput(pool, cores, per_step, offset=s * per_step)
    for s in range(args.steps):
        v, dt, n = oracle_throughput(pool, cores, per_step, offset=(args.warmup + s) * per_step)
        vals.append(v)
        n_total += n
        t_total += dt
    pool.close()
    value = n_total / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_step": per_step, "iterations": ITERS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} instances per step of the same workload, numpy float64 oracle, "
                                   f"one process per core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_e2e(solver, pk, batch, args, dist, dev, world):
    """The same metric through the host-buffer API: host (pinned) inputs
    copied in and the WSR copied out inside the timed region.  ``solver``
    is a Solver (amm_solve_host on one context) or a HostPipeline (one
    context and stream per part of the batch, copies overlapping solves)."""
    import torch
    Hh = torch.from_numpy(pk.H).pin_memory()
    G0h = torch.from_numpy(pk.G0).pin_memory()
    ah = torch.from_numpy(pk.alpha).pin_memory()
    sh = torch.from_numpy(pk.sigma2).pin_memory()
    Ph = torch.from_numpy(pk.P).pin_memory()
    wsr_h = torch.empty(batch, dtype=torch.float64).pin_memory()
    solver.solve_host(Hh, ah, sh, Ph, G0h, ITERS, wsr_h)  # warm-up (allocates its input buffers)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve_host(Hh, ah, sh, Ph, G0h, ITERS, wsr_h)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    h2d = pk.H.nbytes + pk.G0.nbytes + pk.alpha.nbytes + pk.sigma2.nbytes + pk.P.nbytes
    return whole_job_rate(world, batch, args.steps, e2e_s), h2d, batch * 8, wsr_h.numpy().copy()


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = make_pool(cores)  # spawned before the first CUDA call

    import torch
    import workloads as wl
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    dev = torch.device("cuda", local)

    # inputs of this rank (rank r uses a disjoint seed range)
    insts = wl.single_cell_64(N_PER_P, base_seed=rank_base_seed(rank))
    if args.instances:
        # an evenly spread subset of the batch (all seven P values), for profiling
        step = max(1, len(insts) // args.instances)
        insts = insts[::step][:args.instances]
    pk = wl.pack(insts)
    batch = len(insts)
    C, K, Nt, Nr, d = pk.dims[0]
    stream = torch.cuda.Stream(device=dev)
    opts = pkg.default_opts(precision=args.precision, fp64_solves=SOLVES[args.solves])
    if args.smem_budget:
        opts.smem_budget = args.smem_budget
    solver = pkg.Solver(batch, pk.dims[0], opts=opts, stream=stream)
    H = torch.from_numpy(pk.H).to(dev)
    G0 = torch.from_numpy(pk.G0).to(dev)
    alpha = torch.from_numpy(pk.alpha).to(dev)
    sigma2 = torch.from_numpy(pk.sigma2).to(dev)
    P = torch.from_numpy(pk.P).to(dev)
    wsr = torch.empty(batch, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    ev_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]

    def one_step(pair=None):
        solver.set_problem(H, alpha, sigma2, P)
        solver.warmstart(G0)
        if pair is not None:
            pair[0].record(stream)
        solver.step(ITERS)
        if pair is not None:
            pair[1].record(stream)
        solver.wsr(wsr)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = solver.launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for s in range(args.steps):
            step_ev[s].record(stream)
            one_step(ev_pairs[s])
        step_ev[args.steps].record(stream)
        ev1.record(stream)
    torch.cuda.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    step_ms = [a.elapsed_time(b) for a, b in zip(step_ev, step_ev[1:])]
    launches = solver.launches - l0
    # duration of each launch of the iteration kernel, from events on its stream
    iter_ms = [a.elapsed_time(b) for a, b in ev_pairs]
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    value = whole_job_rate(world, batch, args.steps, elapsed_ms / 1000.0)

    # ---- the plain FP32 GEMM path on the same inputs, timed the same way
    plain = None
    if args.precision != "fp32" and not args.no_plain:
        popts = pkg.default_opts(precision="fp32", fp64_solves=opts.fp64_solves)
        psolver = pkg.Solver(batch, pk.dims[0], opts=popts, stream=stream)

        def plain_step():
            psolver.set_problem(H, alpha, sigma2, P)
            psolver.warmstart(G0)
            psolver.step(ITERS)
            psolver.wsr(wsr)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                plain_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            p0.record(stream)
            for _ in range(args.steps):
                plain_step()
            p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(p0.elapsed_time(p1), dist, dev)
        pval = whole_job_rate(world, batch, args.steps, pms / 1000.0)
        plain = {"precision": "fp32", "value": pval, "unit": UNIT, "ms_per_step": pms / args.steps}
        psolver.close()
        # restore this step's result for the parity sample below
        with torch.cuda.stream(stream):
            one_step()
        torch.cuda.synchronize()

    # ---- the same tensor-core path with FP64 per-user solves, timed the same way
    fp64_leg = None
    if args.solves != "fp64" and not args.no_plain:
        fopts = pkg.default_opts(precision=args.precision, fp64_solves=SOLVES["fp64"])
        fsolver = pkg.Solver(batch, pk.dims[0], opts=fopts, stream=stream)

        def fp64_step():
            fsolver.set_problem(H, alpha, sigma2, P)
            fsolver.warmstart(G0)
            fsolver.step(ITERS)
            fsolver.wsr(wsr)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fp64_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            f0.record(stream)
            for _ in range(args.steps):
                fp64_step()
            f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        fp64_leg = {"small_solves": "f64", "value": whole_job_rate(world, batch, args.steps, fms / 1000.0),
                    "unit": UNIT, "ms_per_step": fms / args.steps}
        fsolver.close()
        with torch.cuda.stream(stream):
            one_step()
        torch.cuda.synchronize()

    # ---- end to end through the C-ABI with host buffers (pinned)
    e2e_value, h2d, d2h, e2e_single = None, 0, 0, None
    if not args.no_e2e:
        # HostPipeline: the batch in parts, each on its own context and stream,
        # so each part's upload overlaps the solves of the others
        pipe = pkg.HostPipeline(batch, pk.dims[0], chunks=args.e2e_chunks, opts=opts)
        e2e_value, h2d, d2h, wsr_pipe = run_e2e(pipe, pk, batch, args, dist, dev, world)
        pipe.close()
        e2e_single, _, _, wsr_one = run_e2e(solver, pk, batch, args, dist, dev, world)
        if not np.array_equal(wsr_pipe, wsr_one):  # same instances, same kernels: identical results
            raise RuntimeError("HostPipeline and amm_solve_host disagree")
    st = torch.empty(batch, dtype=torch.int32, device=dev)
    solver.status(st)
    torch.cuda.synchronize()
    n_bad_status = int((st != 0).sum().item())
    got = wsr.cpu().numpy()

    # ---- roofline of the dominant kernel (the fused iteration kernel)
    peaks, src = measured_peaks()
    flops_launch = algorithmic_gemm_flops(C, K, Nt, Nr, d) * ITERS * batch
    avg_iter_ms = statistics.mean(iter_ms)
    achieved = flops_launch / (avg_iter_ms / 1000.0) / 1e12
    kname = "iterate_kernel" if args.precision == "fp32" else "tc_iterate_kernel"
    same_sources = kernel_digest() == TRAFFIC["digest"]
    traffic = TRAFFIC[kname] * batch if same_sources and kname in TRAFFIC else None
    if args.precision == "fp32":
        peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "iterate_kernel",
                "peak_note": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                             f"(derived from the unit counts and the maximum clock, not measured; {src} clocks)"}
    else:
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "tc_iterate_kernel", "peak_note": f"bf16 burst, {src}"}
    roof["ncu_pipes"] = PIPES.get(kname) if same_sources else None

    # ---- the CPU baseline: the oracle on a sample of this batch (every
    #      stride-th instance, all seven P values), timed; its results are
    #      also the reference for the WSR gap of the GPU's solves
    cpu, parity = None, {"bad_status": n_bad_status}
    if pool is not None:
        stride = max(1, batch // args.oracle_sample) if not args.instances else 1
        idx = list(range(0, batch, stride))[:args.oracle_sample] if not args.instances else None
        if args.instances:  # a profiling subset: the instances it holds
            step = max(1, 7 * N_PER_P // args.instances)
            idx = list(range(0, 7 * N_PER_P, step))[:batch]
            pos = {b: k for k, b in enumerate(idx)}
        else:
            pos = {b: b for b in idx}
        res, dt = oracle_solve(pool, idx)
        cpu = {"value": len(res) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(res)} instances of the batch (every {stride if not args.instances else 1}-th, "
                         f"all seven P values), numpy float64 oracle, {ITERS} iterations each, one process per "
                         f"core, {dt:.1f} s"}
        parity.update(gap_check(pool, {b: got[pos[b]] for b in idx}, res))
        # the same oracle on one core, on a smaller part of the sample
        one = idx[::max(1, len(idx) // args.oracle_one_core)][:args.oracle_one_core]
        if one:
            t0 = time.perf_counter()
            n1 = len(pool.apply(_oracle_serial, ([(b, 1, ITERS) for b in one],)))
            dt1 = time.perf_counter() - t0
            cpu["one_core"] = {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                               "sample": f"{n1} of those instances in one process, {dt1:.1f} s"}
        pool.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": batch, "iterations": ITERS,
                   "precision": args.precision, "small_solves": SOLVE_NAMES[args.solves],
                   "l2": "inputs larger than L2 (H: %.0f MB per GPU)" % (pk.H.nbytes / 1e6)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "api": f"HostPipeline, {args.e2e_chunks} parts (amm_solve_host per part)",
                 "single_context": e2e_single}
                if e2e_value is not None else None),
        "gpu_launches": launches,
        "clocks": clk,
        "iterate_kernel_ms": avg_iter_ms,
        # per timed step (CUDA events at the step boundaries, this rank)
        "ms_per_step_best": min(step_ms),
        "ms_per_step_median": statistics.median(step_ms),
        "plain_path": plain,
        "speedup_vs_plain": (value / plain["value"]) if plain else None,
        "fp64_solves": fp64_leg,
        "parity": parity,
    }
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _unrolled_worker(args):
    """Oracle forward of the unrolled map (oracle.solvers.ammmse_unrolled) on
    one instance of the unrolled workload: (index, WSR(V^T) in bits)."""
    b, n, T, sw, gam = args
    import numpy as np
    import workloads as wl
    from oracle import solvers as osv
    inst = _round32(wl.unrolled_64(n=n, first=b, count=1)[0])
    V0 = osv.initial_precoder(inst.G0, inst.P)
    g = float(np.float32(gam))
    return b, osv.ammmse_unrolled(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, [g] * T,
                                  switch_iter=sw)[1]


def run_unrolled(args):
    """The differentiable unrolled workload: 1024 instances of Nt=64, K=16,
    Nr=2, d=2 at 20 dB, T=20 iterations, checkpoints every 5, forward
    (WSR) plus the hand-written adjoint (gradients in every gamma_t and in
    H) per step.  Metric: instance-gradients/s (one JSON line)."""
    pool, cores = None, os.cpu_count() or 1
    if not args.no_cpu_baseline:
        pool = make_pool(cores)  # spawned before the first CUDA call
    import numpy as np
    import torch
    import workloads as wl
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    from paper_2510_20507_gb300.unrolled import unrolled_wsr
    T, ck, sw, n = 20, 5, 4, args.instances or 1024
    insts = wl.unrolled_64(n=n)
    dev = torch.device("cuda", 0)
    H = torch.from_numpy(np.stack([i.H[0] for i in insts]).astype(np.complex64)).to(dev).requires_grad_(True)
    al = torch.from_numpy(np.stack([i.alpha for i in insts]).astype(np.float32)).to(dev)
    s2 = torch.from_numpy(np.stack([i.sigma2 for i in insts]).astype(np.float32)).to(dev)
    P = torch.from_numpy(np.array([i.P[0] for i in insts], dtype=np.float32)).to(dev)
    G0 = np.stack([i.G0[0] for i in insts]).astype(np.complex64)
    scale = np.sqrt(np.minimum(1.0, P.cpu().numpy() / (np.abs(G0) ** 2).sum(axis=(1, 2))))
    V0 = torch.from_numpy((G0 * scale[:, None, None]).astype(np.complex64)).to(dev)  # eq. (15) projection
    gam = torch.full((T,), 0.004, dtype=torch.float32, device=dev, requires_grad=True)
    solver = pkg.UnrolledSolver(n, (1, 16, 64, 2, 2), T, ckpt_every=ck, switch_iter=sw)

    def step():
        H.grad = None
        gam.grad = None
        unrolled_wsr(solver, H, gam, al, s2, P, V0).sum().backward()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # roofline: algorithmic flops of a forward + adjoint step = per iteration
    # the two forward GEMMs (Z = H V, G = H^H Y) and the two adjoint products
    # of each (C = A B: Abar = Cbar B^H, Bbar = A^H Cbar), six GEMMs of
    # (K Nr) x Nt x (K d) complex multiply-adds, against the FP32 FFMA peak
    peaks, src = measured_peaks()
    flops = 3 * algorithmic_gemm_flops(1, 16, 64, 2, 2) * T * n
    achieved = flops / (ms / args.steps / 1000.0) / 1e12
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "u_forward_kernel + u_backward_kernel",
            "peak_note": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                         f"(derived from the unit counts and the maximum clock, not measured; {src} clocks)"}
    # the CPU baseline: the oracle's forward of the unrolled map on a sample
    # (the oracle has no adjoint; the gradients are checked in the tests
    # against FP64 finite differences and a float64 autograd restatement),
    # timed, and the reference of the forward WSR gap
    cpu, parity = None, None
    if pool is not None:
        with torch.no_grad():
            got = unrolled_wsr(solver, H.detach(), gam.detach(), al, s2, P, V0).cpu().numpy()
        idx = list(range(0, n, max(1, n // 64)))[:64]
        t0 = time.perf_counter()
        res = pool.map(_unrolled_worker, [(b, n, T, sw, 0.004) for b in idx], chunksize=1)
        dt = time.perf_counter() - t0
        pool.close()
        gaps = np.array([(got[b] - w) / w for b, w in res])
        cpu = {"value": len(res) / dt, "unit": "instance-forwards/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(res)} instances (every {max(1, n // 64)}-th), forward WSR of the unrolled map only "
                         f"(the oracle has no adjoint), numpy float64, one process per core, {dt:.1f} s"}
        parity = {"forward_wsr_checked": len(res), "max_abs_gap": float(np.abs(gaps).max()),
                  "median_abs_gap": float(np.median(np.abs(gaps))), "mean_signed_gap": float(gaps.mean()),
                  "within_1e-3": int(np.sum(np.abs(gaps) <= 1e-3))}
    print(json.dumps({"metric": "instance-gradients/s (unrolled A-MMMSE, forward + adjoint)",
                      "value": n * args.steps / (ms / 1000.0), "unit": "instance-gradients/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "unrolled: Nt=64, K=16, Nr=2, d=2, P=20 dB, T=20, checkpoints every 5, "
                                             "stage II from iteration 4", "instances": n},
                      "roofline": roof, "clocks": clk, "cpu_baseline": cpu, "parity": parity}))
    solver.close()
    return 0


def run_other(args):
    """Solve throughput of the other workloads (one JSON line, FP32-GEMM path
    unless --precision says otherwise): hex7 = 256 seven-cell instances
    (Nt=128, K=10, Nr=2, d=2, path loss and shadowing), 50 iterations;
    uneven = 4096 single-cell instances of mixed sizes in one launch
    (longest first), 30 iterations.  With the CPU-baseline leg the oracle
    solves an evenly spread sample of the batch on the host cores, timed,
    and its WSR is the reference for the gap of the GPU's solves."""
    pool, cores = None, os.cpu_count() or 1
    if not args.no_cpu_baseline:
        pool = make_pool(cores)  # spawned before the first CUDA call
    import torch
    import workloads as wl
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    name = args.workload
    if name == "hex7":
        insts, iters, desc = wl.hex7(n=HEX7_N), HEX7_ITERS, "seven hexagonal cells, Nt=128, K=10, Nr=2, d=2, 256 instances"
        sample_n = 32
    else:
        insts, iters, desc = wl.uneven(n=UNEVEN_N), UNEVEN_ITERS, ("uneven single-cell batch: Nt 16..256, K 4..64, "
                                                                "Nr 1/2/4, 4096")
        sample_n = 128
    if args.instances:  # an evenly spread subset (profiling runs)
        insts = insts[::max(1, len(insts) // args.instances)][:args.instances]
    pk = wl.pack(insts)
    dims = pk.dims[0] if pk.uniform else pk.dims
    prec = args.precision if args.precision != "bf16x6" else "fp32"  # tensor-core path: single cell, Nt <= 64 only
    dev = torch.device("cuda", 0)
    s = pkg.Solver(len(insts), dims, precision=prec, fp64_solves=SOLVES[args.solves])
    path = s.path
    H, G0 = torch.from_numpy(pk.H).to(dev), torch.from_numpy(pk.G0).to(dev)
    al, s2, P = (torch.from_numpy(x).to(dev) for x in (pk.alpha, pk.sigma2, pk.P))
    wsr = torch.empty(len(insts), dtype=torch.float64, device=dev)

    def step():
        s.set_problem(H, al, s2, P)
        s.warmstart(G0)
        s.step(iters)
        s.wsr(wsr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    got = wsr.cpu().numpy()
    st = torch.empty(len(insts), dtype=torch.int32, device=dev)
    s.status(st)
    n_bad = int((st != 0).sum().item())
    s.close()
    # the uneven batch also under the persistent schedule (device queue, longest first)
    persistent = None
    if name == "uneven":
        s = pkg.Solver(len(insts), dims, precision=prec, fp64_solves=SOLVES[args.solves], schedule=1)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record()
        for _ in range(args.steps):
            step()
        q1.record()
        torch.cuda.synchronize()
        persistent = {"schedule": "persistent blocks, device queue, longest first",
                      "value": len(insts) * args.steps / (q0.elapsed_time(q1) / 1000.0), "unit": UNIT,
                      "ms_per_step": q0.elapsed_time(q1) / args.steps}
        s.close()

    # roofline: the algorithmic GEMM flops of a whole step (set-up, solve and
    # WSR evaluation all inside it) against the FP32 FFMA peak
    peaks, src = measured_peaks()
    flops = sum(algorithmic_gemm_flops(x.C, x.K, x.Nt, x.Nr, x.d) for x in insts) * iters
    achieved = flops / (ms / args.steps / 1000.0) / 1e12
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    kname = "cluster_iterate_kernel" if path == "cluster" else "iterate_kernel"
    same_sources = kernel_digest() == TRAFFIC["digest"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC[kname] * len(insts) if same_sources and kname in TRAFFIC else None,
            "ncu_pipes": PIPES.get(kname) if same_sources else None, "kernel": kname,
            "peak_note": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                         f"(derived from the unit counts and the maximum clock, not measured); "
                         f"achieved over the whole step"}

    cpu, parity = None, {"bad_status": n_bad}
    if pool is not None:
        stride = max(1, len(insts) // sample_n)
        idx = list(range(0, len(insts), stride))[:sample_n]
        t0 = time.perf_counter()
        res = [x for r in pool.map(_oracle_worker, [(b, 1, iters, name) for b in idx], chunksize=1) for x in r]
        dt = time.perf_counter() - t0
        cpu = {"value": len(res) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(res)} instances of the batch (every {stride}-th), numpy float64 oracle, {iters} "
                         f"iterations each, one process per core, {dt:.1f} s"}
        parity.update(gap_check(pool, {b: got[b] for b in idx}, res, name=name, iters=iters))
        pool.close()
    print(json.dumps({"metric": "instance-solves/s", "value": len(insts) * args.steps / (ms / 1000.0),
                      "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms / args.steps, "higher_is_better": True, "dtype": prec, "data": "synthetic",
                      "config": {"workload": desc, "iterations": iters, "small_solves": SOLVE_NAMES[args.solves],
                                 "kernel": path},
                      "roofline": roof, "cpu_baseline": cpu, "parity": parity, "clocks": clk,
                      "persistent_schedule": persistent}))
    return 0


def run_wmmse(args):
    """Plain WMMSE (Algorithm 2) on the GPU, the comparison method of the
    paper: 1024 single-cell instances (Nt=64, K=16, Nr=2, d=2, 20 dB), 10
    iterations per solve, the V update of eq. (12) by the Jacobi
    eigen-decomposition of A_k (amm_wmmse_step_eig; timed) and by a Cholesky
    factorisation per bisection point (amm_wmmse_step; timed beside it).
    The CPU-baseline leg runs the oracle's WMMSE on a sample, timed, and its
    WSR is the reference for the gap."""
    pool, cores = None, os.cpu_count() or 1
    if not args.no_cpu_baseline:
        pool = make_pool(cores)  # spawned before the first CUDA call
    import numpy as np
    import torch
    import workloads as wl
    import __graft_entry__ as ge
    ge.build()
    import paper_2510_20507_gb300 as pkg
    insts = wl.unrolled_64(n=WMMSE_N)
    if args.instances:
        insts = insts[::max(1, len(insts) // args.instances)][:args.instances]
    iters = WMMSE_ITERS
    pk = wl.pack(insts)
    dev = torch.device("cuda", 0)
    H, G0 = torch.from_numpy(pk.H).to(dev), torch.from_numpy(pk.G0).to(dev)
    al, s2, P = (torch.from_numpy(x).to(dev) for x in (pk.alpha, pk.sigma2, pk.P))
    wsr = torch.empty(len(insts), dtype=torch.float64, device=dev)

    def timed(eig):
        s = pkg.Solver(len(insts), pk.dims[0], precision="fp32")

        def step():
            s.set_problem(H, al, s2, P)
            s.warmstart(G0)
            s.wmmse_step(iters, 1e-4, 100, eig=eig)
            s.wsr(wsr)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        st = torch.empty(len(insts), dtype=torch.int32, device=dev)
        s.status(st)
        bad = int((st != 0).sum().item())
        got = wsr.cpu().numpy()
        s.close()
        return e0.elapsed_time(e1), clk, bad, got

    ms, clk, n_bad, got = timed(True)
    ms_chol, _, bad_chol, got_chol = timed(False)
    peaks, src = measured_peaks()
    x = insts[0]
    m, n, Nt = x.K * x.Nr, x.K * x.d, x.Nt
    # the GEMM-shaped work of one iteration per instance: Z = H V, A = H^H (D H), the
    # two products with Q (Q^H B and Q Y) and the Jacobi rotations counted as
    # 24 Nt^3 flops per sweep for six sweeps (the measured typical count)
    flops = (8 * m * Nt * n + 8 * Nt * Nt * m + 2 * 8 * Nt * Nt * n + 6 * 24 * Nt ** 3) * iters * len(insts)
    achieved = flops / (ms / args.steps / 1000.0) / 1e12
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "wmmse_kernel (eig)",
            "peak_note": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                         f"(derived, not measured); achieved over the whole step, nominal flops"}
    cpu, parity = None, {"bad_status": n_bad + bad_chol}
    if pool is not None:
        sample_n = 32
        stride = max(1, len(insts) // sample_n)
        idx = list(range(0, len(insts), stride))[:sample_n]
        t0 = time.perf_counter()
        res = pool.map(_wmmse_worker, [(b, iters) for b in idx], chunksize=1)
        dt = time.perf_counter() - t0
        cpu = {"value": len(res) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(res)} instances (every {stride}-th), the oracle's WMMSE, {iters} iterations each, "
                         f"one process per core, {dt:.1f} s"}
        gaps = np.array([abs(got[b] - w) / w for b, w in res])
        gaps_c = np.array([abs(got_chol[b] - w) / w for b, w in res])
        parity.update({"checked": len(res), "max_wsr_gap": float(gaps.max()), "median_wsr_gap": float(np.median(gaps)),
                       "within_1e-3": int(np.sum(gaps <= 1e-3)),
                       "cholesky_max_wsr_gap": float(gaps_c.max()), "cholesky_within_1e-3": int(np.sum(gaps_c <= 1e-3))})
        pool.close()
    print(json.dumps({"metric": "instance-solves/s (plain WMMSE, 10 iterations)",
                      "value": len(insts) * args.steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                      "higher_is_better": True, "dtype": "fp32", "data": "synthetic",
                      "config": {"workload": "WMMSE: Nt=64, K=16, Nr=2, d=2, P=20 dB, 1024 instances",
                                 "iterations": iters, "v_update": "Jacobi eigen-decomposition of A_k"},
                      "roofline": roof, "cpu_baseline": cpu, "parity": parity, "clocks": clk,
                      "cholesky_bisection": {"value": len(insts) * args.steps / (ms_chol / 1000.0), "unit": UNIT,
                                             "ms_per_step": ms_chol / args.steps}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "unrolled", "hex7", "uneven", "wmmse"],
                    help="sweep: the timed P-sweep solve (default); unrolled: the differentiable unrolled workload; "
                         "hex7 / uneven: solve throughput of the seven-cell and mixed-size workloads; wmmse: the "
                         "plain WMMSE comparison method")
    ap.add_argument("--precision", default="bf16x6", choices=["fp32", "bf16", "bf16x3", "bf16x6"])
    ap.add_argument("--smem-budget", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="(kept for compatibility; the gap check rides on "
                    "the CPU-baseline leg, see --no-cpu-baseline)")
    ap.add_argument("--oracle-sample", type=int, default=1024,
                    help="instances of the batch the CPU-baseline leg solves with the oracle (gap reference)")
    ap.add_argument("--oracle-one-core", type=int, default=32,
                    help="instances of that sample solved again in one process (the one-core figure)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=4,
                    help="parts of the batch (contexts and streams) of the end-to-end host-buffer leg")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 path alongside")
    ap.add_argument("--fp32-solves", action="store_true",
                    help="run the per-user Hermitian solves in FP32 instead of FP64")
    ap.add_argument("--solves", default=None, choices=["fp64", "ff", "fp32"],
                    help="arithmetic of the per-user Hermitian solves (default ff = float-float pairs, which "
                         "give the FP64 solves' results on the parity tests; the sweep also times fp64)")
    ap.add_argument("--instances", type=int, default=0,
                    help="solve an evenly spread subset of the batch (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.solves is None:
        args.solves = "fp32" if args.fp32_solves else "ff"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "unrolled":
        return run_unrolled(args)
    if args.workload in ("hex7", "uneven"):
        return run_other(args)
    if args.workload == "wmmse":
        return run_wmmse(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
