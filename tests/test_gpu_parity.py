"""GPU path (through the C-ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances.  The GPU's GEMMs and iterate are FP32, its small Hermitian
solves FP64; the oracle is FP64 throughout.  One iteration from the
oracle's own state (teacher forcing) must reproduce the oracle's V^t within
1e-5 relative Frobenius error, as a whole and for every user's block
(relative to that block or the cell's average block, whichever is larger),
the WSR R^t it computes within 1e-5, the stage, the stage's iteration count
and a frozen step gamma_c (1e-5); a free-running solve must end within 1e-3
relative WSR of the oracle (the accuracy target of the hot path) by the
rule of oracle.parity; the WSR evaluation itself within 1e-6 (FP32 inputs,
FP64 log-det).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import solvers as osv

from gpu_util import (GpuRun, assert_step_bounds, check_free_running, oracle_run, oracle_wsr_bits, rel,
                      round_inputs, spawn_pool, teacher_forced)

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
WSR_TOL = 1e-3
EVAL_TOL = 1e-6

SHAPES = [
    # (C, K, Nt, Nr, d): several register tiles with ragged tails, every (Nr, d) class
    (1, 4, 8, 2, 2),
    (1, 5, 33, 4, 3),
    (2, 3, 17, 3, 2),
    (3, 2, 9, 2, 1),
    (1, 1, 5, 1, 1),
    (1, 7, 40, 4, 4),
    (2, 2, 12, 1, 1),
]


def small_batch(shape, n, seed):
    rng = np.random.default_rng(seed)
    return round_inputs([wl.random_small(rng, *shape) for _ in range(n)])


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


@pytest.mark.parametrize("shape", SHAPES)
def test_wsr_evaluation(shape):
    insts = small_batch(shape, 6, 1000 + sum(shape))
    g = GpuRun(insts)
    g.warmstart()
    got = g.wsr()
    for b, inst in enumerate(insts):
        V0 = osv.initial_precoder(inst.G0, inst.P)
        want = oracle_wsr_bits(inst, V0)
        assert abs(got[b] - want) <= EVAL_TOL * abs(want), (b, got[b], want)
    g.close()


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_initial_projection(shape):
    insts = small_batch(shape, 5, 2000 + sum(shape))
    for inst in insts:
        inst.G0 *= 3.0  # make the projection active on every cell
    g = GpuRun(insts)
    g.warmstart()
    Vs = g.V()
    for b, inst in enumerate(insts):
        want = osv.initial_precoder(inst.G0, inst.P)
        assert rel(Vs[b], want) <= 1e-6
        for k in range(inst.C):
            assert np.sum(np.abs(Vs[b][k].astype(complex)) ** 2) <= inst.P[k] * (1 + 1e-5)
    g.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_teacher_forced_step(shape):
    """Load the oracle's state before iteration t into the GPU, run one
    iteration, compare the state after it (every t of a 12-iteration run:
    stage I, the switch, spectral and frozen steps, extrapolation)."""
    insts = small_batch(shape, 6, 3000 + sum(shape))
    assert_step_bounds(teacher_forced(insts, 12), f"teacher-forced {shape}")


@pytest.mark.parametrize("shape", SHAPES)
def test_free_running(shape):
    n, iters = 8, 30
    insts = small_batch(shape, n, 4000 + sum(shape))
    g = GpuRun(insts)
    g.warmstart()
    g.step(iters)
    got = g.wsr()
    check_free_running(got, insts, iters, f"free-running {shape}")
    g.close()


def test_tiny_fp64_workload_free_running():
    """100 realizations, single cell, Nt=8, K=4, Nr=2, d=2, P=10 dB, 50 iterations."""
    insts = wl.tiny_fp64(100)
    g = GpuRun(insts)
    g.warmstart()
    g.step(50)
    got = g.wsr()
    Vs = g.V()
    g.close()
    check_free_running(got, insts, 50, "tiny")
    verr = [rel(Vs[b], oracle_run(insts[b], 50).V) for b in range(0, 100, 10)]
    print(f"tiny: median V err {np.median(verr):.2e}")


@pytest.mark.parametrize("opt", [dict(step_rule=1), dict(extrapolate=0), dict(switch_iter=1),
                                 dict(step_rule=2, gamma_c=0.02), dict(switch_iter=4, tc=2)])
def test_option_variants(opt):
    """A-WMMSE (switch at t = 1), no extrapolation, spectral step every
    iteration, fixed step, forced switch: same iterates as the oracle."""
    insts = wl.tiny_fp64(12)
    iters = 25
    g = GpuRun(insts, **opt)
    g.warmstart()
    g.step(iters)
    got = g.wsr()
    g.close()
    oopt = {{"tc": "Tc"}.get(k, k): (bool(v) if k == "extrapolate" else v) for k, v in opt.items()}
    check_free_running(got, insts, iters, f"option variant {opt}", opt_kw=oopt)


def test_single_cell_64_full_batch_sampled():
    """The timed workload at full size (7 x 1024 instances, Nt=64, K=16,
    Nr=4, d=4, 50 iterations, one launch as bench.py runs it); eight
    instances spread over the P sweep are re-solved by the oracle."""
    insts = wl.single_cell_64()
    g = GpuRun(insts)
    g.warmstart()
    g.step(50)
    got = g.wsr()
    assert np.all(g.status() == 0)
    assert np.all(np.isfinite(got))
    check_free_running(got, insts, 50, "full batch", sample=[0, 1500, 2100, 3333, 4200, 5000, 6000, 7167])
    g.close()


def test_nonfinite_input_sets_status():
    insts = wl.tiny_fp64(4)
    insts[1].H[0, 0, 0] = np.nan
    insts[2].sigma2[0] = 0.0
    g = GpuRun(insts)
    g.warmstart()
    g.step(10)
    st = g.status()
    got = g.wsr()
    assert st[0] == 0 and st[3] == 0
    assert st[1] == 4 and st[2] == 4  # AMM_ENUMERIC
    assert np.isnan(got[1]) and np.isnan(got[2])
    for b in (0, 3):
        ref = oracle_run(insts[b], 10)
        want = oracle_wsr_bits(insts[b], ref.V)
        assert abs(got[b] - want) <= WSR_TOL * want
    g.close()


def test_checkpoint_resume_is_exact():
    insts = small_batch((2, 3, 17, 3, 2), 4, 77)
    a = GpuRun(insts)
    a.warmstart()
    a.step(11)
    Va = a.V()
    b = GpuRun(insts)
    b.warmstart()
    b.step(5)
    st = b.get_state()
    c = GpuRun(insts)
    c.s.set_state(**st)
    c.step(6)
    Vc = c.V()
    for x, y in zip(Va, Vc):
        assert np.array_equal(x, y)
    for r in (a, b, c):
        r.close()


def test_solve_tolerance_mode():
    """amm_solve stops with Algorithm 3's eps2 test after a stage-II
    iteration; iteration counts match the oracle's."""
    import torch
    insts = wl.tiny_fp64(10)
    g = GpuRun(insts)
    g.warmstart()
    iters = torch.zeros(len(insts), dtype=torch.int32, device="cuda:0")
    g.s.solve(200, iters)
    it = iters.cpu().numpy()
    st = g.status()
    got = g.wsr()
    for b, inst in enumerate(insts):
        V0 = osv.initial_precoder(inst.G0, inst.P)
        ref = osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, 4, 2, 2, V0, 200, tolerance_stop=True)
        rhos = [h.rho for h in ref.history]
        # no stage or stopping decision of these instances lies near its threshold
        assert all(abs(abs(y - x) / x - 1e-3) >= 1e-6 and abs(abs(y - x) / x - 0.1) >= 1e-4
                   for x, y in zip(rhos, rhos[1:])), b
        assert it[b] == ref.iters, (b, it[b], ref.iters)
        assert st[b] == (0 if ref.converged else 6)
        want = oracle_wsr_bits(inst, ref.V)
        assert abs(got[b] - want) <= WSR_TOL * want
    g.close()


def test_solve_host_matches_device_path():
    import torch
    insts = wl.tiny_fp64(6)
    g = GpuRun(insts)
    g.warmstart()
    g.step(20)
    dev_wsr = g.wsr()
    pk = g.pk
    wsr = torch.empty(len(insts), dtype=torch.float64).pin_memory()
    V = torch.empty(g.s.v_elems, dtype=torch.complex64).pin_memory()
    g.s.solve_host(torch.from_numpy(pk.H), torch.from_numpy(pk.alpha), torch.from_numpy(pk.sigma2),
                   torch.from_numpy(pk.P), torch.from_numpy(pk.G0), 20, wsr, V)
    assert np.array_equal(wsr.numpy(), dev_wsr)
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_host_pipeline_matches_single_context(prec):
    """HostPipeline (the batch in parts, one context and stream each, run
    from concurrent host threads) gives the single-context results bit for
    bit, V included, for uneven part sizes."""
    import torch
    import paper_2510_20507_gb300 as pkg
    insts = round_inputs(wl.single_cell_64(2, first=0, count=11))
    pk = wl.pack(insts)
    host = [torch.from_numpy(x).pin_memory() for x in (pk.H, pk.alpha, pk.sigma2, pk.P, pk.G0)]
    one = pkg.Solver(len(insts), pk.dims[0], precision=prec)
    w1 = torch.empty(len(insts), dtype=torch.float64).pin_memory()
    V1 = torch.empty(one.v_elems, dtype=torch.complex64).pin_memory()
    one.solve_host(*host, 50, w1, V1)
    pipe = pkg.HostPipeline(len(insts), pk.dims[0], chunks=3, precision=prec)
    w2 = torch.zeros(len(insts), dtype=torch.float64).pin_memory()
    V2 = torch.zeros(one.v_elems, dtype=torch.complex64).pin_memory()
    pipe.solve_host(*host, 50, w2, V2)
    assert np.array_equal(w1.numpy(), w2.numpy())
    assert np.array_equal(V1.numpy(), V2.numpy())
    assert [b - a for a, b in pipe.parts] == [3, 4, 4]
    pipe.close()
    one.close()


@pytest.mark.parametrize("eig", [False, True])
@pytest.mark.parametrize("shape", [(1, 4, 8, 2, 2), (2, 2, 6, 2, 1), (1, 6, 24, 4, 2), (1, 5, 7, 1, 1),
                                   (1, 8, 33, 2, 2)])
def test_wmmse_step_matches_oracle(shape, eig):
    """amm_wmmse_step (Algorithm 2: eq. (9), eq. (10), eq. (12) with
    bisection to width 1e-4, at most 100 halvings; eig: the multiplier and
    V_k from a Jacobi eigen-decomposition of A_k) against the oracle's
    WMMSE from the same projected V^0; odd Nt and K d < Nt (a singular A_k,
    so the bisection runs) included."""
    iters = 12
    insts = small_batch(shape, 6, 7000 + sum(shape))
    g = GpuRun(insts)
    g.warmstart()
    g.s.wmmse_step(iters, 1e-4, 100, eig=eig)
    got = g.wsr()
    assert np.all(g.status() == 0)
    for b, inst in enumerate(insts):
        V0 = osv.initial_precoder(inst.G0, inst.P)
        _, hist, _ = osv.wmmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, iters,
                               tol=1e-4, max_bisect=100)
        want = hist[-1] / np.log(2.0)
        assert abs(got[b] - want) <= WSR_TOL * want, (shape, b, got[b], want)
    g.close()


@pytest.mark.parametrize("shape", [(1, 16, 64, 2, 2), (2, 3, 17, 3, 2), (1, 8, 33, 2, 2)])
def test_wmmse_eig_step_matches_cholesky_step(shape):
    """One WMMSE iteration from the same V^0: the V update from the Jacobi
    eigen-decomposition of A_k agrees with the Cholesky-bisection update
    (the same multiplier to the bisection width, the same V up to FP32
    rounding of the two factorisations)."""
    insts = small_batch(shape, 4, 7100 + sum(shape))
    Vs = []
    for eig in (False, True):
        g = GpuRun(insts)
        g.warmstart()
        g.s.wmmse_step(1, 1e-6, 100, eig=eig)
        assert np.all(g.status() == 0)
        Vs.append(g.V())
        g.close()
    for b in range(len(insts)):
        err = np.linalg.norm(Vs[1][b] - Vs[0][b]) / np.linalg.norm(Vs[0][b])
        assert err <= 2e-3, (shape, b, err)


@pytest.mark.parametrize("solves", [0, 2])
@pytest.mark.parametrize("shape", [(1, 16, 64, 4, 4), (2, 3, 17, 3, 2), (1, 5, 33, 4, 3), (1, 7, 40, 4, 4),
                                   (3, 2, 9, 2, 1), (1, 1, 5, 1, 1)])
def test_teacher_forced_step_other_solves(shape, solves):
    """fp64_solves = 0: the per-user Cholesky solves in FP32 (log-det from
    log1p of the pivots of I + M computed from M); fp64_solves = 2: in
    float-float (pairs of FP32).  Both still reproduce the oracle's step
    within the FP64 solves' bounds."""
    insts = small_batch(shape, 4, 8000 + sum(shape))
    assert_step_bounds(teacher_forced(insts, 10, gpu_opts=dict(fp64_solves=solves)), f"solves {solves} {shape}")


def test_contexts_of_different_sizes_coexist():
    """A small context created after a large one must not shrink the large
    one's shared-memory allowance."""
    big = wl.single_cell_64(first=0, count=4)
    small = wl.tiny_fp64(4)
    a = GpuRun(big)
    b = GpuRun(small)
    a.warmstart()
    a.step(3)
    b.warmstart()
    b.step(3)
    assert np.all(np.isfinite(a.wsr())) and np.all(np.isfinite(b.wsr()))
    a.close()
    b.close()


def test_uneven_batch_per_step():
    """An uneven batch (Nt in 16..256, K in 4..64, Nr in {1, 2, 4},
    d = min(Nr, 2), P = 0..30 dB) in one launch, blocks ordered longest
    first; the largest instances keep H, V and Z in global memory.  One
    iteration from the oracle's state matches it within 1e-5."""
    insts = round_inputs(wl.uneven(n=4096, count=192))
    cost = [i.K * i.K * i.Nr * i.Nt * i.d for i in insts]
    order = np.argsort(cost)
    picks = [int(order[0]), int(order[1]), int(order[len(order) // 2]), 183, int(order[-1])]
    assert_step_bounds(teacher_forced(insts, 6, picks), "uneven")


def test_seven_cell_layout_per_step():
    """Seven hexagonal cells (Nt=128, K=10, Nr=2, d=2, path loss and
    shadowing, -104 dBm noise, 46 dBm per BS): all 50 iterations of 16
    instances, each started from the oracle's state, match it per step (V,
    every user's block, R^t, stage, gamma_c).  Channels are normalised by
    the noise level inside amm_set_problem."""
    insts = round_inputs(wl.hex7(n=256, count=16))
    with spawn_pool() as pool:
        assert_step_bounds(teacher_forced(insts, 50, pool=pool), "seven cells, 50 iterations")


def _free_running(insts, iters):
    g = GpuRun(insts)
    g.warmstart()
    g.step(iters)
    got = g.wsr()
    assert np.all(g.status() == 0)
    g.close()
    return got


def test_uneven_batch_free_running():
    """The whole uneven batch (4096 instances, 30 iterations) in one launch;
    every 32nd instance (128, the bench's oracle sample) judged."""
    insts = round_inputs(wl.uneven(n=4096))
    got = _free_running(insts, 30)
    with spawn_pool() as pool:
        check_free_running(got, insts, 30, "uneven", sample=range(0, 4096, 32), pool=pool)


def test_seven_cell_free_running():
    """The whole seven-cell batch (256 instances, 50 iterations), every
    instance judged."""
    insts = round_inputs(wl.hex7(n=256))
    got = _free_running(insts, 50)
    with spawn_pool() as pool:
        check_free_running(got, insts, 50, "seven cells", pool=pool)


@pytest.mark.parametrize("shape", [(1, 48, 16, 2, 2), (1, 8, 256, 1, 1), (1, 35, 256, 1, 1), (1, 64, 256, 2, 2),
                                   (1, 4, 64, 1, 1), (1, 16, 64, 4, 4), (2, 3, 17, 3, 2)])
def test_spectral_step_every_iteration(shape):
    """step_rule 1 takes gamma = 1/||F_k||_2 in every iteration, so every
    step checks the Lanczos estimate of the largest eigenvalue of F_k:
    shapes where the Krylov space fills all of C^Nt (Nt = 16), where
    rank(F_k) is far below Nt, and where the top of the spectrum is dense
    (K d = 128 of Nt = 256)."""
    insts = small_batch(shape, 3, 7000 + sum(shape))
    assert_step_bounds(teacher_forced(insts, 8, step_rule=1), f"spectral every iteration {shape}")


@pytest.mark.parametrize("prec,solves", [("fp32", 1), ("bf16x6", 1), ("bf16x6", 2), ("fp32", 2)])
def test_timed_workload_high_snr_per_step(prec, solves):
    """All 50 iterations of timed-workload instances at 0, 25 and 30 dB,
    each started from the oracle's state: the per-step bound holds on the
    instances whose free-running trajectories are FP32-sensitive too, for
    FP64 and float-float solves."""
    picks = [100, 5488, 5570, 6495, 6992]
    sub = round_inputs([wl.single_cell_64(first=b, count=1)[0] for b in picks])
    assert_step_bounds(teacher_forced(sub, 50, gpu_opts=dict(precision=prec, fp64_solves=solves)),
                       f"timed workload {prec} solves {solves}")


def test_persistent_schedule_matches_one_block_per_instance():
    """schedule = 1 (persistent blocks taking instances from a device
    counter, longest first) computes every instance exactly as the
    one-block-per-instance launch: identical iterates and WSR, including
    the instances whose channel stays in global memory (staged GEMMs)."""
    insts = round_inputs(wl.uneven(n=4096, count=192))
    out = []
    for sched in (0, 1):
        g = GpuRun(insts, schedule=sched)
        g.warmstart()
        g.step(6)
        out.append((g.V(), g.wsr(), g.status()))
        g.close()
    assert all(np.array_equal(a, b) for a, b in zip(out[0][0], out[1][0]))
    assert np.array_equal(out[0][1], out[1][1]) and np.all(out[1][2] == 0)
