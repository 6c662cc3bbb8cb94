"""Drive the GPU solver through the C-ABI binding on seeded instances and
collect results as numpy arrays, plus oracle counterparts."""
from __future__ import annotations

import numpy as np

import workloads as wl
from oracle import model as om
from oracle import solvers as osv


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda:0") if dtype is None else t.to(device="cuda:0", dtype=dtype)


def round_inputs(insts):
    """Round every input to the nearest value the GPU receives (complex64 /
    float32) in place, so the oracle solves exactly the same problem."""
    for inst in insts:
        inst.H = inst.H.astype(np.complex64).astype(np.complex128)
        inst.G0 = inst.G0.astype(np.complex64).astype(np.complex128)
        inst.alpha = inst.alpha.astype(np.float32).astype(np.float64)
        inst.sigma2 = inst.sigma2.astype(np.float32).astype(np.float64)
        inst.P = inst.P.astype(np.float32).astype(np.float64)
    return insts


class GpuRun:
    """One Solver over a packed list of instances (inputs rounded in place)."""

    def __init__(self, insts, **opts):
        import torch
        import paper_2510_20507_gb300 as pkg
        self.insts = round_inputs(insts)
        self.pk = wl.pack(insts)
        dims = self.pk.dims[0] if self.pk.uniform else self.pk.dims
        self.s = pkg.Solver(len(insts), dims, **opts)
        self.H = to_dev(self.pk.H)
        self.G0 = to_dev(self.pk.G0)
        self.alpha = to_dev(self.pk.alpha)
        self.sigma2 = to_dev(self.pk.sigma2)
        self.P = to_dev(self.pk.P)
        self.s.set_problem(self.H, self.alpha, self.sigma2, self.P)
        self.torch = torch

    def warmstart(self):
        self.s.warmstart(self.G0)

    def step(self, n):
        self.s.step(n)

    def wsr(self):
        out = self.torch.empty(len(self.insts), dtype=self.torch.float64, device="cuda:0")
        self.s.wsr(out)
        self.torch.cuda.synchronize()
        return out.cpu().numpy()

    def V(self):
        out = self.torch.empty(self.s.v_elems, dtype=self.torch.complex64, device="cuda:0")
        self.s.get_V(out)
        self.torch.cuda.synchronize()
        return wl.unpack_V(self.pk, out.cpu().numpy())

    def status(self):
        out = self.torch.empty(len(self.insts), dtype=self.torch.int32, device="cuda:0")
        self.s.status(out)
        self.torch.cuda.synchronize()
        return out.cpu().numpy()

    def get_state(self):
        T = self.torch
        n, nc = len(self.insts), self.s.n_cells
        st = dict(V=T.empty(self.s.v_elems, dtype=T.complex64, device="cuda:0"),
                  Vprev=T.empty(self.s.v_elems, dtype=T.complex64, device="cuda:0"),
                  t=T.empty(n, dtype=T.int32, device="cuda:0"), stage=T.empty(n, dtype=T.int32, device="cuda:0"),
                  stage_iter=T.empty(n, dtype=T.int32, device="cuda:0"),
                  rho_prev=T.empty(n, dtype=T.float64, device="cuda:0"),
                  gamma_c=T.empty(nc, dtype=T.float32, device="cuda:0"))
        self.s.get_state(**st)
        T.cuda.synchronize()
        return st

    def set_state_from_oracle(self, states):
        """states: list of oracle AState, one per instance."""
        T = self.torch
        V = np.concatenate([st.V.reshape(-1) for st in states]).astype(np.complex64)
        Vp = np.concatenate([st.Vprev.reshape(-1) for st in states]).astype(np.complex64)
        t = np.array([st.t for st in states], dtype=np.int32)
        stage = np.array([st.stage for st in states], dtype=np.int32)
        si = np.array([st.stage_iter for st in states], dtype=np.int32)
        rp = np.array([np.nan if st.rho_prev is None else st.rho_prev for st in states], dtype=np.float64)
        gc = np.concatenate([np.zeros(inst.C) if st.gamma_c is None else st.gamma_c
                             for st, inst in zip(states, self.insts)]).astype(np.float32)
        self.s.set_state(V=to_dev(V), Vprev=to_dev(Vp), t=to_dev(t), stage=to_dev(stage), stage_iter=to_dev(si),
                         rho_prev=to_dev(rp), gamma_c=to_dev(gc))

    def close(self):
        self.s.close()


def oracle_run(inst, iters, **opt):
    V0 = osv.initial_precoder(inst.G0, inst.P)
    return osv.ammmse(inst.H, inst.sigma2, inst.alpha, inst.P, inst.K, inst.Nr, inst.d, V0, iters,
                      osv.Options(**opt))


def oracle_wsr_bits(inst, V):
    return om.wsr_bits(inst.H, V, inst.sigma2, inst.alpha, inst.K, inst.Nr, inst.d)


# An instance is FP32-sensitive when perturbations of the size of FP32
# rounding move the oracle's own final WSR by more than this (relative).
# Instances off the sensitive regime move by 1e-7 or less.
SENSITIVE = 1e-5


def oracle_fp32_spread(inst, iters):
    """oracle.sensitivity.fp32_spread: the largest relative change of the
    oracle's final WSR under FP32-sized perturbations of its arithmetic."""
    from oracle.sensitivity import fp32_spread
    return fp32_spread(inst, iters)


def check_free_running(got, insts, iters, label, sample=None, tol=1e-3):
    """Final WSR of a free-running GPU solve against the oracle, instance by
    instance: within tol, unless the instance is FP32-sensitive (its
    trajectory is then not fixed to tol by any FP32 arithmetic; such
    instances are bounded by 5e-2 and reported).  Instances whose oracle
    trajectory takes the stage decision within 1e-4 of eps1 are skipped.
    Returns the list of (index, gap, spread) of sensitive instances beyond
    tol."""
    excused = []
    for b in (range(len(insts)) if sample is None else sample):
        ref = oracle_run(insts[b], iters)
        if switch_margin(ref) < 1e-4:
            continue
        want = oracle_wsr_bits(insts[b], ref.V)
        gap = abs(got[b] - want) / want
        if gap > tol:
            spread = oracle_fp32_spread(insts[b], iters)
            print(f"{label}: instance {b} gap {gap:.2e}, oracle spread under FP32-sized perturbation {spread:.2e}")
            assert spread > SENSITIVE and gap <= 5e-2, (label, b, got[b], want, spread)
            excused.append((b, gap, spread))
    return excused


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def switch_margin(result, eps1=0.1):
    """Smallest |relative WSR change - eps1| over a trajectory's stage-I
    iterations: how close the oracle came to flipping the stage decision."""
    m = np.inf
    h = result.history
    for a, b in zip(h, h[1:]):
        if a.stage == 1:
            m = min(m, abs(abs(b.rho - a.rho) / abs(a.rho) - eps1))
    return m
