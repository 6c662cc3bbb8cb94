"""Python binding of the C-ABI in include/amm.h (argument marshalling only).

Every step of the solver runs in the CUDA kernels of ``libamm.so``; this
module converts torch tensors (used for device memory and streams) to raw
pointers and status codes to exceptions.  There is no fallback: without the
compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple, Union

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libamm.so")

AMM_OK, AMM_EINVAL, AMM_ENOMEM, AMM_ECUDA, AMM_ENUMERIC, AMM_ETIMEOUT, AMM_ENOTCONV, AMM_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "AMM_OK", 1: "AMM_EINVAL", 2: "AMM_ENOMEM", 3: "AMM_ECUDA", 4: "AMM_ENUMERIC",
                5: "AMM_ETIMEOUT", 6: "AMM_ENOTCONV", 7: "AMM_EUNSUPPORTED"}
PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3}


class AmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Dims(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int), ("users", ctypes.c_int), ("nt", ctypes.c_int),
                ("nr", ctypes.c_int), ("d", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("eps1", ctypes.c_double), ("eps2", ctypes.c_double), ("tc", ctypes.c_int),
                ("gamma_c", ctypes.c_double), ("extrapolate", ctypes.c_int), ("switch_iter", ctypes.c_int),
                ("step_rule", ctypes.c_int), ("precision", ctypes.c_int), ("u_at_extrapolated", ctypes.c_int),
                ("lanczos_steps", ctypes.c_int), ("spin_budget", ctypes.c_longlong),
                ("smem_budget", ctypes.c_int), ("fp64_solves", ctypes.c_int), ("gemm_tile", ctypes.c_int),
                ("cluster_cells", ctypes.c_int), ("schedule", ctypes.c_int)]


class State(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("Vprev", ctypes.c_void_p), ("t", ctypes.c_void_p),
                ("stage", ctypes.c_void_p), ("stage_iter", ctypes.c_void_p), ("rho_prev", ctypes.c_void_p),
                ("gamma_c", ctypes.c_void_p)]


EXPORTS = ["amm_default_opts", "amm_create", "amm_sizes", "amm_set_problem", "amm_warmstart", "amm_step",
           "amm_solve", "amm_wsr", "amm_wmmse_step", "amm_wmmse_step_eig", "amm_get_V", "amm_get_state", "amm_set_state",
           "amm_status_dev", "amm_solve_host", "amm_destroy", "amm_last_error", "amm_launch_count", "amm_path",
           "amm_solve_noalloc", "amm_test_fail_alloc", "amm_graph_create", "amm_graph_launch", "amm_graph_destroy", "amm_unrolled_create", "amm_unrolled_forward", "amm_unrolled_backward",
           "amm_unrolled_status", "amm_unrolled_last_error", "amm_unrolled_destroy"]

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libamm.so and declare the signatures.  Raises ImportError when
    the library has not been built (``python -m paper_2510_20507_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2510_20507_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "amm_default_opts": (None, [ctypes.POINTER(Opts)]),
        "amm_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(Dims), i32, ctypes.POINTER(Opts), vp]),
        "amm_sizes": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                            ctypes.POINTER(i64)]),
        "amm_set_problem": (i32, [vp, vp, vp, vp, vp]),
        "amm_warmstart": (i32, [vp, vp]),
        "amm_step": (i32, [vp, i32]),
        "amm_solve": (i32, [vp, i32, vp]),
        "amm_wsr": (i32, [vp, vp]),
        "amm_wmmse_step": (i32, [vp, i32, dbl, i32]),
        "amm_wmmse_step_eig": (i32, [vp, i32, dbl, i32]),
        "amm_get_V": (i32, [vp, vp]),
        "amm_get_state": (i32, [vp, ctypes.POINTER(State)]),
        "amm_set_state": (i32, [vp, ctypes.POINTER(State)]),
        "amm_status_dev": (i32, [vp, vp]),
        "amm_solve_host": (i32, [vp, vp, vp, vp, vp, vp, i32, vp, vp]),
        "amm_destroy": (None, [vp]),
        "amm_last_error": (ctypes.c_char_p, [vp]),
        "amm_launch_count": (i64, [vp]),
        "amm_path": (i32, [vp]),
        "amm_solve_noalloc": (i32, [i32, ctypes.POINTER(Dims), ctypes.POINTER(Opts), vp, vp, vp, vp, vp, i32, vp,
                                    vp, vp, ctypes.c_char_p, i32]),
        "amm_test_fail_alloc": (None, [i32]),
        "amm_graph_create": (i32, [vp, vp, vp, vp, vp, vp, i32, vp, ctypes.POINTER(vp)]),
        "amm_graph_launch": (i32, [vp]),
        "amm_graph_destroy": (None, [vp]),
        "amm_unrolled_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(Dims), i32, i32, i32, i32, vp]),
        "amm_unrolled_forward": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "amm_unrolled_backward": (i32, [vp, vp, vp, vp]),
        "amm_unrolled_status": (i32, [vp, vp]),
        "amm_unrolled_last_error": (ctypes.c_char_p, [vp]),
        "amm_unrolled_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_opts(**overrides) -> Opts:
    lib = load_library()
    o = Opts()
    lib.amm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def solve_noalloc(batch, dims, H, alpha, sigma2, P, V0, n_iters, V_out, wsr_out, opts=None, stream=None):
    """amm_solve_noalloc: a whole solve that allocates no device memory (its
    workspace is a static device array inside the library), for callers that
    may not allocate device memory while they run.  All tensors are
    caller-owned device buffers in the C-ABI layouts."""
    lib = load_library()
    if opts is None:
        opts = default_opts()
    err = ctypes.create_string_buffer(256)
    d = Dims(*dims)
    st = lib.amm_solve_noalloc(batch, ctypes.byref(d), ctypes.byref(opts), _ptr(H), _ptr(alpha), _ptr(sigma2),
                               _ptr(P), _ptr(V0), n_iters, _ptr(V_out), _ptr(wsr_out), _stream_handle(stream),
                               err, len(err))
    if st != AMM_OK:
        raise AmmError(st, err.value.decode())


DimsLike = Union[Tuple[int, int, int, int, int], Sequence[Tuple[int, int, int, int, int]]]


class Solver:
    """A batch of instances behind one amm_ctx.

    ``dims`` is one (C, K, Nt, Nr, d) tuple for a uniform batch or a list of
    ``batch`` tuples for an uneven one.  ``stream`` is a torch.cuda.Stream (or
    a raw cudaStream_t); every call is asynchronous on it.
    """

    def __init__(self, batch: int, dims: DimsLike, opts: Optional[Opts] = None, stream=None, **overrides):
        self.lib = load_library()
        if opts is None:
            opts = default_opts(**overrides)
        if isinstance(dims[0], int):
            arr = (Dims * 1)(Dims(*dims))
            nd = 1
        else:
            arr = (Dims * len(dims))(*[Dims(*t) for t in dims])
            nd = len(dims)
        h = ctypes.c_void_p()
        st = self.lib.amm_create(ctypes.byref(h), batch, arr, nd, ctypes.byref(opts), _stream_handle(stream))
        if st != AMM_OK:
            raise AmmError(st, self.lib.amm_last_error(None).decode())
        self.h = h
        self.batch = batch
        self.opts = opts
        he, ve, nu, nc = (ctypes.c_int64() for _ in range(4))
        self._check(self.lib.amm_sizes(self.h, ctypes.byref(he), ctypes.byref(ve), ctypes.byref(nu),
                                       ctypes.byref(nc)))
        self.h_elems, self.v_elems, self.n_users, self.n_cells = he.value, ve.value, nu.value, nc.value

    # -- helpers
    def _check(self, st: int):
        if st != AMM_OK:
            raise AmmError(st, self.lib.amm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.amm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points
    def set_problem(self, H, alpha, sigma2, P):
        self._check(self.lib.amm_set_problem(self.h, _ptr(H), _ptr(alpha), _ptr(sigma2), _ptr(P)))

    def warmstart(self, V0):
        self._check(self.lib.amm_warmstart(self.h, _ptr(V0)))

    def step(self, n_iters: int):
        self._check(self.lib.amm_step(self.h, n_iters))

    def solve(self, max_iter: int, iters=None):
        self._check(self.lib.amm_solve(self.h, max_iter, _ptr(iters)))

    def wsr(self, out):
        self._check(self.lib.amm_wsr(self.h, _ptr(out)))
        return out

    def wmmse_step(self, n_iters: int, bisect_tol: float = 1e-4, bisect_max: int = 100, eig: bool = False):
        """Plain WMMSE iterations (amm_wmmse_step, or amm_wmmse_step_eig when eig)."""
        f = self.lib.amm_wmmse_step_eig if eig else self.lib.amm_wmmse_step
        self._check(f(self.h, n_iters, bisect_tol, bisect_max))

    def get_V(self, out):
        self._check(self.lib.amm_get_V(self.h, _ptr(out)))
        return out

    def get_state(self, V, Vprev, t, stage, stage_iter, rho_prev, gamma_c):
        st = State(_ptr(V), _ptr(Vprev), _ptr(t), _ptr(stage), _ptr(stage_iter), _ptr(rho_prev), _ptr(gamma_c))
        self._check(self.lib.amm_get_state(self.h, ctypes.byref(st)))

    def set_state(self, V, Vprev, t, stage, stage_iter, rho_prev, gamma_c):
        st = State(_ptr(V), _ptr(Vprev), _ptr(t), _ptr(stage), _ptr(stage_iter), _ptr(rho_prev), _ptr(gamma_c))
        self._check(self.lib.amm_set_state(self.h, ctypes.byref(st)))

    def status(self, out):
        self._check(self.lib.amm_status_dev(self.h, _ptr(out)))
        return out

    def solve_host(self, H, alpha, sigma2, P, V0, n_iters: int, wsr_out, V_out=None):
        self._check(self.lib.amm_solve_host(self.h, _ptr(H), _ptr(alpha), _ptr(sigma2), _ptr(P), _ptr(V0),
                                            n_iters, _ptr(wsr_out), _ptr(V_out)))

    @property
    def launches(self) -> int:
        return int(self.lib.amm_launch_count(self.h))

    @property
    def path(self) -> str:
        """The iteration kernel this context runs: "block" (CUDA-core GEMMs),
        "tensor" (tcgen05 GEMMs) or "cluster" (one cluster per multi-cell
        instance)."""
        return {0: "block", 1: "tensor", 2: "cluster"}[int(self.lib.amm_path(self.h))]

    def capture(self, H, alpha, sigma2, P, V0, n_iters: int, wsr_out) -> "Graph":
        """Record set_problem + warmstart + step(n_iters) + wsr as a CUDA graph
        (amm_graph_create); Graph.launch() replays it."""
        g = ctypes.c_void_p()
        self._check(self.lib.amm_graph_create(self.h, _ptr(H), _ptr(alpha), _ptr(sigma2), _ptr(P), _ptr(V0),
                                              n_iters, _ptr(wsr_out), ctypes.byref(g)))
        return Graph(self, g, (H, alpha, sigma2, P, V0, wsr_out))


class HostPipeline:
    """A host-resident uniform batch solved in ``chunks`` parts, one context
    and one CUDA stream per part: ``solve_host`` runs amm_solve_host for every
    part from its own host thread, so the host-to-device copy of one part
    overlaps the solve of another.  Inputs and outputs are the host buffers
    of Solver.solve_host for the whole batch (pinned memory, batch-major);
    results are those of one context over the whole batch, instance by
    instance."""

    def __init__(self, batch: int, dims, chunks: int = 4, opts: Optional[Opts] = None, **overrides):
        import concurrent.futures
        import torch
        if not isinstance(dims[0], int):
            raise ValueError("HostPipeline takes one (C, K, Nt, Nr, d) for the whole batch")
        chunks = max(1, min(int(chunks), batch))
        edges = [batch * k // chunks for k in range(chunks + 1)]
        self.parts = [(a, b) for a, b in zip(edges, edges[1:]) if b > a]
        self.streams = [torch.cuda.Stream() for _ in self.parts]
        self.solvers = [Solver(b - a, dims, opts, stream=st, **overrides) for (a, b), st in zip(self.parts, self.streams)]
        s0 = self.solvers[0]
        nb = self.parts[0][1] - self.parts[0][0]
        # per-instance sizes of the packed host buffers
        self.per = {"H": s0.h_elems // nb, "V": s0.v_elems // nb, "u": s0.n_users // nb, "c": s0.n_cells // nb}
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=len(self.parts))
        self.batch = batch

    def solve_host(self, H, alpha, sigma2, P, V0, n_iters: int, wsr_out, V_out=None):
        per = self.per

        def run(k):
            a, b = self.parts[k]
            self.solvers[k].solve_host(H[a * per["H"]:b * per["H"]], alpha[a * per["u"]:b * per["u"]],
                                       sigma2[a * per["u"]:b * per["u"]], P[a * per["c"]:b * per["c"]],
                                       V0[a * per["V"]:b * per["V"]], n_iters, wsr_out[a:b],
                                       None if V_out is None else V_out[a * per["V"]:b * per["V"]])

        for f in [self.pool.submit(run, k) for k in range(len(self.parts))]:
            f.result()

    @property
    def launches(self) -> int:
        return sum(s.launches for s in self.solvers)

    def close(self):
        for s in self.solvers:
            s.close()
        self.pool.shutdown(wait=True)


class Graph:
    """A recorded solve of one Solver (amm_graph_*)."""

    def __init__(self, solver: Solver, handle, keep):
        self.solver, self.h, self._keep = solver, handle, keep

    def launch(self):
        self.solver._check(self.solver.lib.amm_graph_launch(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.solver.lib.amm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UnrolledSolver:
    """The differentiable unrolled A-MMMSE of include/amm.h (amm_unrolled_*):
    T iterations with step sizes gamma_t and a fixed stage schedule, its
    WSR(V^T) and the hand-written adjoint.  One cell per instance."""

    def __init__(self, batch: int, dims, T: int, ckpt_every: int = 5, switch_iter: int = -1,
                 extrapolate: bool = True, stream=None):
        self.lib = load_library()
        d = Dims(*dims)
        h = ctypes.c_void_p()
        st = self.lib.amm_unrolled_create(ctypes.byref(h), batch, ctypes.byref(d), T, ckpt_every, switch_iter,
                                          1 if extrapolate else 0, _stream_handle(stream))
        if st != AMM_OK:
            raise AmmError(st, self.lib.amm_unrolled_last_error(None).decode())
        self.h = h
        self.batch, self.dims, self.T = batch, tuple(dims), T
        self._keep = None
        self.generation = 0  # forward calls so far: which call the stored checkpoints belong to

    def _check(self, st: int):
        if st != AMM_OK:
            raise AmmError(st, self.lib.amm_unrolled_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.amm_unrolled_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, H, alpha, sigma2, P, V0, gamma, wsr_out):
        self._keep = (H, alpha, sigma2, P, V0, gamma)  # read again by backward
        self.generation += 1
        self._check(self.lib.amm_unrolled_forward(self.h, _ptr(H), _ptr(alpha), _ptr(sigma2), _ptr(P), _ptr(V0),
                                                  _ptr(gamma), _ptr(wsr_out)))
        return wsr_out

    def backward(self, wsr_bar, gamma_bar, H_bar):
        self._check(self.lib.amm_unrolled_backward(self.h, _ptr(wsr_bar), _ptr(gamma_bar), _ptr(H_bar)))

    def status(self, out):
        self._check(self.lib.amm_unrolled_status(self.h, _ptr(out)))
        return out
