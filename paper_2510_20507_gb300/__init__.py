"""Batched A-MMMSE / WMMSE multi-cell MU-MIMO precoding on GB300 (sm_103a).

The solver is the C-ABI library ``lib/libamm.so`` (declared in
``include/amm.h``); :mod:`.amm` is its thin Python binding.  Build it with
``python -m paper_2510_20507_gb300.build``.
"""
from .amm import (AmmError, Solver, HostPipeline, UnrolledSolver, default_opts, load_library, solve_noalloc, LIB_PATH,  # noqa: F401
                  EXPORTS,
                  AMM_OK, AMM_EINVAL, AMM_ENOMEM, AMM_ECUDA, AMM_ENUMERIC, AMM_ETIMEOUT, AMM_ENOTCONV,
                  AMM_EUNSUPPORTED, PRECISIONS)
