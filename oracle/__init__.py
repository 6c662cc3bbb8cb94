"""FP64 CPU oracle for A-MMMSE / WMMSE (arXiv 2510.20507).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the GPU library, with which
it shares no code.  Pins against the paper and the mathematics live in
``tests/test_oracle_pins.py``.

Parity status: every function here is pinned (closed forms, invariants,
perturbation and finite-difference checks, the paper's lemmas).  The WSR
values in the paper's figures are not printed in its text, so the match
with the paper's own numbers is parity unpinned.
"""
from . import model, solvers, closed_forms, sensitivity  # noqa: F401
