"""Host-side checks of the C-ABI library: it builds, loads, exports every
entry point include/amm.h declares, and rejects bad arguments before any
CUDA call (so these run without a GPU)."""
import ctypes
import os
import re

import pytest

import __graft_entry__ as ge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ge.build()
    import paper_2510_20507_gb300 as pkg
    return pkg.load_library()


def header_functions():
    text = open(os.path.join(ROOT, "include", "amm.h")).read()
    return sorted(set(re.findall(r"AMM_API\s+[\w\s\*]+?\b(amm_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = header_functions()
    for must in ["amm_create", "amm_warmstart", "amm_step", "amm_solve", "amm_wsr", "amm_wmmse_step",
                 "amm_wmmse_step_eig",
                 "amm_set_problem", "amm_get_state", "amm_set_state", "amm_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2510_20507_gb300 as pkg
    for name in header_functions():
        assert hasattr(lib, name), name
    assert sorted(pkg.EXPORTS) == header_functions()


def _create(lib, batch, dims, n_dims=None, **opts):
    import paper_2510_20507_gb300 as pkg
    o = pkg.default_opts(**opts)
    arr = (pkg.amm.Dims * len(dims))(*[pkg.amm.Dims(*d) for d in dims])
    h = ctypes.c_void_p()
    st = lib.amm_create(ctypes.byref(h), batch, arr, n_dims or len(dims), ctypes.byref(o), None)
    return st, h


@pytest.mark.parametrize("dims", [
    (1, 4, 8, 2, 3),      # d > Nr
    (1, 4, 8, 5, 2),      # Nr > 4
    (0, 4, 8, 2, 2),      # no cells
    (17, 1, 8, 2, 2),     # too many cells
    (1, 0, 8, 2, 2),      # no users
    (1, 4, 0, 2, 2),      # no antennas
    (1, 2000, 8, 4, 1),   # m > 4096
])
def test_create_rejects_bad_dims(lib, dims):
    import paper_2510_20507_gb300 as pkg
    st, h = _create(lib, 3, [dims])
    assert st == pkg.AMM_EINVAL
    assert not h.value
    assert b"dims" in lib.amm_last_error(None) or b"large" in lib.amm_last_error(None)


def test_create_rejects_bad_batch_and_options(lib):
    import paper_2510_20507_gb300 as pkg
    assert _create(lib, 0, [(1, 4, 8, 2, 2)])[0] == pkg.AMM_EINVAL
    assert _create(lib, 3, [(1, 4, 8, 2, 2)] * 2, n_dims=2)[0] == pkg.AMM_EINVAL        # n_dims != 1, batch
    assert _create(lib, 2, [(1, 4, 8, 2, 2), (2, 4, 8, 2, 2)])[0] == pkg.AMM_EINVAL     # mixed cell counts
    assert _create(lib, 1, [(1, 4, 8, 2, 2)], step_rule=2)[0] == pkg.AMM_EINVAL          # fixed step, no gamma_c
    assert _create(lib, 1, [(1, 4, 8, 2, 2)], step_rule=0, tc=0)[0] == pkg.AMM_EINVAL
    assert _create(lib, 1, [(1, 4, 8, 2, 2)], lanczos_steps=0)[0] == pkg.AMM_EINVAL
    assert _create(lib, 1, [(1, 4, 8, 2, 2)], precision=9)[0] == pkg.AMM_EINVAL
    assert _create(lib, 1, [(1, 4, 8, 2, 2)], u_at_extrapolated=1)[0] == pkg.AMM_EUNSUPPORTED
    # the tensor-core path covers one cell with 2m <= 128, 2Nt <= 128
    assert _create(lib, 1, [(2, 4, 8, 2, 2)], precision="bf16x3")[0] == pkg.AMM_EUNSUPPORTED
    assert _create(lib, 1, [(1, 4, 80, 2, 2)], precision="bf16")[0] == pkg.AMM_EUNSUPPORTED
    assert _create(lib, 1, [(1, 40, 16, 2, 2)], precision="bf16x3")[0] == pkg.AMM_EUNSUPPORTED
    st = lib.amm_create(None, 1, None, 1, None, None)
    assert st == pkg.AMM_EINVAL


def test_null_context_is_rejected(lib):
    import paper_2510_20507_gb300 as pkg
    assert lib.amm_step(None, 1) == pkg.AMM_EINVAL
    assert lib.amm_wsr(None, None) == pkg.AMM_EINVAL
    assert lib.amm_wmmse_step(None, 1, 1e-4, 100) == pkg.AMM_EINVAL
    assert lib.amm_wmmse_step_eig(None, 1, 1e-4, 100) == pkg.AMM_EINVAL
    lib.amm_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2510_20507_gb300.amm as b
    saved = b._lib
    b._lib = None
    try:
        with pytest.raises(ImportError):
            b.load_library(str(tmp_path / "missing.so"))
    finally:
        b._lib = saved


def test_injected_allocation_failure_gives_enomem(lib):
    """A device allocation failure inside amm_create (injected on the host:
    the first allocation fails, no CUDA call is made) is reported as
    AMM_ENOMEM with no context returned."""
    import paper_2510_20507_gb300 as pkg
    lib.amm_test_fail_alloc(1)
    try:
        st, h = _create(lib, 4, [(1, 4, 8, 2, 2)])
    finally:
        lib.amm_test_fail_alloc(0)
    assert st == pkg.AMM_ENOMEM and not h.value
    assert b"allocation" in lib.amm_last_error(None)


def _noalloc(lib, **opts):
    import paper_2510_20507_gb300 as pkg
    o = pkg.default_opts(**opts)
    d = pkg.amm.Dims(1, 4, 8, 2, 2)
    err = ctypes.create_string_buffer(256)
    fake = ctypes.c_void_p(256)  # never dereferenced: the options are rejected first
    st = lib.amm_solve_noalloc(4, ctypes.byref(d), ctypes.byref(o), fake, fake, fake, fake, fake, 10, fake, fake,
                               None, err, len(err))
    return st, err.value


def test_noalloc_checks_options_like_create(lib):
    import paper_2510_20507_gb300 as pkg
    assert _noalloc(lib, eps1=float("nan"))[0] == pkg.AMM_EINVAL
    assert _noalloc(lib, eps1=-0.1)[0] == pkg.AMM_EINVAL
    assert _noalloc(lib, eps2=float("nan"))[0] == pkg.AMM_EINVAL
    assert _noalloc(lib, step_rule=2)[0] == pkg.AMM_EINVAL          # fixed step without gamma_c
    assert _noalloc(lib, precision=9)[0] == pkg.AMM_EINVAL
    st, msg = _noalloc(lib, u_at_extrapolated=1)
    assert st == pkg.AMM_EUNSUPPORTED and b"u_at_extrapolated" in msg
    st, msg = _noalloc(lib, precision="bf16x6")
    assert st == pkg.AMM_EUNSUPPORTED and b"FP32" in msg
