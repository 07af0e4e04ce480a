"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports every
entry point include/lp.h declares; parameter and status plumbing work without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_08072_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for need in ("lp_create", "lp_normal_solve", "lp_ipm_solve", "lp_destroy", "lp_residuals",
                 "lp_sketch", "lp_factor", "lp_normal_matvec", "lp_step", "lp_sketch_indices"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2003_08072_gb300 import _binding

    assert set(_declared_functions()) <= set(_binding._SIGNATURES)


def test_params_default_and_status_strings(lib):
    import paper_2003_08072_gb300 as pkg

    p = pkg.lp_params_default()
    assert p.tol == 1e-8 and p.sigma == 0.5 and p.sketch_s == 4 and p.cg_rel_tol == 1e-6
    assert ctypes.sizeof(pkg.lp_params) == 104
    assert p.use_graphs == 1 and p.gram_tensor_cores == 1 and p.autotune == 1
    assert p.shared_cg == 0 and p.persistent_cg == 0 and p.factor_dag == 1
    from paper_2003_08072_gb300 import _binding

    assert _binding.status_str(0) == "LP_OK"
    assert _binding.status_str(4) == "LP_ERR_BREAKDOWN"


def test_argument_errors_need_no_device(lib):
    """Invalid sizes are rejected before any CUDA call."""
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    with pytest.raises(pkg.LPError) as e:
        B.lp_create(0, 10, B.LP_DENSE_COLMAJOR, B.LP_F64, 1, None, None, 0, 1, 1)
    assert e.value.status == B.LP_ERR_ARG
    with pytest.raises(pkg.LPError) as e:
        B.lp_create(20, 10, B.LP_DENSE_COLMAJOR, B.LP_F64, 1, None, None, 0, 1, 1)
    assert e.value.status == B.LP_ERR_ARG
    bad = pkg.lp_params_default()
    bad.sigma = 0.9   # Alg. 2 needs sigma < 4/5
    with pytest.raises(pkg.LPError):
        B.lp_create(4, 10, B.LP_DENSE_COLMAJOR, B.LP_F64, 1, None, None, 0, 1, 1, params=bad)
    bad = pkg.lp_params_default()
    bad.sketch_w = 18   # not a multiple of s = 4
    with pytest.raises(pkg.LPError):
        B.lp_create(4, 10, B.LP_DENSE_COLMAJOR, B.LP_F64, 1, None, None, 0, 1, 1, params=bad)
    bad = pkg.lp_params_default()
    bad.inner_solver = 2   # neither CG nor Richardson
    with pytest.raises(pkg.LPError):
        B.lp_create(4, 10, B.LP_DENSE_COLMAJOR, B.LP_F64, 1, None, None, 0, 1, 1, params=bad)
    bad = pkg.lp_params_default()
    bad.sketch_kind = B.LP_SKETCH_GAUSSIAN   # needs a dense A
    with pytest.raises(pkg.LPError):
        B.lp_create(4, 10, B.LP_CSR, B.LP_F64, 1, 1, 1, 4, 1, 1, params=bad)
    with pytest.raises(pkg.LPError):
        B.lp_sketch_indices(0, 0, 10, 3, 16, 1, 1)   # w % s != 0
    # serving loop: bad sizes rejected before any CUDA call
    for budget, live in ((0, 4), (1 << 30, 0), (1 << 30, 257)):
        with pytest.raises(pkg.LPError) as e:
            B.lp_server_create(budget, live)
        assert e.value.status == B.LP_ERR_ARG
    # checkpoint / resume: plain-data state, NULL context rejected before any CUDA call
    assert ctypes.sizeof(B.lp_ipm_state) == 24
    with pytest.raises(pkg.LPError) as e:
        B.lp_ipm_get_state(None)
    assert e.value.status == B.LP_ERR_ARG
    st = B.lp_ipm_state(k=3, stream_switch_iter=-1, r0=1.0, mu0=1.0)
    with pytest.raises(pkg.LPError) as e:
        B.lp_ipm_resume(None, 1, 1, 1, st)
    assert e.value.status == B.LP_ERR_ARG


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle."""
    pkgdir = os.path.join(ROOT, "paper_2003_08072_gb300")
    for fn in os.listdir(pkgdir):
        if fn.endswith(".py"):
            src = open(os.path.join(pkgdir, fn)).read()
            assert not re.search(r"^\s*(from|import)\s+(\.\.)?oracle", src, flags=re.M), fn


def test_footprint_bound_is_host_only_and_monotone(lib):
    """lp_footprint_bytes (admission control of the serving loop) is a pure host computation:
    zero for invalid shapes, at least the matrix copies it must hold, growing with m, n, the
    nonzeros and an extra low-precision copy."""
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    def f(m, n, layout=B.LP_DENSE_COLMAJOR, dt=B.LP_F32, nnz=0, sd=None):
        p = pkg.lp_params_default()
        if sd is not None:
            p.stream_dtype = sd
        return B.lp_footprint_bytes(m, n, layout, dt, nnz, p, 152)

    assert f(0, 10) == 0 and f(20, 10) == 0
    base = f(100, 10_000)
    assert base >= 100 * 10_000 * 4
    assert f(200, 10_000) > base and f(100, 20_000) > base
    # an FP64 A doubles the matrix bytes; an FP32 A also holds 4 double-float column scalars
    # (32 bytes per column) for its FP64-class passes
    assert f(100, 10_000, dt=B.LP_F64) >= base + 100 * 10_000 * 4 - 32 * 10_000
    assert f(100, 10_000, sd=B.LP_BF16) >= base + 100 * 10_000 * 2
    assert f(100, 10_000, layout=B.LP_DENSE_ROWMAJOR) >= base + 100 * 10_000 * 4
    sp = f(100, 10_000, layout=B.LP_CSR, nnz=40_000)
    assert f(100, 10_000, layout=B.LP_CSR, nnz=80_000) >= sp + 40_000 * 8
    assert sp < base
