"""The allocation-free A D^2 A^T v entry point against the context-based one and against FP64.

Some callers cannot allocate device memory (a framework that owns all device memory through
its own pool, or a loop that cannot absorb cudaMalloc's implicit synchronisation), so
lp_normal_matvec_noalloc keeps its partial sums in a static device array.  This file is
collected last so that a failure here does not hide earlier results; it passes alone in a
fresh process (the first call does the per-device set-up) and after the other tests.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCRATCH_BYTES = 4 << 20


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _codes():
    import paper_2003_08072_gb300 as pkg

    return {"f64": pkg.LP_F64, "f32": pkg.LP_F32, "bf16": pkg.LP_BF16, "f16": pkg.LP_F16}


TORCH_DT = {"f64": "float64", "f32": "float32", "bf16": "bfloat16", "f16": "float16"}


def _tol(dt, m):
    # FP64 rounding of the passes, or FP32 accumulation of a streamed copy (the matvec tests)
    return 1e-12 if dt == "f64" else 64 * 2.0**-24 * math.sqrt(m)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16", "f16"])
def test_noalloc_matches_context_entry_point_twice(dt):
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    assert torch.cuda.is_available()
    m, n = 300, 20_011
    code = _codes()[dt]
    lp = synth.dense_lp(21, m, n, dtype=np.float64 if dt == "f64" else np.float32)
    prm = pkg.lp_params_default()
    if dt in ("bf16", "f16"):
        prm.stream_dtype = code
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    # the caller's own copy of A: column-major with lda = m rounded up to 16 bytes (zero rows)
    tdt = getattr(torch, TORCH_DT[dt])
    esz = torch.empty(0, dtype=tdt).element_size()
    lda = m + (-m) % (16 // esz)
    A_dev = torch.zeros(n, lda, dtype=tdt, device="cuda")
    A_dev[:, :m] = T(lp.At).to(tdt)
    A64 = A_dev[:, :m].double().cpu().numpy().T        # the exact values the kernels stream
    x, y, s = synth.iterate_point(22, m, n, spread=3.0)
    d2h = x / s
    d2 = T(d2h)
    rng = np.random.default_rng(23)
    stream = torch.cuda.current_stream().cuda_stream
    tol = _tol(dt, m)
    for call in range(2):
        v = rng.standard_normal(m)
        y_ctx = solver.normal_matvec(d2, T(v), pkg.LP_F64 if dt == "f64" else code).cpu().numpy()
        y_na = torch.empty(m, dtype=torch.float64, device="cuda")
        t_na = torch.empty(n, dtype=torch.float64, device="cuda")
        B.lp_normal_matvec_noalloc(A_dev, code, m, n, lda, d2, T(v), y_na, t_na, stream)
        torch.cuda.synchronize()
        y_na = y_na.cpu().numpy()
        ref = A64 @ (d2h * (A64.T @ v))
        scale = np.abs(A64) @ (d2h * (np.abs(A64).T @ np.abs(v)))
        assert np.all(np.abs(y_na - ref) <= tol * scale), call
        # both entry points stream the same rounded A (the context's 16-bit copy is scaled by
        # powers of two), each within the bound, so within twice the bound of each other
        assert np.all(np.abs(y_na - y_ctx) <= 2 * tol * scale), call
        ref_t = A64.T @ v
        tscale = np.abs(A64).T @ np.abs(v)
        assert np.all(np.abs(t_na.cpu().numpy() - ref_t) <= tol * tscale), call
    solver.close()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_noalloc_ignores_nonfinite_padding_rows(dt):
    """lda > m with NaN and Inf in rows m..lda-1: the padding must not reach y or t."""
    from paper_2003_08072_gb300 import _binding as B

    code = _codes()[dt]
    m, n, pad = 37, 5_003, 11 if dt == "f32" else 3   # lda * element size a multiple of 16
    lda = m + pad
    rng = np.random.default_rng(31)
    A = rng.standard_normal((n, m))
    buf = np.full((n, lda), np.nan)
    buf[:, :m] = A
    buf[::2, m] = np.inf
    tdt = getattr(torch, TORCH_DT[dt])
    A_dev = torch.from_numpy(buf).to(tdt).cuda().contiguous()
    A64 = A_dev[:, :m].double().cpu().numpy().T
    d2h = rng.uniform(0.1, 10.0, n)
    v = rng.standard_normal(m)
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    B.lp_normal_matvec_noalloc(A_dev, code, m, n, lda, T(d2h), T(v), y, t)
    torch.cuda.synchronize()
    ref = A64 @ (d2h * (A64.T @ v))
    scale = np.abs(A64) @ (d2h * (np.abs(A64).T @ np.abs(v)))
    yh = y.cpu().numpy()
    assert np.isfinite(yh).all() and np.isfinite(t.cpu().numpy()).all()
    assert np.all(np.abs(yh - ref) <= _tol(dt, m) * scale)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_scratch_limit_edge(dt):
    """The largest m the 4 MiB scratch admits on this GPU works; the next one is rejected."""
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    acc = 8 if dt == "f64" else 4
    m_max = min(8192, SCRATCH_BYTES // (acc * sms))
    # round m_max down so that m * element size is a multiple of 16 (lda = m)
    esz = 8 if dt == "f64" else 4
    step = 16 // esz
    m_ok = m_max - m_max % step
    n = 64
    rng = np.random.default_rng(41)
    At = rng.standard_normal((n, m_ok))
    tdt = getattr(torch, TORCH_DT[dt])
    A_dev = torch.from_numpy(At).to(tdt).cuda().contiguous()
    A64 = A_dev.double().cpu().numpy().T
    d2h = rng.uniform(0.5, 2.0, n)
    v = rng.standard_normal(m_ok)
    y = torch.empty(m_ok, dtype=torch.float64, device="cuda")
    B.lp_normal_matvec_noalloc(A_dev, _codes()[dt], m_ok, n, m_ok, T(d2h), T(v), y)
    torch.cuda.synchronize()
    ref = A64 @ (d2h * (A64.T @ v))
    scale = np.abs(A64) @ (d2h * (np.abs(A64).T @ np.abs(v)))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= _tol(dt, m_ok) * scale)
    # one row more than the scratch admits (lda rounded up to a 16-byte multiple)
    m_bad = m_max + 1
    lda_bad = m_bad + (-m_bad) % step
    A_bad = torch.zeros(n, lda_bad, dtype=tdt, device="cuda")
    vb = torch.ones(m_bad, dtype=torch.float64, device="cuda")
    yb = torch.empty(m_bad, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LPError) as e:
        B.lp_normal_matvec_noalloc(A_bad, _codes()[dt], m_bad, n, lda_bad, T(d2h), vb, yb)
    assert e.value.status == B.LP_ERR_ARG
    assert "scratch limit" in str(e.value)


def test_noalloc_allocates_no_device_memory():
    """Across a warmed-up call neither torch's allocator nor the driver's free memory moves."""
    from paper_2003_08072_gb300 import _binding as B

    m, n = 256, 30_000
    rng = np.random.default_rng(51)
    A_dev = T(rng.standard_normal((n, m)).astype(np.float32))
    d2 = T(rng.uniform(0.5, 2.0, n))
    v = T(rng.standard_normal(m))
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    B.lp_normal_matvec_noalloc(A_dev, _codes()["f32"], m, n, m, d2, v, y, t, stream)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.lp_normal_matvec_noalloc(A_dev, _codes()["f32"], m, n, m, d2, v, y, t, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
