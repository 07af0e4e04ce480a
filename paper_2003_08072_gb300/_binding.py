"""ctypes binding of the C ABI in include/lp.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards plain pointers
and sizes; all arithmetic runs in the CUDA library.  Pointers may be given as integers, as
torch tensors (``data_ptr()``) or as numpy arrays (host memory).  A non-OK status raises
``LPError`` carrying the status and the library's message.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from . import build as _build

LP_OK, LP_ERR_ARG, LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_BREAKDOWN = 0, 1, 2, 3, 4
LP_ERR_NOT_CONVERGED, LP_ERR_TIMEOUT, LP_ERR_NUMERIC = 5, 6, 7
LP_DENSE_COLMAJOR, LP_DENSE_ROWMAJOR, LP_CSR = 0, 1, 2
LP_F64, LP_F32, LP_BF16, LP_F16 = 0, 1, 2, 3

LP_INNER_CG, LP_INNER_RICHARDSON = 0, 1
LP_SKETCH_SPARSE, LP_SKETCH_GAUSSIAN = 0, 1
DTYPE_CODES = {"f64": LP_F64, "f32": LP_F32, "bf16": LP_BF16, "f16": LP_F16}


class lp_params(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("cg_rel_tol", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("cg_max_iter", ctypes.c_int32),
        ("ipm_max_iter", ctypes.c_int32),
        ("refine_max", ctypes.c_int32),
        ("sketch_s", ctypes.c_int32),
        ("sketch_w", ctypes.c_int32),
        ("cg_theory_rule", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("stream_dtype", ctypes.c_int),
        ("cg_batch", ctypes.c_int32),
        ("inner_solver", ctypes.c_int32),
        ("sketch_kind", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("gram_tensor_cores", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("shared_cg", ctypes.c_int32),
        ("persistent_cg", ctypes.c_int32),
        ("factor_dag", ctypes.c_int32),
    ]


class lp_info(ctypes.Structure):
    _fields_ = [
        ("ipm_iters", ctypes.c_int32),
        ("cg_iters_total", ctypes.c_int32),
        ("cg_iters_last", ctypes.c_int32),
        ("refine_steps", ctypes.c_int32),
        ("rp_rel", ctypes.c_double),
        ("rd_rel", ctypes.c_double),
        ("gap_rel", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("obj", ctypes.c_double),
        ("alpha_max", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("f_norm", ctypes.c_double),
        ("v_norm", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("f_target", ctypes.c_double),
        ("stream_dtype", ctypes.c_int32),
        ("stream_switch_iter", ctypes.c_int32),
        ("factor_two_stage", ctypes.c_int32),
        ("cg_precise_iter", ctypes.c_int32),
        ("cg_graph_solves", ctypes.c_int32),
        ("cg_persistent_solves", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lp_ipm_state(ctypes.Structure):
    """Algorithm 2's state beyond the iterate (include/lp.h): iteration counter, stream switch,
    and the start point's residual norm and mu."""
    _fields_ = [
        ("k", ctypes.c_int32),
        ("stream_switch_iter", ctypes.c_int32),
        ("r0", ctypes.c_double),
        ("mu0", ctypes.c_double),
    ]


class lp_profile(ctypes.Structure):
    _fields_ = [
        ("phase_ms", ctypes.c_double * 8),
        ("phase_calls", ctypes.c_int64 * 8),
        ("matvec_ms", ctypes.c_double),
        ("matvec_count", ctypes.c_int64),
        ("matvec_bytes", ctypes.c_double),
        ("launches", ctypes.c_int64),
        ("tune_tc", ctypes.c_int32),
        ("tune_stages", ctypes.c_int32),
        ("tune_ctas", ctypes.c_int32),
        ("tune_us", ctypes.c_double),
        ("tune_rule_us", ctypes.c_double),
    ]

    PHASES = ("residuals", "sketch", "factor", "pcg", "rtilde", "correction", "update", "other")

    def as_dict(self):
        return {
            "phase_ms": {k: self.phase_ms[i] for i, k in enumerate(self.PHASES)},
            "phase_calls": {k: int(self.phase_calls[i]) for i, k in enumerate(self.PHASES)},
            "matvec_ms": self.matvec_ms, "matvec_count": int(self.matvec_count),
            "matvec_bytes": self.matvec_bytes, "launches": int(self.launches),
            "tune": {"tc": self.tune_tc, "stages": self.tune_stages,
                     "ctas_per_sm": self.tune_ctas, "us": self.tune_us,
                     "rule_us": self.tune_rule_us},
        }


class lp_server_stats_t(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("queued", ctypes.c_int64), ("live", ctypes.c_int64), ("peak_live", ctypes.c_int64),
        ("mem_in_use", ctypes.c_uint64), ("mem_peak", ctypes.c_uint64),
        ("mem_budget", ctypes.c_uint64),
        ("batched_rounds", ctypes.c_int64), ("batched_cg_solves", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class LPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_str(status)}: {msg}")
        self.status = status


_LIB: Optional[ctypes.CDLL] = None
_VP = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

_SIGNATURES = {
    "lp_params_default": (ctypes.c_int, [ctypes.POINTER(lp_params)]),
    "lp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "lp_last_error": (ctypes.c_char_p, []),
    "lp_create": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I64, ctypes.c_int, ctypes.c_int, _VP,
                                 _VP, _VP, _I64, _VP, _VP, ctypes.POINTER(lp_params), _VP]),
    "lp_destroy": (None, [_VP]),
    "lp_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(lp_params)]),
    "lp_ipm_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, ctypes.POINTER(lp_info)]),
    "lp_ipm_get_state": (ctypes.c_int, [_VP, ctypes.POINTER(lp_ipm_state)]),
    "lp_ipm_resume": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(lp_ipm_state),
                                     ctypes.POINTER(lp_info)]),
    "lp_normal_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP,
                                       ctypes.POINTER(lp_info)]),
    "lp_residuals": (ctypes.c_int, [_VP, _VP, _VP, _VP, _D, _VP, _VP, _VP, ctypes.POINTER(_D)]),
    "lp_sketch_indices": (ctypes.c_int, [ctypes.c_uint64, _I32, _I64, _I32, _I32, _VP, _VP, _VP]),
    "lp_sketch": (ctypes.c_int, [_VP, _VP, _I32, _VP]),
    "lp_factor": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "lp_normal_matvec": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "lp_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _D, _D, _D, _VP, _VP,
                               _VP]),
    "lp_normal_matvec_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, _I32, _I64, _I64, _VP, _VP,
                                                _VP, _VP, _VP]),
    "lp_profile_enable": (ctypes.c_int, [_VP, _I32]),
    "lp_footprint_bytes": (ctypes.c_uint64, [_I32, _I64, ctypes.c_int, ctypes.c_int, _I64,
                                             ctypes.POINTER(lp_params), _I32]),
    "lp_server_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_uint64, _I32,
                                        ctypes.POINTER(lp_params)]),
    "lp_server_submit": (ctypes.c_int, [_VP, _I32, _I64, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                        _VP, _I64, _VP, _VP, ctypes.POINTER(_I64)]),
    "lp_server_wait_any": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I64)]),
    "lp_server_result": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, ctypes.POINTER(lp_info),
                                        ctypes.POINTER(_D)]),
    "lp_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(lp_server_stats_t)]),
    "lp_server_destroy": (None, [_VP]),
    "lp_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(lp_profile), _I32]),
    "lp_test_stall_copy": (ctypes.c_int, [_VP, _I32, ctypes.c_uint64]),
}


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads (building first if needed) the CUDA library; raises if it cannot."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing: run the build first")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _p(x) -> Optional[int]:
    """Pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(st: int):
    if st != LP_OK:
        raise LPError(st, last_error())


def status_str(st: int) -> str:
    return load().lp_status_str(st).decode()


def last_error() -> str:
    return load().lp_last_error().decode()


def lp_params_default() -> lp_params:
    p = lp_params()
    _check(load().lp_params_default(ctypes.byref(p)))
    return p


def lp_create(m, n, layout, a_dtype, A_vals, indptr, indices, nnz, b, c, params=None,
              stream=None) -> int:
    ctx = _VP()
    prm = params if params is not None else lp_params_default()
    _check(load().lp_create(ctypes.byref(ctx), m, n, layout, a_dtype, _p(A_vals), _p(indptr),
                            _p(indices), nnz, _p(b), _p(c), ctypes.byref(prm), _p(stream)))
    return ctx.value


def lp_destroy(ctx: int):
    if ctx:
        load().lp_destroy(ctx)


def lp_set_params(ctx, params: lp_params):
    _check(load().lp_set_params(ctx, ctypes.byref(params)))


def lp_ipm_solve(ctx, x, y, s, start_given=False, check=True) -> lp_info:
    info = lp_info()
    st = load().lp_ipm_solve(ctx, _p(x), _p(y), _p(s), 1 if start_given else 0, ctypes.byref(info))
    if check and st not in (LP_OK,):
        raise LPError(st, last_error())
    return info


def lp_ipm_get_state(ctx) -> lp_ipm_state:
    st = lp_ipm_state()
    _check(load().lp_ipm_get_state(ctx, ctypes.byref(st)))
    return st


def lp_ipm_resume(ctx, x, y, s, state: lp_ipm_state, check=True) -> lp_info:
    info = lp_info()
    st = load().lp_ipm_resume(ctx, _p(x), _p(y), _p(s), ctypes.byref(state), ctypes.byref(info))
    if check and st not in (LP_OK,):
        raise LPError(st, last_error())
    return info


def lp_normal_solve(ctx, x, s, p, k, dy, rtil=None, u=None, Wu=None, Atdy=None) -> lp_info:
    info = lp_info()
    _check(load().lp_normal_solve(ctx, _p(x), _p(s), _p(p), k, _p(dy), _p(rtil), _p(u), _p(Wu),
                                  _p(Atdy), ctypes.byref(info)))
    return info


def lp_residuals(ctx, x, y, s, sigma, rp, rd, p) -> float:
    mu = _D()
    _check(load().lp_residuals(ctx, _p(x), _p(y), _p(s), sigma, _p(rp), _p(rd), _p(p),
                               ctypes.byref(mu)))
    return mu.value


def lp_sketch_indices(seed, k, n, s, w, bucket, sign, stream=None):
    _check(load().lp_sketch_indices(seed, k, n, s, w, _p(bucket), _p(sign), _p(stream)))


def lp_sketch(ctx, d, k, G):
    _check(load().lp_sketch(ctx, _p(d), k, _p(G)))


def lp_factor(ctx, G, Q=None, Minv=None):
    _check(load().lp_factor(ctx, _p(G), _p(Q), _p(Minv)))


def lp_normal_matvec(ctx, d2, v, y, t=None, stream_dtype=LP_F64):
    _check(load().lp_normal_matvec(ctx, _p(d2), _p(v), _p(y), _p(t), stream_dtype))


def lp_step(ctx, x, y, s, rd, dy, Atdy, Wu, mu, eta, mu0, dx=None, ds=None):
    out = (ctypes.c_double * 4)()
    _check(load().lp_step(ctx, _p(x), _p(y), _p(s), _p(rd), _p(dy), _p(Atdy), _p(Wu), mu, eta,
                          mu0, _p(dx), _p(ds), ctypes.cast(out, _VP)))
    return tuple(out)


def lp_profile_enable(ctx, on=True):
    _check(load().lp_profile_enable(ctx, 1 if on else 0))


def lp_profile_read(ctx, reset=False) -> lp_profile:
    p = lp_profile()
    _check(load().lp_profile_read(ctx, ctypes.byref(p), 1 if reset else 0))
    return p


def lp_test_stall_copy(ctx, group, wait_ns):
    """Failure-detection hook: the next staged CG product skips one bulk copy and its bounded
    wait (wait_ns) runs out, so that call returns LP_ERR_TIMEOUT."""
    _check(load().lp_test_stall_copy(ctx, int(group), int(wait_ns)))


def lp_normal_matvec_noalloc(A, a_dtype, m, n, lda, d2, v, y, t=None, stream=None):
    """Context-free A D^2 A^T v that allocates nothing (scratch in a static device array)."""
    _check(load().lp_normal_matvec_noalloc(_p(A), a_dtype, m, n, lda, _p(d2), _p(v), _p(y),
                                           _p(t), _p(stream)))


# ---- memory footprint and the serving loop ----------------------------------------------------

def lp_footprint_bytes(m, n, layout, a_dtype, nnz=0, params: Optional[lp_params] = None,
                       num_sms=0) -> int:
    prm = params if params is not None else lp_params_default()
    return int(load().lp_footprint_bytes(m, n, layout, a_dtype, nnz, ctypes.byref(prm), num_sms))


def lp_server_create(mem_budget_bytes: int, max_live: int, params: Optional[lp_params] = None):
    srv = _VP()
    prm = params if params is not None else lp_params_default()
    _check(load().lp_server_create(ctypes.byref(srv), int(mem_budget_bytes), int(max_live),
                                   ctypes.byref(prm)))
    return srv.value


def lp_server_submit(srv, m, n, layout, a_dtype, A_vals, indptr, indices, nnz, b, c) -> int:
    t = _I64()
    _check(load().lp_server_submit(srv, m, n, layout, a_dtype, _p(A_vals), _p(indptr),
                                   _p(indices), nnz, _p(b), _p(c), ctypes.byref(t)))
    return t.value


def lp_server_wait_any(srv, timeout_ms: int):
    """Ticket of the next finished request, or None after timeout_ms."""
    t = _I64()
    st = load().lp_server_wait_any(srv, int(timeout_ms), ctypes.byref(t))
    if st == LP_ERR_TIMEOUT:
        return None
    _check(st)
    return t.value


def lp_server_result(srv, ticket, x, y, s):
    """(status, lp_info, (queued_s, solve_s, latency_s)); x, y, s host float64 arrays or None."""
    info = lp_info()
    times = (_D * 3)()
    st = load().lp_server_result(srv, ticket, _p(x), _p(y), _p(s), ctypes.byref(info), times)
    return st, info, (times[0], times[1], times[2])


def lp_server_stats(srv) -> lp_server_stats_t:
    out = lp_server_stats_t()
    _check(load().lp_server_stats(srv, ctypes.byref(out)))
    return out


def lp_server_destroy(srv):
    if srv:
        load().lp_server_destroy(srv)
