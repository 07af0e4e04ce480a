"""``LPSolver``: one library context driven with torch tensors (marshalling only).

Device buffers are allocated with PyTorch; every computation is a call into the CUDA library
(include/lp.h).  Inputs given as numpy arrays or CPU tensors are copied by the library
(cudaMemcpyDefault); outputs are CUDA float64 tensors unless stated otherwise.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _binding as B


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("LPSolver needs a CUDA device (no CPU fallback exists)")
    return torch


def _keep(x):
    """Returns an object whose pointer stays valid for the call (contiguous arrays)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x)
    if hasattr(x, "is_contiguous"):
        return x.contiguous()
    return x


class LPSolver:
    """Standard-form LP  min c^T x, A x = b, x >= 0  on one GPU (Sec. 1 of the paper)."""

    def __init__(self, m: int, n: int, layout: int, a_dtype: int, A_vals, b, c, indptr=None,
                 indices=None, nnz: int = 0, params: Optional[B.lp_params] = None, stream=None):
        torch = _torch()
        self.m, self.n = int(m), int(n)
        self.params = params if params is not None else B.lp_params_default()
        self._stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        keep = [_keep(v) for v in (A_vals, b, c, indptr, indices)]
        self.ctx = B.lp_create(self.m, self.n, layout, a_dtype, keep[0], keep[3], keep[4], nnz,
                               keep[1], keep[2], self.params, self._stream)
        self.w = self.params.sketch_w or 4 * self.m

    # ---- constructors ----------------------------------------------------------------------
    @classmethod
    def dense(cls, At, b, c, params=None, stream=None):
        """A given as A^T with shape (n, m), C-contiguous (A column-major); float64 or float32."""
        n, m = At.shape
        dt = B.LP_F32 if str(At.dtype).endswith("float32") else B.LP_F64
        return cls(m, n, B.LP_DENSE_COLMAJOR, dt, At, b, c, params=params, stream=stream)

    @classmethod
    def csr(cls, m, n, indptr, indices, values, b, c, params=None, stream=None):
        dt = B.LP_F32 if str(values.dtype).endswith("float32") else B.LP_F64
        return cls(m, n, B.LP_CSR, dt, values, b, c, indptr=indptr, indices=indices,
                   nnz=int(len(values)), params=params, stream=stream)

    # ---- helpers ---------------------------------------------------------------------------
    def _vec(self, k):
        torch = _torch()
        return torch.empty(k, dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "ctx", None):
            B.lp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: B.lp_params):
        B.lp_set_params(self.ctx, params)
        self.params = params

    # ---- entry points ----------------------------------------------------------------------
    def solve(self, x=None, y=None, s=None, check: bool = True):
        """Algorithm 2 end to end; returns (x, y, s, info).  x, y, s: optional start (device)."""
        start = x is not None
        xv = x.clone() if start else self._vec(self.n)
        yv = y.clone() if start else self._vec(self.m)
        sv = s.clone() if start else self._vec(self.n)
        info = B.lp_ipm_solve(self.ctx, xv, yv, sv, start_given=start, check=check)
        return xv, yv, sv, info

    def solve_host(self, x: np.ndarray, y: np.ndarray, s: np.ndarray, start_given: bool = False,
                   check: bool = True):
        """Algorithm 2 with host (numpy float64) iterate buffers, copied inside the call."""
        return B.lp_ipm_solve(self.ctx, x, y, s, start_given=start_given, check=check)

    def state(self):
        """Algorithm 2's state after the last solve or resume (a checkpoint with x, y, s)."""
        return B.lp_ipm_get_state(self.ctx)

    def resume(self, x, y, s, state, check: bool = True):
        """Continues a solve from the iterate (x, y, s) (device) and its saved state; returns
        (x, y, s, info) with info.ipm_iters the total iteration count."""
        xv, yv, sv = x.clone(), y.clone(), s.clone()
        info = B.lp_ipm_resume(self.ctx, xv, yv, sv, state, check=check)
        return xv, yv, sv, info

    def residuals(self, x, y, s, sigma=None):
        sigma = self.params.sigma if sigma is None else sigma
        rp, rd, p = self._vec(self.m), self._vec(self.n), self._vec(self.m)
        mu = B.lp_residuals(self.ctx, x, y, s, sigma, rp, rd, p)
        return rp, rd, p, mu

    def normal_solve(self, x, s, p, k: int):
        dy, rtil, u = self._vec(self.m), self._vec(self.m), self._vec(self.w)
        Wu, Atdy = self._vec(self.n), self._vec(self.n)
        info = B.lp_normal_solve(self.ctx, x, s, p, k, dy, rtil, u, Wu, Atdy)
        return dict(dy=dy, rtil=rtil, u=u, Wu=Wu, Atdy=Atdy, info=info)

    def sketch(self, d, k: int):
        torch = _torch()
        G = torch.empty(self.w, self.m, dtype=torch.float64, device="cuda")  # G^T rows = columns of G
        B.lp_sketch(self.ctx, d, k, G)
        return G.T  # (m, w) view of the column-major result

    def factor(self, G_colmajor):
        """G_colmajor: (w, m) contiguous tensor holding G column-major.  Returns (Q, Minv)."""
        torch = _torch()
        Q = torch.empty(self.m, self.m, dtype=torch.float64, device="cuda")
        Mi = torch.empty(self.m, self.m, dtype=torch.float64, device="cuda")
        B.lp_factor(self.ctx, G_colmajor, Q, Mi)
        return Q, Mi

    def normal_matvec(self, d2, v, stream_dtype=B.LP_F64, want_t=False):
        y = self._vec(self.m)
        t = self._vec(self.n) if want_t else None
        B.lp_normal_matvec(self.ctx, d2, v, y, t, stream_dtype)
        return (y, t) if want_t else y

    def step(self, x, y, s, rd, dy, Atdy, Wu, mu, eta, mu0):
        dx, ds = self._vec(self.n), self._vec(self.n)
        out = B.lp_step(self.ctx, x, y, s, rd, dy, Atdy, Wu, mu, eta, mu0, dx, ds)
        return dx, ds, out
