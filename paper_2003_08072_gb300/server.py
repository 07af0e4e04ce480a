"""``LPServer``: the library's serving loop (continuous batching) driven from Python.

Requests are host arrays (numpy); the library copies them at submission, admits them by
device-memory footprint, solves up to ``max_live`` of them concurrently on the GPU and hands
results back in completion order.  This module only marshals arguments.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _binding as B


class LPServer:
    def __init__(self, mem_budget_bytes: int, max_live: int = 8,
                 params: Optional[B.lp_params] = None):
        self.params = params if params is not None else B.lp_params_default()
        self.srv = B.lp_server_create(int(mem_budget_bytes), int(max_live), self.params)
        self._shape = {}

    def submit(self, m: int, n: int, layout: int, A_vals: np.ndarray, b: np.ndarray,
               c: np.ndarray, indptr: Optional[np.ndarray] = None,
               indices: Optional[np.ndarray] = None) -> int:
        """Queues min c^T x, A x = b, x >= 0.  Dense: A_vals holds A column-major
        (LP_DENSE_COLMAJOR, e.g. A^T as an (n, m) C array) or row-major; CSR: values with
        int64 indptr and int32 column ids.  FP32 or FP64 values."""
        A_vals = np.ascontiguousarray(A_vals)
        if A_vals.dtype == np.float32:
            dt = B.LP_F32
        elif A_vals.dtype == np.float64:
            dt = B.LP_F64
        else:
            raise TypeError("A must be float32 or float64")
        b = np.ascontiguousarray(b, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        nnz = 0
        if layout == B.LP_CSR:
            indptr = np.ascontiguousarray(indptr, dtype=np.int64)
            indices = np.ascontiguousarray(indices, dtype=np.int32)
            nnz = int(indices.size)
        t = B.lp_server_submit(self.srv, int(m), int(n), layout, dt, A_vals, indptr, indices,
                               nnz, b, c)
        self._shape[t] = (int(m), int(n))
        return t

    def wait_any(self, timeout_ms: int = 1000) -> Optional[int]:
        return B.lp_server_wait_any(self.srv, timeout_ms)

    def result(self, ticket: int) -> dict:
        m, n = self._shape.pop(ticket)
        x, y, s = np.empty(n), np.empty(m), np.empty(n)
        st, info, (queued, solve, latency) = B.lp_server_result(self.srv, ticket, x, y, s)
        return dict(status=st, error=B.last_error() if st else "", x=x, y=y, s=s, info=info,
                    queued_s=queued, solve_s=solve, latency_s=latency)

    def stats(self) -> dict:
        return B.lp_server_stats(self.srv).as_dict()

    def close(self):
        if self.srv:
            B.lp_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
