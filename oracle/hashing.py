"""Counter-based hash that generates the sparse sketching matrix W.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper asks for a sparse embedding W (n x w) with O(log(r/delta)) nonzeros
per row (Sec. 2, Eq. pdprec) and calls it a Count-Min / CountSketch matrix
(Sec. 5); it does not fix how the random buckets and signs are drawn.  This
module fixes them from two published definitions so that the oracle and the
GPU path can generate the same W independently:

* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one step from state x
  outputs mix(x + 0x9E3779B97F4A7C15), where mix is the 64-bit finaliser with
  shifts 30/27/31 and multipliers 0xBF58476D1CE4E5B9 / 0x94D049BB133111EB.
  ``splitmix64(x)`` below is that first output for state x.
* Lemire's multiply-shift range reduction (Lemire, ACM TOMS 2019):
  floor(u32 * range / 2^32) maps a 32-bit value into [0, range).

Entry (i, j) of the s nonzeros in row i of W for IPM iteration k:
    key_k  = splitmix64(seed ^ splitmix64(k))
    h      = splitmix64(key_k ^ (i*s + j))
    bucket = j*(w/s) + ((h >> 32) * (w/s)) >> 32     (block j of width w/s)
    sign   = -1 if (h & 1) else +1;   value = sign / sqrt(s)
The block layout (one bucket per block) keeps the s buckets of a row
distinct, as in OSNAP; with s = 1 this is CountSketch.  W is redrawn each IPM
iteration (Algorithm 2, step (a)) by changing k, and the same W serves the
preconditioner and the correction vector of that iteration (Sec. 4, after
Lemma 4.1).

The Gaussian W (Sec. 5, and the sketch of the experiments, Sec. 6) is drawn from the same key
by inverting the normal CDF on 2^14 equiprobable cells, its values rounded to a grid of 2^-8
(``gaussian_W``), so that both sides produce it exactly.
"""
from __future__ import annotations

import numpy as np
from scipy import special

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """First SplitMix64 output for state ``x`` (uint64 scalar or array)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def iteration_key(seed: int, k: int) -> np.uint64:
    """Per-IPM-iteration key: W depends only on (seed, k)."""
    return np.uint64(splitmix64(np.uint64(seed) ^ splitmix64(np.uint64(k))))


def lemire_reduce(u32, rng_size: int):
    """floor(u32 * rng_size / 2^32) for 32-bit ``u32`` (uint64 array)."""
    with np.errstate(over="ignore"):
        return (np.asarray(u32, dtype=np.uint64) * np.uint64(rng_size)) >> np.uint64(32)


def sketch_indices(seed: int, k: int, n: int, s: int, w: int):
    """Buckets and signs of W for iteration k.

    Returns ``bucket`` (int64, shape (n, s)) and ``sign`` (float64, +-1,
    shape (n, s)).  Requires w % s == 0.
    """
    if w % s != 0:
        raise ValueError("w must be a multiple of s")
    width = w // s
    key = iteration_key(seed, k)
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(s, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        h = splitmix64(key ^ (i * np.uint64(s) + j))
    bucket = (np.arange(s, dtype=np.int64)[None, :] * width
              + lemire_reduce(h >> np.uint64(32), width).astype(np.int64))
    sign = np.where((h & np.uint64(1)) == 1, -1.0, 1.0)
    return bucket, sign


GAUSS_BITS = 14   # the Gaussian W draws from 2^14 equiprobable quantile cells


def gaussian_grid() -> np.ndarray:
    """Values of the Gaussian sketch's entries times sqrt(w) 2^8: for cell j of 2^14 equally
    likely cells, q_j = round(2^8 Phi^{-1}((j + 1/2) 2^-14)) (Phi the standard normal CDF, by
    scipy's ndtri), an integer with |q_j| <= 1026."""
    j = np.arange(2**GAUSS_BITS, dtype=np.float64)
    return np.rint(256.0 * special.ndtri((j + 0.5) * 2.0**-GAUSS_BITS))


def gaussian_W(seed: int, k: int, n: int, w: int, rows=None) -> np.ndarray:
    """Dense Gaussian sketching matrix W (n x w) of iteration k, entries ~ N(0, 1/w).

    The Gaussian sketch of the paper's experiments (Sec. 6) and of Sec. 5, generated from the
    same per-iteration key by inversion of the normal CDF: for entry (i, b), with t = i*w + b,
        h = splitmix64(key_k ^ t),  j = h >> 50  (one of 2^14 equiprobable cells),
        W[i, b] = q_j / (2^8 sqrt(w)),  q_j = round(2^8 Phi^{-1}((j + 1/2) 2^-14)).
    The entries are N(0, 1) quantiles on a grid of 2^-8 (the distribution's mass per cell is
    2^-14, its tails cut at 4.0 sigma), scaled by 1/sqrt(w); being integers over 2^8 sqrt(w),
    they are the same on every side that evaluates them, and the sketch A D W can be formed
    exactly from a fixed-point split of A D.
    ``rows`` restricts the output to those row indices (default: all n).
    """
    key = iteration_key(seed, k)
    i = (np.arange(n, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64))[:, None]
    b = np.arange(w, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        t = i * np.uint64(w) + b
        h = splitmix64(key ^ t)
    cell = (h >> np.uint64(64 - GAUSS_BITS)).astype(np.int64)
    return gaussian_grid()[cell] / (256.0 * np.sqrt(w))
