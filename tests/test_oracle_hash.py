"""Pins of the oracle's sketch generator (oracle/hashing.py) to published facts."""
import os

import numpy as np
import pytest

from oracle import hashing

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    vals = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    return vals


def test_splitmix64_published_sequence():
    """The generator's state advances by the golden gamma; outputs match the published ones."""
    gamma = 0x9E3779B97F4A7C15
    want = _golden_splitmix()
    got = [int(hashing.splitmix64(np.uint64((gamma * k) % 2**64))) for k in range(3)]
    assert got == want


def test_lemire_reduction_bounds_and_monotone():
    width = 1000
    u = np.array([0, 1, 2**31, 2**32 - 1], dtype=np.uint64)
    r = hashing.lemire_reduce(u, width)
    assert r[0] == 0 and r[-1] == width - 1
    assert r[2] == width // 2
    u = np.sort(np.random.default_rng(0).integers(0, 2**32, 10000, dtype=np.uint64))
    r = hashing.lemire_reduce(u, width)
    assert np.all(np.diff(r.astype(np.int64)) >= 0)
    assert r.max() < width


@pytest.mark.parametrize("s", [1, 4])
def test_buckets_in_range_distinct_and_uniform(s):
    n, w = 200_000, 400
    b, sg = hashing.sketch_indices(seed=3, k=5, n=n, s=s, w=w)
    width = w // s
    assert b.shape == (n, s) and b.dtype == np.int64
    for j in range(s):
        assert b[:, j].min() >= j * width and b[:, j].max() < (j + 1) * width
    # chi-square of bucket counts (df = w - 1); 6 sigma band
    cnt = np.bincount(b.reshape(-1), minlength=w)
    e = n * s / w
    chi2 = ((cnt - e) ** 2 / e).sum()
    df = w - 1
    assert abs(chi2 - df) < 6 * np.sqrt(2 * df)
    # signs are balanced
    assert abs(sg.mean()) < 6 / np.sqrt(sg.size)
    assert set(np.unique(sg)) == {-1.0, 1.0}


def test_fresh_w_per_iteration_and_seed():
    b0, s0 = hashing.sketch_indices(1, 0, 1000, 1, 64)
    b1, s1 = hashing.sketch_indices(1, 1, 1000, 1, 64)
    c0, t0 = hashing.sketch_indices(2, 0, 1000, 1, 64)
    assert (b0 != b1).mean() > 0.9 and (b0 != c0).mean() > 0.9
    b0b, s0b = hashing.sketch_indices(1, 0, 1000, 1, 64)
    assert np.array_equal(b0, b0b) and np.array_equal(s0, s0b)


def test_sketch_preserves_norms_in_expectation():
    """E ||W^T z||^2 = ||z||^2 for entries +-1/sqrt(s) with independent signs."""
    from oracle import iipm

    rng = np.random.default_rng(0)
    z = rng.standard_normal(300)
    for s in (1, 4):
        ratios = []
        for k in range(400):
            b, sg = hashing.sketch_indices(9, k, z.size, s, 64)
            W = iipm.sketch_W_dense(b, sg, 64)
            ratios.append(np.sum((W.T @ z) ** 2) / np.sum(z ** 2))
        assert abs(np.mean(ratios) - 1.0) < 0.05


# ------------------------------------------------------------------ Gaussian sketch generator

def test_gaussian_W_moments_and_normality():
    """W's entries times sqrt(w) are N(0, 1): moments within 5 sigma of their sampling error,
    and a Kolmogorov-Smirnov test against the normal CDF."""
    from scipy import stats

    n, w = 5000, 400
    z = (hashing.gaussian_W(0, 3, n, w) * np.sqrt(w)).ravel()
    N = z.size
    assert abs(z.mean()) <= 5 / np.sqrt(N)
    assert abs(z.var() - 1.0) <= 5 * np.sqrt(2.0 / N)
    assert abs(np.mean(z**4) - 3.0) <= 5 * np.sqrt(96.0 / N)
    assert stats.kstest(z[:200_000], "norm").pvalue > 1e-3


def _grid_pin_holds(q):
    """q / 2^8 is the normal quantile of cell j's midpoint to within the 2^-9 rounding: the CDF
    at q_j / 2^8 is (j + 1/2) 2^-14 within phi_max 2^-9 (plus FP64 rounding); the table is odd
    (q_{N-1-j} = -q_j), non-decreasing, integer; each grid value occurs for a run of
    consecutive cells whose count matches the normal mass of its rounding interval to within
    two cells."""
    from scipy import stats

    N = q.size
    if N != 2**14 or not np.array_equal(q, np.rint(q)):
        return False
    if not (np.array_equal(q[::-1], -q) and np.all(np.diff(q) >= 0)):
        return False
    mid = (np.arange(N) + 0.5) / N
    if np.abs(stats.norm.cdf(q / 256.0) - mid).max() > 2.0**-9 / np.sqrt(2 * np.pi) + 1e-15:
        return False
    vals, counts = np.unique(q, return_counts=True)
    mass = stats.norm.cdf((vals + 0.5) / 256) - stats.norm.cdf((vals - 0.5) / 256)
    return bool(np.abs(counts - mass * N).max() <= 2.0)


def test_gaussian_grid_is_the_rounded_normal_quantile_table():
    q = hashing.gaussian_grid()
    assert _grid_pin_holds(q)
    assert np.abs(q).max() == 1026


def test_gaussian_grid_pin_catches_planted_mistakes():
    """Plausible slips in the table each fail the pin: the cell's left edge instead of its
    midpoint, a grid of 2^-7 instead of 2^-8, truncation instead of rounding."""
    from scipy import special

    j = np.arange(2**14, dtype=np.float64)
    left = np.rint(256.0 * special.ndtri(np.maximum(j, 0.5) / 2**14))
    coarse = 2.0 * np.rint(128.0 * special.ndtri((j + 0.5) / 2**14))
    trunc = np.trunc(256.0 * special.ndtri((j + 0.5) / 2**14))
    for bad in (left, coarse, trunc):
        assert not _grid_pin_holds(bad)


def test_gaussian_W_is_a_function_of_seed_and_iteration_only():
    a = hashing.gaussian_W(7, 2, 300, 64)
    assert np.array_equal(a, hashing.gaussian_W(7, 2, 300, 64))
    assert np.array_equal(a[[5, 17]], hashing.gaussian_W(7, 2, 300, 64, rows=[5, 17]))
    assert not np.allclose(a, hashing.gaussian_W(7, 3, 300, 64))
    assert not np.allclose(a, hashing.gaussian_W(8, 2, 300, 64))
    # neighbouring entries are uncorrelated
    z = hashing.gaussian_W(1, 0, 4000, 100).ravel()
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) <= 5 / np.sqrt(z.size)


def test_gaussian_W_is_an_isometry_in_expectation():
    """W W^T -> I_n (entries N(0, 1/w)): for w >> n the deviation is O(sqrt(n/w))."""
    n, w = 40, 40_000
    W = hashing.gaussian_W(0, 1, n, w)
    dev = np.linalg.norm(W @ W.T - np.eye(n), 2)
    assert dev <= 3 * (2 * np.sqrt(n / w) + n / w)


def test_gaussian_sketch_spectrum_within_marchenko_pastur_edges():
    """For the Gaussian sketch, eig(V^T W W^T V) (V: right singular vectors of A D, m of them)
    lie close to the Marchenko-Pastur support [(1 - sqrt(m/w))^2, (1 + sqrt(m/w))^2]."""
    m, n, w = 30, 3000, 600
    rng = np.random.default_rng(4)
    AD = rng.standard_normal((m, n)) * np.exp(rng.uniform(-2, 2, n))[None, :]
    _, _, Vt = np.linalg.svd(AD, full_matrices=False)
    W = hashing.gaussian_W(0, 5, n, w)
    ev = np.linalg.eigvalsh(Vt @ W @ W.T @ Vt.T)
    r = np.sqrt(m / w)
    assert ev.min() >= (1 - r) ** 2 - 0.1 and ev.max() <= (1 + r) ** 2 + 0.1
