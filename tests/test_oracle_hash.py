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
