"""Host-side tables of the library, compiled from its headers with the host C++ compiler (no GPU).

* The Gaussian sketch's quantile table (gauss_grid.h, bisection on erfc) equals the oracle's
  (scipy's ndtri), integer for integer: the two sides draw the same W.
* The task list of the one-launch Cholesky sweep (chol_tasks.h) is complete and in an order in
  which the launch always makes progress, and every tile receives its operations in the order
  of the block-step sweep (so both routes give bitwise the same factor).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hashing

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2003_08072_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "chol_tasks.h"
#include "gauss_grid.h"
int main(int argc, char** argv) {
  if (argc > 1) {
    const int nbk = std::atoi(argv[1]);
    std::vector<uint32_t> t(lpk::chol_dag_tasks(nbk, nullptr));
    lpk::chol_dag_tasks(nbk, t.data());
    for (uint32_t c : t) std::printf("%u\n", c);
    return 0;
  }
  static int16_t q[1 << lpk::kGaussBits];
  lpk::gauss_grid(q);
  for (int16_t v : q) std::printf("%d\n", v);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("host_tables")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(exe, *args):
    out = subprocess.run([exe, *map(str, args)], check=True, capture_output=True, text=True).stdout
    return np.array([int(x) for x in out.split()], dtype=np.int64)


def test_gaussian_table_matches_oracle(harness):
    q = run(harness)
    assert np.array_equal(q, hashing.gaussian_grid().astype(np.int64))


F, T, U, XS, XU = 0, 1, 2, 3, 4


def simulate(codes, nbk):
    """Runs the tasks in list order on one worker, advancing the chain task F whenever the next
    task's inputs are not ready (as a waiting CTA leaves F, claimed first, running).  The waits
    are the kernel's: per tile a counter, cA[i][j] = trailing updates applied, j + 1 once final
    (L_ij; for i = j also X_jj), cX[i][j] = updates of X_ij applied, i - j + 1 once final.
    Returns the per-tile operation sequences; fails on a task that can never run."""
    cA, cX = {}, {}
    g = lambda d, i, j: d.get((i, j), 0)
    opsA, opsX = {}, {}
    fk = [0]   # the chain's next block step

    def f_ready():
        k = fk[0]
        return k < nbk and (k == 0 or (g(cA, k, k - 1) >= k - 1 and g(cA, k, k) >= k - 1))

    def f_run():
        k = fk[0]
        if k > 0:
            assert g(cA, k - 1, k - 1) == k
            cA[(k, k - 1)] = k
            opsA.setdefault((k, k - 1), []).append(("final", k - 1))
            opsA.setdefault((k, k), []).append(("upd", k - 1))
        cA[(k, k)] = k + 1
        opsA.setdefault((k, k), []).append(("final", k))
        fk[0] += 1

    def ready(kind, i, j, k):
        if kind == T:
            return g(cA, i, k) >= k and g(cA, k, k) >= k + 1
        if kind == U:
            return g(cA, i, k) >= k + 1 and g(cA, j, k) >= k + 1 and g(cA, i, j) >= k
        if kind == XS:
            return g(cA, k, k) >= k + 1 and g(cX, k, j) >= k - j
        xkj = g(cA, k, k) >= k + 1 if j == k else g(cX, k, j) >= k - j + 1
        return g(cA, i, k) >= k + 1 and xkj and g(cX, i, j) >= k - j

    assert codes[0] >> 27 == F
    for c in codes[1:]:
        kind, i, j, k = c >> 27, (c >> 18) & 511, (c >> 9) & 511, c & 511
        while not ready(kind, i, j, k):
            assert f_ready(), ("no task can run", nbk, kind, i, j, k)
            f_run()
        if kind == T:
            assert g(cA, i, k) == k
            cA[(i, k)] = k + 1
            opsA.setdefault((i, k), []).append(("final", k))
        elif kind == U:
            assert g(cA, i, j) == k
            cA[(i, j)] = k + 1
            opsA.setdefault((i, j), []).append(("upd", k))
        elif kind == XS:
            assert g(cX, k, j) == k - j
            cX[(k, j)] = k - j + 1
            opsX.setdefault((k, j), []).append(("final", k))
        else:
            assert g(cX, i, j) == k - j
            cX[(i, j)] = k - j + 1
            opsX.setdefault((i, j), []).append(("upd", k))
    while f_ready():
        f_run()
    assert fk[0] == nbk
    return opsA, opsX


@pytest.mark.parametrize("nbk", [1, 2, 3, 4, 7, 17, 32])
def test_cholesky_task_list(harness, nbk):
    codes = run(harness, nbk)
    assert len(codes) == len(set(codes.tolist()))
    # F once, T per (i >= k + 2), XS per j < k, U per k < j <= i but (k+1, k+1), XU per i > k >= j
    r = np.arange(nbk)
    expect = 1 + sum(max(0, nbk - k - 2) for k in r) + sum(k for k in r) \
        + sum((nbk - k - 1) * (nbk - k) // 2 - (1 if k + 1 < nbk else 0) for k in r) \
        + sum((nbk - k - 1) * (k + 1) for k in r)
    assert len(codes) == expect
    opsA, opsX = simulate(codes, nbk)
    # the block-step sweep: tile (i, j) of A gets the updates of steps 0 .. j-1, then becomes
    # final at step j; tile (i, j) of X (i > j) the updates of steps j .. i-1, then its scaling
    for i in range(nbk):
        for j in range(i + 1):
            assert opsA[(i, j)] == [("upd", q) for q in range(j)] + [("final", j)]
            if i > j:
                assert opsX[(i, j)] == [("upd", q) for q in range(j, i)] + [("final", i)]
