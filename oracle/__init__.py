"""FP64 CPU oracle of the sketch-preconditioned infeasible IPM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The CUDA library never calls it, shares no code with it and has no fallback
to it.

Contents
  hashing.py  SplitMix64 counter hash and Lemire range reduction that define
              the sparse sketching matrix W (Sec. 2, Eq. pdprec; the paper
              leaves the construction open, we fix one from its published
              definitions).
  iipm.py     Algorithm 2 (infeasible IPM) with Algorithm 1 (sketch-
              preconditioned CG) as the inner solver, plus the exact
              Cholesky variant ("IPM w/ Dir." of Sec. 6).  Plain numpy/scipy
              in float64; every function cites the passage it follows.
  vertex.py   brute-force vertex enumeration for tiny LPs.

Parity status per function is recorded in the module docstrings; every
function is pinned by at least one ``-m "not gpu"`` test against a fact the
paper or the mathematics fixes (see tests/test_oracle_*.py).
"""
