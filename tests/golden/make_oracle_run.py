"""Writes the FP64 oracle's own end-to-end run of a workload instance to a JSON file here.

The oracle (oracle/iipm.py, Algorithm 2 with the sketch-preconditioned CG of Algorithm 1) is
run to the stopping rule on the seeded synthetic instance, and its IPM iteration count, CG
product count, objective, scaled KKT residual and wall time are stored.  bench.py uses the
iteration count to convert the oracle's measured time per IPM iteration into LPs/s, so that
its CPU baseline and its reference arm count the iterations the oracle itself takes on the
very instance the GPU solves.  Calls only oracle/ and synth/.

    python tests/golden/make_oracle_run.py dense 1000 200000 f32 4
    python tests/golden/make_oracle_run.py scaled 2000 500000 f32 4   (columns scaled by 10^U(-3,3))
    python tests/golden/make_oracle_run.py sparse 5000 2000000 f32 4  (CSR, 8 nonzeros per column)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import iipm  # noqa: E402


def main():
    kind, m, n, dt, s = sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), sys.argv[4], int(sys.argv[5])
    assert kind in ("dense", "scaled", "sparse")
    if kind == "sparse":
        lp = synth.sparse_lp(0, m, n, nnz_per_col=8)
        A = lp.to_scipy().astype(np.float64)
    else:
        lp = synth.dense_lp(0, m, n, dtype=np.float32 if dt == "f32" else np.float64,
                            col_scale=(-3, 3) if kind == "scaled" else None)
        A = np.ascontiguousarray(lp.A, dtype=np.float64)
    t0 = time.perf_counter()
    r = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_s=s))
    secs = time.perf_counter() - t0
    if kind == "sparse":
        desc, gen = "sparse LP, 8 nonzeros per column, CSR", "synth.sparse_lp"
    else:
        desc = "dense Gaussian LP" + (" with column scales 10^U(-3,3)" if kind == "scaled" else "")
        gen = "synth.dense_lp"
    out = {"workload": f"{desc} m={m} n={n} A {dt.upper()} seed 0 ({gen})",
           "sketch_s": s, "ipm_iters": int(r.iters), "cg_total": int(r.cg_total),
           "objective": float(r.obj), "kkt": float(r.kkt), "converged": bool(r.converged),
           "seconds": secs, "cores": os.cpu_count(),
           "command": "python tests/golden/make_oracle_run.py " + " ".join(sys.argv[1:])}
    path = os.path.join(HERE, f"oracle_run_{kind}_m{m}_n{n}_{dt}_s{s}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
