"""Writes the FP64 oracle's per-iteration trace of a workload instance to a JSON file here.

The oracle (oracle/iipm.py, Algorithm 2 with the sketch-preconditioned CG of Algorithm 1) runs
on the seeded synthetic instance for at most `max_iter` IPM iterations; every iteration's mu,
scaled KKT residuals, CG iteration count (the cap is Params.cg_max_iter = 500), ||f|| at the end
of CG and step lengths are stored.  Used to tell whether a sketch's behaviour on the GPU is the
method's own: e.g. CountSketch (s = 1, w = 4m) at m = 1000, n = 200000.  Calls only oracle/ and
synth/.

    python tests/golden/make_oracle_trace.py dense 1000 200000 f32 1 60
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
    kind, m, n, dt = sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), sys.argv[4]
    s, max_iter = int(sys.argv[5]), int(sys.argv[6])
    assert kind == "dense"
    lp = synth.dense_lp(0, m, n, dtype=np.float32 if dt == "f32" else np.float64)
    A = np.ascontiguousarray(lp.A, dtype=np.float64)
    t0 = time.perf_counter()
    trace = []

    def cb(k, loc):
        L = loc["log"][-1]
        row = {"k": k, "mu": L.mu, "rp_rel": L.rp_rel, "rd_rel": L.rd_rel, "gap_rel": L.gap_rel,
               "cg_iters": L.cg_iters, "f_norm": L.f_norm, "alpha_max": L.alpha_max,
               "alpha": L.alpha, "seconds": time.perf_counter() - t0}
        trace.append(row)
        print(json.dumps(row), flush=True)

    r = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_s=s, ipm_max_iter=max_iter), callback=cb)
    out = {"workload": f"dense Gaussian LP m={m} n={n} A {dt.upper()} seed 0 (synth.dense_lp)",
           "sketch_s": s, "cg_max_iter": iipm.Params().cg_max_iter, "ipm_max_iter": max_iter,
           "ipm_iters": int(r.iters), "converged": bool(r.converged), "kkt": float(r.kkt),
           "objective": float(r.obj), "cg_total": int(r.cg_total),
           "seconds": time.perf_counter() - t0, "cores": os.cpu_count(), "trace": trace,
           "command": "python tests/golden/make_oracle_trace.py " + " ".join(sys.argv[1:])}
    path = os.path.join(HERE, f"oracle_trace_{kind}_m{m}_n{n}_{dt}_s{s}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "trace"}))


if __name__ == "__main__":
    main()
