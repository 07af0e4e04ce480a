"""Serving loop (continuous batching): a mixed stream of dense and CSR LPs of different sizes
submitted at once to a server that can hold only a few of them at a time.  Every request
finishes, the admitted footprints never exceed the budget, and each result is the same as the
instance solved alone (scaled KKT <= 1e-8 recomputed in FP64, objective within 1e-6, IPM
iterations within 1)."""
import numpy as np
import pytest

import synth
from oracle import iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def instance(kind, m, n, seed):
    if kind == "dense":
        lp = synth.dense_lp(seed, m, n, dtype=np.float32)
        return lp, lp.A.astype(np.float64)
    lp = synth.sparse_lp(seed, m, n, nnz_per_col=max(2, m // 50))
    return lp, lp.to_scipy()


def submit(srv, lp, kind):
    import paper_2003_08072_gb300 as pkg

    if kind == "dense":
        return srv.submit(lp.m, lp.n, pkg.LP_DENSE_COLMAJOR, lp.At, lp.b, lp.c)
    return srv.submit(lp.m, lp.n, pkg.LP_CSR, lp.values, lp.b, lp.c, indptr=lp.indptr,
                      indices=lp.indices)


def alone(lp, kind, prm=None):
    import paper_2003_08072_gb300 as pkg

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    if kind == "dense":
        s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    else:
        s = pkg.LPSolver.csr(lp.m, lp.n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                             T(lp.c), params=prm)
    x, y, sv, info = s.solve()
    s.close()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("stream,shared", [("same", 0), ("same", 1), ("bf16", 1)])
def test_mixed_stream_matches_solves_alone(stream, shared):
    """Instances overlapping on their own streams, or (shared) with the dense ones' CG
    iterations in shared launches of the batch engine: every result must still be the
    instance's own."""
    import paper_2003_08072_gb300 as pkg

    pkg.load()
    prm = pkg.lp_params_default()
    prm.shared_cg = shared
    if stream == "bf16":
        prm.stream_dtype = pkg.LP_BF16
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(24):
        kind = "dense" if i % 2 == 0 else "sparse"
        m = int(rng.integers(16, 129))
        n = m * int(rng.integers(20, 61))
        reqs.append((kind, m, n, 100 + i))
    fps = [pkg.lp_footprint_bytes(m, n, pkg.LP_DENSE_COLMAJOR if k == "dense" else pkg.LP_CSR,
                                  pkg.LP_F32, n * max(2, m // 50)) for k, m, n, _ in reqs]
    budget = 3 * max(fps)
    srv = pkg.LPServer(budget, max_live=6, params=prm)
    inst = {}
    for kind, m, n, seed in reqs:
        lp, A = instance(kind, m, n, seed)
        inst[submit(srv, lp, kind)] = (kind, lp, A)
    got = {}
    while len(got) < len(reqs):
        t = srv.wait_any(120_000)
        assert t is not None, "a request did not finish"
        got[t] = srv.result(t)
    st = srv.stats()
    srv.close()
    bad = [(inst[t][0], inst[t][1].m, inst[t][1].n, r["status"], r["error"])
           for t, r in got.items() if r["status"] != 0]
    assert not bad, bad
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["queued"] == 0, st
    assert st["mem_peak"] <= budget
    assert 1 <= st["peak_live"] <= 6
    if shared:
        assert st["batched_cg_solves"] > 0 and st["batched_rounds"] > 0, st
    else:
        assert st["batched_cg_solves"] == 0, st
    for t, r in got.items():
        kind, lp, A = inst[t]
        assert r["status"] == 0, r["error"]
        assert r["latency_s"] >= r["solve_s"] > 0 and r["queued_s"] >= 0
        x, y, s = r["x"], r["y"], r["s"]
        assert max(iipm.kkt_scaled(A, lp.b, lp.c, x, y, s)) <= 1.01e-8
        sprm = pkg.lp_params_default()
        if stream == "bf16" and kind == "dense":
            sprm.stream_dtype = pkg.LP_BF16
        xa, ia = alone(lp, kind, sprm)
        oa = float(lp.c @ xa)
        assert abs(float(lp.c @ x) - oa) <= 1e-6 * abs(oa)
        assert abs(r["info"].ipm_iters - ia.ipm_iters) <= 1


def test_request_larger_than_budget_is_refused():
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(1, 32, 2000, dtype=np.float32)
    srv = pkg.LPServer(1 << 20, max_live=2)   # 1 MiB: below any instance's footprint
    with pytest.raises(pkg.LPError) as e:
        submit(srv, lp, "dense")
    assert e.value.status == pkg._binding.LP_ERR_OOM
    srv.close()


def test_destroy_with_requests_queued():
    """Closing a server drops queued requests and waits for live ones (no hang, no leak)."""
    import paper_2003_08072_gb300 as pkg

    srv = pkg.LPServer(4 << 30, max_live=1)
    for i in range(4):
        lp = synth.dense_lp(200 + i, 24, 1200, dtype=np.float32)
        submit(srv, lp, "dense")
    srv.close()
