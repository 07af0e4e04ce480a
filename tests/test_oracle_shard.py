"""Column-sharded algebra of one normal-equation solve, checked on the oracle with two gloo ranks.

Every step of the method is a sum over the columns of A (Sec. 4, running time): r_p = A x - b,
the product A D^2 A^T v, the sketch A D W (W's rows are keyed by the global column index, so a
shard draws its own rows without communication) and W u (rows of W, local to a shard).  A solve
split by columns therefore exchanges one m-vector sum per CG step and one m x w sum per sketch;
everything else is either local or replicated.  The GPU library runs one LP per GPU
(replicas); this test fixes what a column-sharded solve would have to reproduce: each rank owns
half of the columns, sums its partials with all_reduce, and must match the unsharded oracle.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

M, NCOL, K, SEED = 40, 2000, 3, 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import synth
    from oracle import hashing, iipm

    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allsum(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    lp = synth.dense_lp(SEED, M, NCOL)
    A = lp.A
    x, y, s = synth.iterate_point(4, M, NCOL, spread=3.0)
    lo, hi = rank * NCOL // world, (rank + 1) * NCOL // world
    J = slice(lo, hi)
    prm = iipm.Params()
    w = 4 * M
    d2 = x / s
    d = np.sqrt(d2)

    # unsharded reference (every rank holds the whole LP here)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, prm.sigma)
    ref = iipm.normal_solve_sketch(A, x, s, p, K, prm)

    # r_p from the shards: sum_g A_g x_g - b
    rp_sh = allsum(A[:, J] @ x[J]) - lp.b
    # the sketch: global-index hash, local rows of W
    bucket, sign = hashing.sketch_indices(prm.seed, K, NCOL, prm.sketch_s, w)
    G_sh = allsum(iipm.sketch_ADW(A[:, J], d[J], bucket[J], sign[J], w))
    # factor replicated from the summed sketch; CG with one all_reduce per product
    R = iipm.factor_R(G_sh)
    mv = lambda v: allsum(iipm.normal_matvec(A[:, J], d2[J], v))
    cg = iipm.pcg(mv, p, lambda r: iipm.q_inverse_apply(R, r), prm.cg_tol, prm.cg_max_iter,
                  abs_tol=iipm.cg_abs_threshold(x, s, prm))
    rtil = mv(cg.dy) - p
    u, _, _ = iipm.correction_u(G_sh, R, rtil, prm.refine_max)
    Wu_local = iipm.apply_W(u, bucket[J], sign[J])
    dist.destroy_process_group()

    rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    q.put((rank, dict(rp=rel(rp_sh, rp), G=rel(G_sh, ref["G"]), dy=rel(cg.dy, ref["dy"]),
                      iters=(cg.iters, ref["cg"].iters),
                      rtil=float(np.abs(rtil - ref["rtil"]).max() / np.abs(p).max()),
                      u=rel(u, ref["u"]), Wu=rel(Wu_local, ref["Wu"][J]))))


def test_column_shards_reproduce_the_unsharded_solve():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, e in out.items():
        it_sh, it_ref = e.pop("iters")
        assert it_sh == it_ref, (rank, it_sh, it_ref)
        # sums in another order agree to rounding; r~ = A D^2 A^T dy - p is a small difference
        # (CG stopped at a relative residual of 1e-6), so it is compared on the scale of p, and
        # u = (A D W)^dagger r~ inherits r~'s relative error
        assert e["rp"] <= 1e-13 and e["G"] <= 1e-13 and e["dy"] <= 1e-12, (rank, e)
        assert e["rtil"] <= 1e-13, (rank, e)
        assert e["u"] <= 1e-6 and e["Wu"] <= 1e-6, (rank, e)
