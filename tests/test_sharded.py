"""The sharded ALS-NCG driver (users and items in contiguous ratings-balanced
blocks, all-gathers of the fixed side, fixed-order reductions of per-row
terms) on CPU ranks over gloo: the iterates are bit-identical for 1, 2 and 3
ranks, and equal the unsharded oracle's ALS-NCG to rounding."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GRAIN = 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sys.path.insert(0, ROOT)
    import synth
    n_u, n_m, n_f, lam = 90, 50, 4, 0.05
    rows, cols, vals = synth.table_problem(n_u, n_m, seed=3, density=0.2)
    x0 = synth.init_factors(n_u, n_m, n_f, 4)
    return n_u, n_m, n_f, lam, rows, cols, vals, x0


def _worker(rank, world, port, iters, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_1508_03110_gb300.sharded import GlooComm, ShardedALSNCG, balanced_blocks
    from shard_backend import OracleShard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    n_u, n_m, n_f, lam, rows, cols, vals, x0 = _problem()
    ub = balanced_blocks(np.bincount(rows, minlength=n_u), world, GRAIN)
    mb = balanced_blocks(np.bincount(cols, minlength=n_m), world, GRAIN)
    be = OracleShard(n_u, n_m, n_f, lam, rows, cols, vals, ub, mb, rank)
    drv = ShardedALSNCG(be, GlooComm(dist), rank, world, n_u, n_m, n_f, lam, ub, mb, GRAIN)
    X = x0.reshape(n_u + n_m, n_f)
    infos = []
    U, M = drv.run(X[ub[rank]:ub[rank + 1]], X[n_u + mb[rank]:n_u + mb[rank + 1]], iters,
                   on_iter=lambda k, i: infos.append(i))
    Ufull, Mfull = drv.gather_rows(U), drv.gather_rows(M)
    out.put((rank, np.concatenate([Ufull.reshape(-1), Mfull.reshape(-1)]),
             [(i["alpha"], i["beta"], i["gnorm"], i["fallback"]) for i in infos], ub, mb))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, iters):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, iters, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_balanced_blocks_on_the_grain():
    from paper_1508_03110_gb300.sharded import balanced_blocks
    rng = np.random.default_rng(0)
    deg = rng.integers(0, 50, size=1000)
    for world in (1, 2, 3, 7):
        b = balanced_blocks(deg, world, 16)
        assert b[0] == 0 and b[-1] == 1000 and all(x % 16 == 0 for x in b[:-1])
        assert all(b[i] <= b[i + 1] for i in range(world))
        w = np.array([np.sum(deg[b[i]:b[i + 1]] + 1) for i in range(world)])
        assert w.max() <= (deg + 1).sum() / world + 16 * 50 + 16


def test_sharded_iterates_bitwise_for_any_rank_count_and_match_oracle():
    import oracle
    iters = 8
    base = _run(1, iters)[0]
    for world in (2, 3):
        res = _run(world, iters)
        for rank, x, infos, ub, mb in res:
            assert len(set(ub)) == world + 1 and len(set(mb)) == world + 1   # every block non-empty
            assert np.array_equal(x, base[1]), (world, rank)        # bit-identical iterates
            assert infos == base[2]                                 # same alpha, beta, |g|, branch
    n_u, n_m, n_f, lam, rows, cols, vals, x0 = _problem()
    P = oracle.build_problem(n_u, n_m, n_f, lam, rows, cols, vals)
    ref = oracle.alsncg(P, x0, iters)
    assert np.linalg.norm(base[1] - ref[-1].x) <= 1e-11 * np.linalg.norm(ref[-1].x)
    for (alpha, beta, gn, fb), r in zip(base[2], ref):
        assert fb == r.fallback and alpha == pytest.approx(r.alpha, rel=1e-12)
        assert gn == pytest.approx(r.gnorm, rel=1e-9)
