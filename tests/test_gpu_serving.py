"""Serving layer (als_server_*): continuous batching of fold-in requests and
budget-admitted factorisation jobs (needs a GB300).

Rows and jobs are independent, so a served result must equal, bit for bit,
what the same kernels give alone: a fold-in request equals als_foldin on the
same model, a job equals a standalone context run for the same iterations.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    r = synth.make_config("tiny")
    return r


def _model(r, n_f, precision, seed=3):
    from paper_1508_03110_gb300 import ALS
    m = ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision=precision)
    m.set_x(synth.init_factors(r.n_u, r.n_m, n_f, seed))
    return m


def _requests(n, n_m, seed):
    ptr, items, vals = synth.foldin_requests(n, n_m, 1, 600, seed=seed)
    return [(items[ptr[q]:ptr[q + 1]], vals[ptr[q]:ptr[q + 1]]) for q in range(n)]


@pytest.mark.parametrize("n_f,precision", [(10, "fp64"), (10, "mixed"), (40, "mixed"), (100, "mixed")])
def test_served_foldin_equals_direct(tiny, n_f, precision):
    from paper_1508_03110_gb300 import Server
    reqs = _requests(300, tiny.n_m, seed=21) + [(np.zeros(0, np.int32), np.zeros(0, np.float32))]
    ptr = np.concatenate([[0], np.cumsum([len(i) for i, _ in reqs])]).astype(np.int64)
    items = np.concatenate([i for i, _ in reqs]).astype(np.int32)
    vals = np.concatenate([v for _, v in reqs]).astype(np.float32)
    with _model(tiny, n_f, precision) as m:
        direct = m.foldin(ptr, items, vals, dtype="float32")
        # small batches, so that requests span many batches and slots
        with Server(m, max_batch=37, max_batch_ratings=20_000, slots=3) as srv:
            tickets = [srv.submit_foldin(i, v) for i, v in reqs]
            got = np.stack([srv.wait(t)[0] for t in tickets])
            st = srv.stats()
    assert np.array_equal(got, direct)
    assert np.all(got[-1] == 0)
    assert st["completed"] == len(reqs)
    assert 0 < st["p50_s"] <= st["p99_s"] and st["requests_per_s"] > 0


def test_served_foldin_matches_oracle(tiny):
    from paper_1508_03110_gb300 import Server
    reqs = _requests(50, tiny.n_m, seed=22)
    x0 = synth.init_factors(tiny.n_u, tiny.n_m, tiny.n_f, 3)
    M = x0[tiny.n_u * tiny.n_f:]
    with _model(tiny, tiny.n_f, "fp64") as m, Server(m) as srv:
        got = np.stack([srv.wait(srv.submit_foldin(i, v))[0] for i, v in reqs])
    for q, (i, v) in enumerate(reqs):
        ref = oracle.foldin(tiny.n_f, tiny.lam, M, np.array([0, len(i)]), i, v.astype(np.float64))[0]
        # FP64 solve, rounded once to FP32 on output
        assert np.max(np.abs(got[q] - ref)) <= 1e-6 * max(np.max(np.abs(ref)), 1e-30) + 1e-30


def test_foldin_from_many_threads(tiny):
    from paper_1508_03110_gb300 import Server
    reqs = _requests(400, tiny.n_m, seed=23)
    ptr = np.concatenate([[0], np.cumsum([len(i) for i, _ in reqs])]).astype(np.int64)
    items = np.concatenate([i for i, _ in reqs]).astype(np.int32)
    vals = np.concatenate([v for _, v in reqs]).astype(np.float32)
    out = [None] * len(reqs)
    with _model(tiny, 40, "mixed") as m:
        direct = m.foldin(ptr, items, vals, dtype="float32")
        with Server(m, max_batch=64) as srv:
            def client(lo):
                for q in range(lo, len(reqs), 4):
                    out[q] = srv.wait(srv.submit_foldin(*reqs[q]))[0]
            th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
            for t in th:
                t.start()
            for t in th:
                t.join()
    assert np.array_equal(np.stack(out), direct)


def _job(seed, n_u=600, n_m=300, nnz=12_000):
    rng = np.random.default_rng(seed)
    key = rng.choice(n_u * n_m, nnz, replace=False)
    rows, cols = (key // n_m).astype(np.int32), (key % n_m).astype(np.int32)
    vals = (rng.integers(1, 11, nnz) * 0.5).astype(np.float32)
    return n_u, n_m, rows, cols, vals


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_served_job_equals_standalone(tiny, precision):
    """A job interleaved with fold-in traffic ends where a standalone context
    ends after the same ALS-NCG iterations."""
    from paper_1508_03110_gb300 import ALS, Server
    n_f, lam, iters = 12, 0.05, 15
    n_u, n_m, rows, cols, vals = _job(5)
    x0 = synth.init_factors(n_u, n_m, n_f, 9)
    with ALS(n_u, n_m, rows, cols, vals, n_f, lam, precision=precision) as a:
        a.set_x(x0)
        for _ in range(iters):
            a.step(info=False)
        ref = a.get_x()
    reqs = _requests(200, tiny.n_m, seed=24)
    with _model(tiny, tiny.n_f, "mixed") as m, Server(m, max_batch=16) as srv:
        tf = [srv.submit_foldin(*q) for q in reqs[:100]]
        tj = srv.submit_job(n_u, n_m, rows, cols, vals, x0, iters, n_f, lam, precision=precision)
        tf += [srv.submit_foldin(*q) for q in reqs[100:]]
        for t in tf:
            srv.wait(t)
        x, lat = srv.wait(tj)
    assert np.array_equal(x.reshape(-1), ref.reshape(-1))
    assert lat > 0


def test_job_admission_by_budget(tiny):
    """A budget that holds one job at a time still runs every job (one after
    another); a job larger than the whole budget is refused at submission."""
    from paper_1508_03110_gb300 import ALS, ALSError, Server
    n_f, lam, iters = 8, 0.05, 5
    jobs = [_job(30 + q) for q in range(3)]
    x0s = [synth.init_factors(j[0], j[1], n_f, 40 + q) for q, j in enumerate(jobs)]
    refs = []
    for (n_u, n_m, rows, cols, vals), x0 in zip(jobs, x0s):
        with ALS(n_u, n_m, rows, cols, vals, n_f, lam) as a:
            a.set_x(x0)
            for _ in range(iters):
                a.step(info=False)
            refs.append(a.get_x())
    with _model(tiny, tiny.n_f, "fp64") as m:
        with Server(m, hbm_budget_bytes=6 << 20, max_jobs=4) as srv:
            ts = [srv.submit_job(*j, x0, iters, n_f, lam) for j, x0 in zip(jobs, x0s)]
            got = [srv.wait(t)[0] for t in ts]
            big = _job(50, n_u=20_000, n_m=5_000, nnz=200_000)
            with pytest.raises(ALSError, match="EBUDGET"):
                srv.submit_job(*big, synth.init_factors(20_000, 5_000, n_f, 1), 1, n_f, lam)
    for g, r_ in zip(got, refs):
        assert np.array_equal(g.reshape(-1), r_.reshape(-1))


def test_server_rejects_bad_requests_and_times_out(tiny):
    from paper_1508_03110_gb300 import ALSError, Server
    with _model(tiny, tiny.n_f, "fp64") as m, Server(m) as srv:
        with pytest.raises(ALSError, match="EINVAL"):
            srv.submit_foldin(np.array([1, tiny.n_m]), np.array([3.0, 4.0]))
        with pytest.raises(ALSError, match="EINVAL"):
            srv.submit_foldin(np.array([1, 2]), np.array([3.0, np.nan]))
        n_u, n_m, rows, cols, vals = _job(7)
        t = srv.submit_job(n_u, n_m, rows, cols, vals, synth.init_factors(n_u, n_m, 8, 2), 40, 8, 0.05)
        with pytest.raises(ALSError, match="ETIMEOUT"):
            srv.wait(t, timeout=0.0)          # just submitted: not finished
        x, _ = srv.wait(t, timeout=120.0)     # the ticket stays valid after a timeout
        assert np.all(np.isfinite(x))


@pytest.mark.parametrize("n_f,precision", [(10, "fp64"), (100, "mixed")])
def test_replayed_load_equals_direct(tiny, n_f, precision):
    """Requests offered by the native open-loop generator (Poisson arrivals at
    2e4 req/s, degrees 1-600, light and heavy rows mixed in every batch) give
    the same answers as als_foldin on the same model, bit for bit."""
    from paper_1508_03110_gb300 import Server
    reqs = _requests(2000, tiny.n_m, seed=24)
    ptr = np.concatenate([[0], np.cumsum([len(i) for i, _ in reqs])]).astype(np.int64)
    items = np.concatenate([i for i, _ in reqs]).astype(np.int32)
    vals = np.concatenate([v for _, v in reqs]).astype(np.float32)
    arrivals = np.cumsum(np.random.default_rng(5).exponential(1.0 / 2e4, size=len(reqs)))
    with _model(tiny, n_f, precision) as m:
        direct = m.foldin(ptr, items, vals, dtype="float32")
        with Server(m, max_batch=128, slots=4) as srv:
            tickets, lag = srv.replay(arrivals, ptr, items, vals)
            got = np.stack([srv.wait(int(t))[0] for t in tickets])
            st = srv.stats()
    assert np.array_equal(got, direct)
    assert st["completed"] == len(reqs) and lag >= 0.0
