"""Batched independent factorisations in one context (block-diagonal layout,
per-problem line search / beta / stopping test) against the oracle run on
each problem alone (needs a GB300)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def batch():
    return synth.make_batch(6, 1_000, 30_000, 0.01, 0.05, seed=4)


@pytest.mark.parametrize("n_f", [5, 40])
def test_batched_fp64_matches_oracle_per_problem(batch, n_f):
    from paper_1508_03110_gb300 import ALSBatch
    lam = 0.05
    xs = [synth.init_factors(nu, nm, n_f, 10 + q) for q, (nu, nm, *_rest) in enumerate(batch)]
    refs = []
    for (nu, nm, r, c, v), x0 in zip(batch, xs):
        P = oracle.build_problem(nu, nm, n_f, lam, r, c, v)
        refs.append(oracle.alsncg(P, x0, 6))
    with ALSBatch(batch, n_f, lam, precision="fp64") as m:
        m.set_x(m.join_x(xs))
        for k in range(6):
            m.step(info=False)
            got = m.split_x(m.get_x())
            for q in range(len(batch)):
                assert _rel(got[q], refs[q][k].x) < 1e-9, (q, k, _rel(got[q], refs[q][k].x))
        infos = m.infos()
    for q in range(len(batch)):
        assert infos[q]["f"] == pytest.approx(refs[q][-1].f, rel=1e-9)
        assert infos[q]["gnorm"] == pytest.approx(refs[q][-1].gnorm, rel=1e-6, abs=1e-9 * infos[q]["gnorm0"])


def test_batched_mixed_converges_each_problem(batch):
    from paper_1508_03110_gb300 import ALSBatch
    n_f = 40
    xs = [synth.init_factors(nu, nm, n_f, 10 + q) for q, (nu, nm, *_rest) in enumerate(batch)]
    with ALSBatch(batch, n_f, 0.05, precision="mixed") as m:
        m.set_x(m.join_x(xs))
        out = m.run(200, rel_tol=1e-4, check_every=10)
        infos = m.infos()
    assert all(i["gnorm"] <= 1e-4 * i["gnorm0"] for i in infos), [i["gnorm"] / i["gnorm0"] for i in infos]
    assert out["iters"] <= 200


def test_batched_matches_standalone_mixed(batch):
    """Each problem's rows are solved by the same row-wise kernels in a batch
    and alone; only the order of the per-problem reductions differs."""
    from paper_1508_03110_gb300 import ALS, ALSBatch
    n_f = 48
    xs = [synth.init_factors(nu, nm, n_f, 20 + q) for q, (nu, nm, *_rest) in enumerate(batch)]
    with ALSBatch(batch, n_f, 0.05, precision="mixed") as m:
        m.set_x(m.join_x(xs))
        for _ in range(5):
            m.step(info=False)
        got = m.split_x(m.get_x())
    for q, ((nu, nm, r, c, v), x0) in enumerate(zip(batch, xs)):
        with ALS(nu, nm, r, c, v, n_f, 0.05, precision="mixed") as s:
            s.set_x(x0)
            for _ in range(5):
                s.step(info=False)
            assert _rel(got[q], s.get_x()) < 1e-4, q


def test_batched_rejects_bad_local_ids(batch):
    from paper_1508_03110_gb300 import ALSBatch, ALSError
    bad = list(batch)
    nu, nm, r, c, v = bad[2]
    r = r.copy(); r[0] = nu          # out of range for problem 2
    bad[2] = (nu, nm, r, c, v)
    with pytest.raises(ALSError, match="EINVAL"):
        ALSBatch(bad, 8, 0.05)
