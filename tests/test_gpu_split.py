"""Heavy rows split across CTAs (segment partials added in FP64): the split
path must give the oracle's rows (FP64 form, 1e-10) and keep the mixed form
within its tolerances.  Splitting is forced on the small problem by a low
split threshold and short, unevenly dividing segments (needs a GB300)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SPLIT = dict(split_min=256, seg_len=100)


@pytest.fixture(scope="module")
def tiny():
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    deg_m = np.bincount(r.cols, minlength=r.n_m)
    deg_u = np.bincount(r.rows, minlength=r.n_u)
    assert deg_m.max() >= 3 * SPLIT["split_min"] and (deg_u >= SPLIT["split_min"]).sum() > 0
    return r, P


def _model(r, n_f, **kw):
    from paper_1508_03110_gb300 import ALS
    return ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n_f", [10, 40])
def test_split_sweep_fp64_matches_oracle(tiny, n_f):
    r, _ = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 5)
    with _model(r, n_f) as m:
        m.set_launch(**SPLIT)
        assert m.get_launch()["split_min"] == SPLIT["split_min"]
        m.set_x(x0)
        m.sweep(2)
        x = m.get_x()
    ref = oracle.sweep(P, oracle.sweep(P, x0))
    assert _rel(x, ref) < 1e-10


def test_split_alsncg_fp64_trajectory(tiny):
    r, P = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    ref = oracle.alsncg(P, x0, 12)
    with _model(r, r.n_f) as m:
        m.set_launch(**SPLIT)
        m.set_x(x0)
        for k in range(12):
            info = m.step()
            assert _rel(m.get_x(), ref[k].x) < 1e-9, k
            assert info["f"] == pytest.approx(ref[k].f, rel=1e-10)


@pytest.mark.parametrize("n_f,gram", [(10, "fma"), (48, "tc"), (100, "tc")])
def test_split_mixed_matches_fp64(tiny, n_f, gram):
    r, _ = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7)
    fs = {}
    for prec in ("fp64", "mixed"):
        kw = dict(precision=prec)
        if prec == "mixed":
            kw["gram_path"] = gram
        with _model(r, n_f, **kw) as m:
            m.set_launch(**SPLIT)
            m.set_x(x0)
            fs[prec] = np.array([m.step()["f"] for _ in range(20)])
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"]))


def test_split_mixed_sweep_close_to_exact(tiny):
    """With the refinement allowed enough corrections the split rows reach
    the exact step (the stopping rule ends it at FP32 resolution)."""
    r, _ = tiny
    n_f = 100
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3)
    with _model(r, n_f, precision="mixed", gram_path="tc", refine_steps=4) as m:
        m.set_launch(**SPLIT)
        m.set_x(x0)
        m.sweep(1)
        x = m.get_x()
    assert _rel(x, oracle.sweep(P, x0)) < 1e-5


def test_split_batched_per_problem(tiny):
    from paper_1508_03110_gb300 import ALSBatch
    probs = synth.make_batch(3, 20_000, 60_000, 0.02, 0.05, seed=9)
    xs = [synth.init_factors(nu, nm, 8, 30 + q) for q, (nu, nm, *_rest) in enumerate(probs)]
    refs = [oracle.alsncg(oracle.build_problem(nu, nm, 8, 0.05, rr, cc, vv), x0, 4)
            for (nu, nm, rr, cc, vv), x0 in zip(probs, xs)]
    with ALSBatch(probs, 8, 0.05) as m:
        m.set_launch(split_min=200, seg_len=64)
        m.set_x(m.join_x(xs))
        for _ in range(4):
            m.step(info=False)
        got = m.split_x(m.get_x())
    for q in range(len(probs)):
        assert _rel(got[q], refs[q][-1].x) < 1e-9


def test_set_launch_rejects_bad_values(tiny):
    from paper_1508_03110_gb300 import ALSError
    r, _ = tiny
    with _model(r, r.n_f) as m:
        for bad in (dict(seg_len=8), dict(heavy_min=0), dict(grid_mult=0), dict(split_min=-1), dict(gram_path="tc")):
            with pytest.raises(ALSError, match="EINVAL"):
                m.set_launch(**bad)
