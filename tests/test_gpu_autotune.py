"""Autotuner (als_autotune): it changes launch shapes only, so results stay
within the parity tolerances and no state is touched (needs a GB300)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

HEAVY = {256, 512, 1024, 2048, 4096, 8192, 1 << 30}
GRID = {4, 8, 16, 32, 64}
BINS = {0, 256, 1024, 4096, 16384}


@pytest.fixture(scope="module")
def tiny():
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    return r, P


def _model(r, n_f, **kw):
    from paper_1508_03110_gb300 import ALS
    return ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_autotune_keeps_fp64_parity_and_state(tiny):
    r, P = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    ref = oracle.alsncg(P, x0, 12)
    with _model(r, r.n_f) as m:
        m.set_x(x0)
        for k in range(4):
            m.step(info=False)
        before = m.get_x()
        rep = m.autotune(reps=2)
        assert np.array_equal(m.get_x(), before)          # no factor state touched
        assert rep["heavy_min"] in HEAVY and rep["grid_mult"] in GRID and rep["sweep_bin_min"] in BINS
        assert rep["candidates"] >= 11 and rep["pass_ms_tuned"] <= rep["pass_ms_default"]
        assert rep["sweep_ms_tuned"] <= rep["sweep_ms_default"]
        for k in range(4, 12):                            # graphs recaptured with the new shapes
            m.step(info=False)
            assert _rel(m.get_x(), ref[k].x) < 1e-9, k


@pytest.mark.parametrize("n_f", [24, 48])
def test_autotune_mixed_matches_fp64(tiny, n_f):
    r, _ = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7)
    fs = {}
    for prec in ("fp64", "mixed"):
        with _model(r, n_f, precision=prec) as m:
            m.set_x(x0)
            rep = m.autotune(reps=1)
            assert rep["gram_path"] in (1, 2)
            fs[prec] = np.array([m.step()["f"] for _ in range(20)])
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"]))


def test_autotune_batched_context(tiny):
    """Batched contexts share the row-wise kernels: tuning keeps the
    per-problem trajectories."""
    from paper_1508_03110_gb300 import ALSBatch
    probs = synth.make_batch(4, 2_000, 20_000, 0.02, 0.05, seed=8)
    xs = [synth.init_factors(nu, nm, 8, 20 + q) for q, (nu, nm, *_rest) in enumerate(probs)]
    refs = [oracle.alsncg(oracle.build_problem(nu, nm, 8, 0.05, rr, cc, vv), x0, 5)
            for (nu, nm, rr, cc, vv), x0 in zip(probs, xs)]
    with ALSBatch(probs, 8, 0.05) as m:
        m.set_x(m.join_x(xs))
        m.autotune(reps=1)
        for _ in range(5):
            m.step(info=False)
        got = m.split_x(m.get_x())
    for q in range(len(probs)):
        assert _rel(got[q], refs[q][-1].x) < 1e-9
