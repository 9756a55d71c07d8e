"""The optimizer variants of Algorithm 2 on the GPU against the FP64 oracle
(needs a GB300): the More-Thuente line search on Q (the paper's serial
experiments, §IV: alpha0 = 1, sufficient decrease 1e-4, curvature 1e-2, at
most 20 evaluations), the Fletcher-Reeves, Hestenes-Stiefel and PR+ forms of
beta-bar, and plain NCG (no ALS preconditioner: gbar = g).

Per iteration (lockstep): from the oracle's state after iteration k, one GPU
iteration must take the same branch and the same number of line-search
evaluations, and give alpha, beta-bar, x_{k+1}, f and p_{k+1} within 1e-10
(per row for the vectors).  The search itself is the same sequence of
correctly rounded FP64 operations on both sides."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10

MT = dict(ls_mode="more-thuente")
MT_ORACLE = dict(mode="mt", alpha0=1.0, cc=1e-4, max_shrinks=20, c2=1e-2)

VARIANTS = {
    "more-thuente": (MT, MT_ORACLE),
    "plain-ncg-more-thuente": (dict(MT, precond="none"), dict(MT_ORACLE, precond="none")),
    "beta-fr": (dict(beta="fr"), dict(beta="fr")),
    "beta-hs": (dict(beta="hs"), dict(beta="hs")),
    "beta-prplus": (dict(beta="prplus"), dict(beta="prplus")),
    "more-thuente-beta-hs": (dict(MT, beta="hs"), dict(MT_ORACLE, beta="hs")),
}


def _row_rel(a, b, n_f, scale=None):
    a = np.asarray(a).reshape(-1, n_f)
    b = np.asarray(b).reshape(-1, n_f)
    s = b if scale is None else np.asarray(scale).reshape(-1, n_f)
    num = np.linalg.norm(a - b, axis=1)
    q = np.where(num == 0.0, 0.0, num / np.maximum(np.linalg.norm(s, axis=1), 1e-300))
    return float(q.max())


@pytest.fixture(scope="module")
def tiny():
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    return r, P, x0


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_lockstep_fp64(tiny, name):
    from paper_1508_03110_gb300 import ALS
    r, P, x0 = tiny
    gpu_kw, orc_kw = VARIANTS[name]
    K = 15
    ref = oracle.alsncg(P, x0, K, **orc_kw)
    g0 = np.linalg.norm(oracle.grad(P, x0))
    nfall = np.cumsum([q.fallback for q in ref])
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, r.n_f, r.lam, **gpu_kw) as m:
        m.set_x(x0)
        for k in range(K):
            if k > 0:
                st = ref[k - 1].state
                m.set_state(ref[k - 1].x, st["p"], ref[k - 1].g, st["gbar"], st["xbar"], st["s"], g0 ** 2, k,
                            int(nfall[k - 1]))
            info = m.step()
            assert info["fallback"] == ref[k].fallback, k
            assert info["shrinks"] == ref[k].shrinks or ref[k].margin < 1e-9, (k, info["shrinks"], ref[k].shrinks)
            assert info["alpha"] == pytest.approx(ref[k].alpha, rel=TOL, abs=0.0), k
            assert info["beta"] == pytest.approx(ref[k].beta, rel=1e-8, abs=1e-14), k
            x = m.get_x()
            assert _row_rel(x, ref[k].x, r.n_f) < TOL, (k, _row_rel(x, ref[k].x, r.n_f))
            assert info["f"] == pytest.approx(ref[k].f, rel=TOL), k
            gs = m.get_state()
            pr = ref[k].state["p"]
            sc = np.abs(pr).reshape(-1, r.n_f) + np.abs(ref[k].x).reshape(-1, r.n_f)
            assert _row_rel(gs["p"], pr, r.n_f, scale=sc) < TOL, k
            if gpu_kw.get("precond") == "none":
                # plain NCG: gbar is the gradient, xbar the iterate
                assert _row_rel(gs["gbar"], gs["g"], r.n_f) == 0.0
                assert np.array_equal(gs["xbar"], gs["x"])


@pytest.mark.parametrize("name", ["more-thuente", "beta-hs"])
def test_variant_free_running_fp64(tiny, name):
    from paper_1508_03110_gb300 import ALS
    r, P, x0 = tiny
    gpu_kw, orc_kw = VARIANTS[name]
    ref = oracle.alsncg(P, x0, 25, **orc_kw)
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, r.n_f, r.lam, **gpu_kw) as m:
        m.set_x(x0)
        for k in range(25):
            info = m.step()
            assert info["fallback"] == ref[k].fallback, k
        x = m.get_x()
    assert np.linalg.norm(x - ref[-1].x) <= 1e-9 * np.linalg.norm(ref[-1].x)
    assert info["f"] == pytest.approx(ref[-1].f, rel=1e-10)


@pytest.mark.parametrize("n_f", [10, 100])
def test_more_thuente_mixed_matches_fp64_run(tiny, n_f):
    """The mixed form with the More-Thuente search: f within 1e-5 of the FP64
    run at equal iteration count."""
    from paper_1508_03110_gb300 import ALS
    r, _, _ = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7)
    fs = {}
    for prec in ("fp64", "mixed"):
        with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision=prec, **MT) as m:
            m.set_x(x0)
            fs[prec] = np.array([m.step()["f"] for _ in range(20)])
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"]))


def test_batched_more_thuente_per_problem():
    """The More-Thuente search runs per problem in a batched context: each
    problem follows the oracle's trajectory run on it alone."""
    from paper_1508_03110_gb300 import ALSBatch
    batch = synth.make_batch(5, 1_000, 20_000, 0.01, 0.05, seed=8)
    n_f, lam = 10, 0.1
    xs = [synth.init_factors(nu, nm, n_f, 20 + q) for q, (nu, nm, *_rest) in enumerate(batch)]
    refs = [oracle.alsncg(oracle.build_problem(nu, nm, n_f, lam, rr, c, v), x0, 8, **MT_ORACLE)
            for (nu, nm, rr, c, v), x0 in zip(batch, xs)]
    with ALSBatch(batch, n_f, lam, precision="fp64", **MT) as m:
        m.set_x(m.join_x(xs))
        for k in range(8):
            m.step(info=False)
        got = m.split_x(m.get_x())
        infos = m.infos()
    for q in range(len(batch)):
        assert np.linalg.norm(got[q] - refs[q][-1].x) <= 1e-9 * np.linalg.norm(refs[q][-1].x), q
        assert infos[q]["f"] == pytest.approx(refs[q][-1].f, rel=1e-9)
