"""Light-row solve of the mixed tensor-core sweep: rows of at most
min(dual_max, n_f) ratings are solved through F F^T + lambda n_i I (Woodbury
identity) instead of the n_f x n_f matrix of Eq. (3) / (4).  Same rows as the
FP64 oracle's solve, same ALS-NCG trajectory as the FP64 run (needs a GB300);
with a CTA per row, and (dual_warp) with a warp per row of at most 32
ratings."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# user degrees around every boundary of the light-row solve (64 ratings, n_f,
# the 4-row tiles of G, the 16-row blocks of its solves)
DEGREES = [0, 1, 2, 3, 4, 5, 15, 16, 17, 31, 32, 33, 35, 36, 37, 47, 48, 49, 50, 51,
           63, 64, 65, 99, 100, 101, 128, 129, 300]


def _dual_problem(copies=6, n_m=400, seed=0):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    degs = [d for d in DEGREES for _ in range(copies)]
    rng.shuffle(degs)
    for i, d in enumerate(degs):
        rows.append(np.full(d, i))
        cols.append(rng.choice(n_m, size=d, replace=False))
    rows = np.concatenate(rows).astype(np.int32)
    cols = np.concatenate(cols).astype(np.int32)
    vals = (np.round(2 * np.clip(rng.normal(3.5, 1, rows.size), 0.5, 5)) / 2).astype(np.float32)
    return len(degs), n_m, rows, cols, vals


def _model(n_u, n_m, rows, cols, vals, n_f, **kw):
    from paper_1508_03110_gb300 import ALS
    return ALS(n_u, n_m, rows, cols, vals, n_f, 0.05, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dual_warp", [0, 1])
@pytest.mark.parametrize("n_f", [36, 50, 98, 100, 128])
@pytest.mark.parametrize("dual_max", [0, 16, 32, 64])
def test_dual_sweep_matches_oracle(n_f, dual_max, dual_warp):
    """One sweep with enough refinement steps: every user row (solved from the
    same item rows as the oracle's) within 1e-5 of the oracle's row, the whole
    x within 1e-5."""
    n_u, n_m, rows, cols, vals = _dual_problem()
    P = oracle.build_problem(n_u, n_m, n_f, 0.05, rows, cols, vals)
    x0 = synth.init_factors(n_u, n_m, n_f, 5)
    ref = oracle.sweep(P, x0)
    with _model(n_u, n_m, rows, cols, vals, n_f, precision="mixed", gram_path="tc", refine_steps=4) as m:
        m.set_launch(dual_max=dual_max, dual_warp=dual_warp)
        assert m.get_launch()["dual_max"] == dual_max and m.get_launch()["dual_warp"] == dual_warp
        m.set_x(x0)
        m.sweep(1)
        x = m.get_x()
    U, Ur = x[:n_u * n_f].reshape(n_u, n_f), ref[:n_u * n_f].reshape(n_u, n_f)
    err = np.linalg.norm(U - Ur, axis=1)
    scale = np.maximum(np.linalg.norm(Ur, axis=1), 1e-30)
    deg = np.bincount(rows, minlength=n_u)
    assert np.all(U[deg == 0] == 0.0)
    assert np.all(err[deg > 0] <= 1e-5 * scale[deg > 0]), (deg[np.argmax(err / scale)], np.max(err / scale))
    assert _rel(x, ref) < 1e-5


@pytest.mark.parametrize("dual_warp", [0, 1])
def test_dual_single_correction_is_accurate(dual_warp):
    """From a random start one correction through G leaves an error of order
    kappa(A) times FP32 rounding on the light rows, far below the tensor-core
    Gram's (BF16 split) first correction."""
    n_u, n_m, rows, cols, vals = _dual_problem(seed=3)
    n_f = 100
    P = oracle.build_problem(n_u, n_m, n_f, 0.05, rows, cols, vals)
    x0 = synth.init_factors(n_u, n_m, n_f, 8)
    ref = oracle.sweep(P, x0)
    deg = np.bincount(rows, minlength=n_u)
    light = (deg > 0) & (deg <= 64)
    with _model(n_u, n_m, rows, cols, vals, n_f, precision="mixed", gram_path="tc", refine_steps=1) as m:
        m.set_launch(dual_max=64, dual_warp=dual_warp)
        m.set_x(x0)
        m.sweep(1)
        x = m.get_x()
    U, Ur = x[:n_u * n_f].reshape(n_u, n_f), ref[:n_u * n_f].reshape(n_u, n_f)
    err = np.linalg.norm(U[light] - Ur[light], axis=1) / np.linalg.norm(Ur[light], axis=1)
    assert np.max(err) < 1e-4, np.max(err)


@pytest.mark.parametrize("dual_max,dual_warp", [(16, 0), (64, 0), (64, 1)])
def test_dual_alsncg_matches_fp64_run(dual_max, dual_warp):
    """ALS-NCG with the light-row solve: f within 1e-5 of the FP64 run at equal
    iteration count, no row left unsolved."""
    n_u, n_m, rows, cols, vals = _dual_problem(copies=10, seed=1)
    n_f = 100
    x0 = synth.init_factors(n_u, n_m, n_f, 4)
    fs = {}
    for prec in ("fp64", "mixed"):
        with _model(n_u, n_m, rows, cols, vals, n_f, precision=prec) as m:
            if prec == "mixed":
                m.set_launch(dual_max=dual_max, dual_warp=dual_warp)
            m.set_x(x0)
            fs[prec] = np.array([m.step()["f"] for _ in range(25)])
            out = m.run(1)
            assert out["notspd"] == 0
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"])), \
        np.max(np.abs(fs["mixed"] - fs["fp64"]) / np.abs(fs["fp64"]))


def test_dual_tiny_workload_trajectory():
    """The shared small workload (2,000 x 1,000, 1e5 ratings; 87% of users and
    41% of items have at most 64 ratings) at n_f = 100, with and without the
    light-row solve: both within 1e-5 of the FP64 run's f."""
    r = synth.make_config("tiny")
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 9)
    fs = {}
    for key, prec, d, w in (("fp64", "fp64", 0, 0), ("dual", "mixed", 64, 0), ("warp", "mixed", 64, 1),
                            ("tc", "mixed", 0, 0)):
        with _model(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, precision=prec) as m:
            if prec == "mixed":
                m.set_launch(dual_max=d, dual_warp=w)
            m.set_x(x0)
            fs[key] = np.array([m.step()["f"] for _ in range(20)])
    for key in ("dual", "warp", "tc"):
        assert np.all(np.abs(fs[key] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"])), key


def test_dual_bound_rejected_out_of_range():
    from paper_1508_03110_gb300 import ALSError
    n_u, n_m, rows, cols, vals = _dual_problem(copies=1)
    with _model(n_u, n_m, rows, cols, vals, 100, precision="mixed") as m:
        with pytest.raises(ALSError, match="EINVAL"):
            m.set_launch(dual_max=65)
        with pytest.raises(ALSError, match="EINVAL"):
            m.set_launch(dual_max=-1)


def test_dual_warp_foldin_matches_oracle():
    """Fold-in requests of 1..40 ratings against fixed item rows (a cold
    start, u0 = 0) with a warp per request of at most 32 ratings: every answer
    within 1e-5 of the oracle's exact solve."""
    n_u, n_m, rows, cols, vals = _dual_problem(copies=2, seed=5)
    n_f = 100
    x0 = synth.init_factors(n_u, n_m, n_f, 6).astype(np.float32).astype(np.float64)
    ptr, items, rv = synth.foldin_requests(48, n_m, 1, 40, seed=12)
    ref = oracle.foldin(n_f, 0.05, x0[n_u * n_f:], ptr, items, rv.astype(np.float64))
    with _model(n_u, n_m, rows, cols, vals, n_f, precision="mixed", gram_path="tc", refine_steps=4) as m:
        m.set_launch(dual_max=64, dual_warp=1)
        m.set_x(x0)
        u = m.foldin(ptr, items, rv).reshape(-1, n_f)
    ref = ref.reshape(-1, n_f)
    err = np.linalg.norm(u - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    assert np.max(err) < 1e-5, np.max(err)


def test_dual_warp_rejected_out_of_range():
    from paper_1508_03110_gb300 import ALSError
    n_u, n_m, rows, cols, vals = _dual_problem(copies=1)
    with _model(n_u, n_m, rows, cols, vals, 100, precision="mixed") as m:
        with pytest.raises(ALSError, match="EINVAL"):
            m.set_launch(dual_warp=2)
