"""The seeded input generators keep the recipe they state (no GPU): the same
seed gives the same data, every (user, item) pair is distinct, degrees hit
their targets, values are half stars in [0.5, 5], x_0 is N(0, 1/n_f)."""
import numpy as np

import synth
from synth.ratings import rank_degrees, sample_distinct


def test_same_seed_same_ratings():
    a, b = synth.make_config("tiny"), synth.make_config("tiny")
    for f in ("rows", "cols", "vals"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = synth.make_config("tiny", seed=2)
    assert not np.array_equal(a.cols, c.cols)


def test_tiny_recipe():
    r = synth.make_config("tiny")
    assert (r.n_u, r.n_m, r.nnz, r.n_f, r.lam) == (2000, 1000, 100_000, 10, 0.05)
    key = r.rows.astype(np.int64) * r.n_m + r.cols
    assert np.unique(key).size == r.nnz                     # distinct (user, item) pairs
    assert r.rows.min() >= 0 and r.rows.max() < r.n_u and r.cols.min() >= 0 and r.cols.max() < r.n_m
    du = np.bincount(r.rows, minlength=r.n_u)
    assert du.min() >= 5 and du.max() <= 1000                # Zipf degrees floored at 5
    assert np.all(np.diff(r.rows) >= 0)                      # grouped by user
    v = r.vals.astype(np.float64)
    assert np.all(v >= 0.5) and np.all(v <= 5.0) and np.all(2 * v == np.round(2 * v))
    assert abs(v.mean() - 3.5) < 0.1


def test_sample_distinct_hits_every_degree():
    """Successive weighted sampling without replacement: each row gets exactly
    its degree in distinct items, even when the degree is close to n_m and the
    weights are very skewed (the exponential-key completion)."""
    rng = np.random.default_rng(3)
    n_m = 50
    deg = np.array([0, 1, 5, 25, 49, 50, 50, 3])
    w = np.arange(1, n_m + 1, dtype=np.float64) ** -2.0
    rows, cols = sample_distinct(deg, w, rng)
    assert np.array_equal(np.bincount(rows, minlength=deg.size), deg)
    key = rows.astype(np.int64) * n_m + cols
    assert np.unique(key).size == rows.size
    assert cols.min() >= 0 and cols.max() < n_m


def test_rank_degrees_sum_and_bounds():
    rng = np.random.default_rng(5)
    d = rank_degrees(1000, 50_000, 3, 400, rng, 1.1)
    assert d.sum() == 50_000 and d.min() >= 3 and d.max() <= 400


def test_foldin_requests_recipe():
    ptr, items, vals = synth.foldin_requests(300, 2000, 1, 500, seed=7)
    deg = np.diff(ptr)
    assert ptr[0] == 0 and ptr[-1] == items.size == vals.size
    assert deg.min() >= 1 and deg.max() <= 500
    for q in range(0, 300, 37):                              # distinct items within a request
        it = items[ptr[q]:ptr[q + 1]]
        assert np.unique(it).size == it.size
    assert np.all(2 * vals == np.round(2 * vals)) and vals.min() >= 0.5 and vals.max() <= 5.0


def test_init_factors_distribution():
    x = synth.init_factors(3000, 2000, 25, seed=11)
    assert x.shape == ((3000 + 2000) * 25,)
    assert abs(x.mean()) < 3e-3 and abs(x.var() * 25 - 1.0) < 0.02
    assert np.array_equal(x, synth.init_factors(3000, 2000, 25, seed=11))


def test_batch_problems_are_independent_and_local():
    probs = synth.make_batch(5, 2_000, 20_000, 0.02, 0.05, seed=8)
    assert len(probs) == 5
    for n_u, n_m, rows, cols, vals in probs:
        assert rows.max() < n_u and cols.max() < n_m and rows.min() >= 0 and cols.min() >= 0
        assert np.unique(rows.astype(np.int64) * n_m + cols).size == rows.size
        assert 2_000 // 2 <= rows.size <= 20_000
