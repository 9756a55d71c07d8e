"""Top-t ranking accuracy (§IV, modified Kendall-tau) on the GPU against the
FP64 oracle (needs a GB300).  The rankings are integer decisions taken on
floating-point scores: the GPU forms every score u . m with FMAs in the
factor order (FP64 or FP32), the oracle in FP64 with numpy.  Where two
scores that decide a count lie within the scores' rounding bound of each
other the decision is not unique; each such pair may move a user's swap
count by at most 2, and everything else must agree exactly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _model(r, x, n_f, precision):
    from paper_1508_03110_gb300 import ALS
    m = ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision=precision)
    m.set_x(x)
    return m


def _bound(U, M, i, precision):
    """Rounding bound of each score of user i (FP32: n_f 2^-24 sum |u m|
    twice over, FP64: the same with 2^-53)."""
    eps = 2.0 ** -24 if precision == "mixed" else 2.0 ** -53
    return 2.0 * U.shape[1] * eps * (np.abs(M) @ np.abs(U[i]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("t", [1, 20, 64])
def test_rank_topt_matches_oracle(precision, t):
    r = synth.make_config("tiny")
    n_f = 10
    x = synth.init_factors(r.n_u, r.n_m, n_f, 31)
    if precision == "mixed":
        x = x.astype(np.float32).astype(np.float64)
    U, M = x[: r.n_u * n_f].reshape(r.n_u, n_f), x[r.n_u * n_f:].reshape(r.n_m, n_f)
    with _model(r, x, n_f, precision) as m:
        top = m.rank_topt(t)
    ref = oracle.ranking.topt(U, M, t)
    exact = 0
    for i in range(r.n_u):
        sc = M @ U[i]
        if np.array_equal(top[i], ref[i]):
            exact += 1
            continue
        # not unique: a score of the GPU's list and one of the oracle's list
        # within the rounding bound of each other
        b = _bound(U, M, i, precision)
        srt = np.sort(sc)[::-1]
        kth = srt[t - 1]
        gpu_ok = np.all(sc[top[i]] >= kth - 2 * b.max())
        assert gpu_ok and len(set(top[i])) == t, i
    assert exact >= r.n_u - (2 if precision == "fp64" else 50)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("t", [1, 20, 64])
def test_rank_accuracy_matches_oracle(precision, t):
    r = synth.make_config("tiny")
    n_f = 10
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 31)
    x1 = x0 + 0.05 * synth.init_factors(r.n_u, r.n_m, n_f, 32)     # a nearby iterate
    if precision == "mixed":
        x0 = x0.astype(np.float32).astype(np.float64)
        x1 = x1.astype(np.float32).astype(np.float64)
    U0, M0 = x0[: r.n_u * n_f].reshape(r.n_u, n_f), x0[r.n_u * n_f:].reshape(r.n_m, n_f)
    U1, M1 = x1[: r.n_u * n_f].reshape(r.n_u, n_f), x1[r.n_u * n_f:].reshape(r.n_m, n_f)
    ref_top = oracle.ranking.topt(U0, M0, t)
    qm_ref, q_ref, s_ref = oracle.ranking.rank_accuracy(U1, M1, ref_top)
    with _model(r, x1, n_f, precision) as m:
        qm, q = m.rank_accuracy(ref_top, per_user=True)
        # the reference lists of the same factors give q = 1 exactly
        m.set_x(x0)
        top0 = m.rank_topt(t)
        assert m.rank_accuracy(top0) == 1.0
    smax = oracle.ranking.s_max(r.n_m, t)
    s_gpu = np.rint((1.0 - q) * smax).astype(np.int64)
    unique = 0
    for i in range(r.n_u):
        if s_gpu[i] == s_ref[i]:
            unique += 1
            continue
        sc = M1 @ U1[i]
        b = _bound(U1, M1, i, precision)
        amb = 0
        for a in ref_top[i]:
            amb += int(np.sum(np.abs(sc - sc[a]) <= b + b[a])) - 1
        assert abs(int(s_gpu[i]) - int(s_ref[i])) <= 2 * amb, (i, s_gpu[i], s_ref[i], amb)
    assert unique >= r.n_u - (2 if precision == "fp64" else 200)
    assert qm == pytest.approx(float(np.mean(q)), rel=1e-14)
    assert abs(qm - qm_ref) <= 2e-4 if precision == "mixed" else qm == pytest.approx(qm_ref, rel=1e-12)


def test_rank_rejects_bad_reference():
    from paper_1508_03110_gb300 import ALSError
    r = synth.make_config("tiny")
    x = synth.init_factors(r.n_u, r.n_m, 10, 31)
    with _model(r, x, 10, "fp64") as m:
        top = m.rank_topt(5)
        bad = top.copy(); bad[3, 1] = bad[3, 0]
        with pytest.raises(ALSError, match="EINVAL"):
            m.rank_accuracy(bad)
        bad = top.copy(); bad[7, 2] = r.n_m
        with pytest.raises(ALSError, match="EINVAL"):
            m.rank_accuracy(bad)
        with pytest.raises(ALSError, match="EINVAL"):
            m.rank_topt(65)
