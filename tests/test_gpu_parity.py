"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances: the FP64 form must match the oracle to 1e-10 relative in f and in
the factors, per iteration; the mixed form must match the FP64 run's f to
1e-5 relative at equal iteration count and its final train RMSE to 1e-4.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _als():
    from paper_1508_03110_gb300 import ALS
    return ALS


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _row_rel(a, b, n_f, scale=None):
    """max over factor rows (users and items) of |a_row - b_row| / |s_row|,
    s = b unless given: a bad row cannot hide under many good ones.  A row
    that is exactly zero in both (an empty row) counts as 0."""
    a = np.asarray(a, np.float64).reshape(-1, n_f)
    b = np.asarray(b, np.float64).reshape(-1, n_f)
    s = b if scale is None else np.asarray(scale, np.float64).reshape(-1, n_f)
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(s, axis=1)
    q = np.where(num == 0.0, 0.0, num / np.maximum(den, 1e-300))
    return float(q.max())


@pytest.fixture(scope="module")
def tiny():
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    return r, P, x0


def _model(r, n_f=None, **kw):
    return _als()(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f or r.n_f, r.lam, **kw)


# -- builder (bit-exact) -----------------------------------------------------------

def test_builder_matches_host_sort(tiny):
    r, P, _ = tiny
    with _model(r) as m:
        R = m.ratings()
    assert np.array_equal(R["uptr"], P.uptr)
    assert np.array_equal(R["uidx"], P.uidx)
    assert np.array_equal(R["uval"].astype(np.float64), P.uval)
    assert np.array_equal(R["mptr"], P.mptr)
    assert np.array_equal(R["midx"], P.midx)
    assert np.array_equal(R["mval"].astype(np.float64), P.mval)
    du = np.diff(P.uptr); dm = np.diff(P.mptr)
    assert np.array_equal(R["uorder"], np.lexsort((np.arange(r.n_u), -du)))
    assert np.array_equal(R["morder"], np.lexsort((np.arange(r.n_m), -dm)))


def test_builder_from_csr_input(tiny):
    r, P, x0 = tiny
    o = np.lexsort((r.cols, r.rows))
    rowptr = np.zeros(r.n_u + 1, np.int64)
    np.cumsum(np.bincount(r.rows, minlength=r.n_u), out=rowptr[1:])
    with _als()(r.n_u, r.n_m, None, r.cols[o], r.vals[o], r.n_f, r.lam, rowptr=rowptr) as m:
        R = m.ratings()
    assert np.array_equal(R["uidx"], P.uidx) and np.array_equal(R["midx"], P.midx)


def test_builder_rejects_bad_input(tiny):
    from paper_1508_03110_gb300 import ALSError
    r, _, _ = tiny
    rows = r.rows.copy(); rows[5] = r.n_u
    with pytest.raises(ALSError, match="EINVAL"):
        _als()(r.n_u, r.n_m, rows, r.cols, r.vals, r.n_f, r.lam)
    vals = r.vals.copy(); vals[7] = np.nan
    with pytest.raises(ALSError, match="EINVAL"):
        _als()(r.n_u, r.n_m, r.rows, r.cols, vals, r.n_f, r.lam)
    rows = np.concatenate([r.rows, r.rows[:1]]); cols = np.concatenate([r.cols, r.cols[:1]])
    vals = np.concatenate([r.vals, r.vals[:1]])
    with pytest.raises(ALSError, match="duplicate"):
        _als()(r.n_u, r.n_m, rows, cols, vals, r.n_f, r.lam)
    with pytest.raises(ALSError, match="EBUDGET"):
        _als()(r.n_u, r.n_m, r.rows, r.cols, r.vals, r.n_f, r.lam, hbm_budget_bytes=1 << 16)


# -- single operators (FP64) --------------------------------------------------------------

def test_loss_grad_fp64(tiny):
    r, P, x0 = tiny
    with _model(r) as m:
        m.set_x(x0)
        assert m.loss() == pytest.approx(oracle.loss(P, x0), rel=1e-12)
        g, gn = m.grad()
        gref = oracle.grad(P, x0)
        assert _rel(g, gref) < 1e-12
        assert _row_rel(g, gref, r.n_f, scale=np.abs(gref) + np.abs(x0)) < 1e-11
        assert gn == pytest.approx(np.linalg.norm(gref), rel=1e-12)


def test_linesearch_coeffs_fp64(tiny):
    r, P, x0 = tiny
    p = np.random.default_rng(3).normal(size=x0.shape[0]) * 0.1
    with _model(r) as m:
        m.set_x(x0)
        c = m.linesearch_coeffs(p)
    cref = oracle.ls_coeffs(P, x0, p)
    assert np.allclose(c, cref, rtol=1e-11, atol=1e-11 * abs(cref[0]))


def test_sweep_fp64(tiny):
    r, P, x0 = tiny
    with _model(r) as m:
        m.set_x(x0)
        m.sweep(1)
        x1 = m.get_x()
    assert _row_rel(x1, oracle.sweep(P, x0), r.n_f) < TOL64


def test_als_trajectory_fp64(tiny):
    """Algorithm 1, 50 sweeps: f and x per sweep within 1e-10 of the oracle."""
    r, P, x0 = tiny
    ref = oracle.als(P, x0, 50, with_grad=False)
    with _model(r) as m:
        m.set_x(x0)
        for k in range(50):
            m.sweep(1)
            if k % 5 == 4 or k < 3:
                x = m.get_x()
                assert _row_rel(x, ref[k].x, r.n_f) < TOL64, k
                assert m.loss() == pytest.approx(ref[k].f, rel=TOL64)


def test_alsncg_lockstep_fp64(tiny):
    """Algorithm 2 per iteration: from the oracle's state after iteration k
    (x_k, p_k, g_k, gbar_k, xbar_k, s_k), one GPU iteration gives x_{k+1} and
    f(x_{k+1}) within 1e-10 of the oracle's, for k = 0 .. 49."""
    r, P, x0 = tiny
    ref = oracle.alsncg(P, x0, 50)
    g0 = np.linalg.norm(oracle.grad(P, x0))
    with _model(r) as m:
        m.set_x(x0)
        info = m.step()                     # k = 0 -> 1 from the GPU's own start
        assert _row_rel(m.get_x(), ref[0].x, r.n_f) < TOL64
        for k in range(1, 50):
            st = ref[k - 1].state
            m.set_state(ref[k - 1].x, st["p"], ref[k - 1].g, st["gbar"], st["xbar"], st["s"], g0 ** 2, k)
            info = m.step()
            assert info["shrinks"] == ref[k].shrinks or ref[k].margin < 1e-9, k
            x = m.get_x()
            assert _row_rel(x, ref[k].x, r.n_f) < TOL64, (k, _row_rel(x, ref[k].x, r.n_f))
            assert info["f"] == pytest.approx(ref[k].f, rel=TOL64), k
            gs = m.get_state()
            # p = -gbar + beta p: gbar = x - P(x) is a difference of rows of the
            # size of x, so a row's error is bounded relative to |p_row| + |x_row|
            pr = ref[k].state["p"]
            sc = np.abs(pr).reshape(-1, r.n_f) + np.abs(ref[k].x).reshape(-1, r.n_f)
            assert _row_rel(gs["p"], pr, r.n_f, scale=sc) < TOL64, (k, _row_rel(gs["p"], pr, r.n_f, scale=sc))
            assert abs(info["gnorm"] - ref[k].gnorm) <= 1e-10 * g0, k


def test_alsncg_trajectory_fp64(tiny):
    """Algorithm 2 run freely for 50 iterations.  Rounding differences of a
    few ulps per iteration accumulate and the iteration amplifies them
    (measured after 48 iterations: 1.5e-10 over the whole x, 1.2e-9 on the
    worst row), so the free-running trajectory is held to 1e-9 over x and
    1e-8 per row; the per-iteration bar of 1e-10 per row is the lockstep test
    above.  |g_k| is a difference of terms of the size of |g_0|, so its error
    is bounded relative to |g_0|."""
    r, P, x0 = tiny
    ref = oracle.alsncg(P, x0, 50)
    g0 = np.linalg.norm(oracle.grad(P, x0))
    with _model(r) as m:
        m.set_x(x0)
        for k in range(50):
            info = m.step()
            x = m.get_x()
            assert info["shrinks"] == ref[k].shrinks or ref[k].margin < 1e-9, k
            assert _rel(x, ref[k].x) < 1e-9, (k, _rel(x, ref[k].x))
            assert _row_rel(x, ref[k].x, r.n_f) < 1e-8, (k, _row_rel(x, ref[k].x, r.n_f))
            assert info["f"] == pytest.approx(ref[k].f, rel=TOL64), k
            assert info["gnorm0"] == pytest.approx(g0, rel=1e-12)
            assert abs(info["gnorm"] - ref[k].gnorm) <= 1e-9 * g0, k


def test_pinned_host_buffers_and_out_arrays(tiny):
    """Inputs from pinned host tensors (ratings, x_0) and factors read into
    given arrays (pinned host, numpy, device) give the same bits as the
    numpy path; wrong out arrays are rejected."""
    import torch
    r, _, x0 = tiny
    nu_f = r.n_u * r.n_f
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    with _model(r, precision="mixed") as m:
        m.set_x(x0)
        m.run(3, 0.0, check_every=3)
        U, M = m.get_factors()
    with _als()(r.n_u, r.n_m, pin(r.rows), pin(r.cols), pin(r.vals), r.n_f, r.lam, precision="mixed") as m:
        m.set_factors(pin(x0[:nu_f].reshape(r.n_u, r.n_f)), pin(x0[nu_f:].reshape(r.n_m, r.n_f)))
        m.run(3, 0.0, check_every=3)
        Up = torch.empty((r.n_u, r.n_f), dtype=torch.float64, pin_memory=True)
        Mp = torch.empty((r.n_m, r.n_f), dtype=torch.float64, pin_memory=True)
        assert m.get_factors(out=(Up, Mp))[0] is Up
        assert np.array_equal(Up.numpy(), U) and np.array_equal(Mp.numpy(), M)
        Un, Mn = np.empty((r.n_u, r.n_f), np.float32), np.empty((r.n_m, r.n_f), np.float32)
        m.get_factors("float32", out=(Un, Mn))
        assert np.array_equal(Un, U.astype(np.float32)) and np.array_equal(Mn, M.astype(np.float32))
        Ud = torch.empty((r.n_u, r.n_f), dtype=torch.float64, device="cuda")
        Md = torch.empty((r.n_m, r.n_f), dtype=torch.float64, device="cuda")
        m.get_factors(out=(Ud, Md))
        assert np.array_equal(Ud.cpu().numpy(), U) and np.array_equal(Md.cpu().numpy(), M)
        with pytest.raises(ValueError):
            m.get_factors(out=(Un, Mn))                       # float32 arrays for float64
        with pytest.raises(ValueError):
            m.get_factors(out=(Up, Md))                       # host and device
        with pytest.raises(ValueError):
            m.get_factors(out=(Up[:, :2], Mp))                # wrong shape


def test_state_roundtrip_resumes_identically(tiny):
    """Checkpoint / resume: get_state after 5 iterations, 5 more iterations;
    set_state from the checkpoint, 5 more: bit-identical."""
    r, _, x0 = tiny
    with _model(r, precision="mixed") as m:
        m.set_x(x0)
        for _ in range(5):
            m.step(info=False)
        st = m.get_state()
        for _ in range(5):
            m.step(info=False)
        xa = m.get_x()
        m.set_state(st["x"], st["p"], st["g"], st["gbar"], st["xbar"], st["s"], st["gg0"], st["k"],
                    st["fallbacks"])
        for _ in range(5):
            m.step(info=False)
        assert np.array_equal(m.get_x(), xa)


def test_fallback_branch_lockstep_fp64(tiny):
    """The fallback / restart branch of Algorithm 2 (no step passes the
    Armijo test: x_{k+1} = xbar_k, beta = 0, p_{k+1} = -gbar_{k+1}).  With no
    shrink allowed, only alpha0 = 10 is tried, and on this problem most steps
    fall back while some pass.  Per iteration, from the oracle's state after
    iteration k, the GPU must take the same branch, give x_{k+1}, f and p_{k+1}
    within 1e-10 per row, and count the same fallbacks.  The free-running
    trajectory takes the same branches too."""
    r, P, x0 = tiny
    K = 20
    ref = oracle.alsncg(P, x0, K, max_shrinks=0)
    branches = [q.fallback for q in ref]
    assert any(branches) and not all(branches)
    assert min(q.margin for q in ref) > 1e-6          # no decision near a tie
    g0 = np.linalg.norm(oracle.grad(P, x0))
    nfall = np.cumsum(branches)
    with _model(r, ls_max_shrinks=0) as m:
        m.set_x(x0)
        for k in range(K):
            if k > 0:
                st = ref[k - 1].state
                m.set_state(ref[k - 1].x, st["p"], ref[k - 1].g, st["gbar"], st["xbar"], st["s"], g0 ** 2, k,
                            int(nfall[k - 1]))
            info = m.step()
            assert info["fallback"] == ref[k].fallback, k
            assert info["fallbacks"] == nfall[k], k
            x = m.get_x()
            assert _row_rel(x, ref[k].x, r.n_f) < TOL64, (k, _row_rel(x, ref[k].x, r.n_f))
            if ref[k].fallback:
                assert info["alpha"] == 0.0 and info["beta"] == 0.0
                xbar_prev = oracle.sweep(P, ref[k - 1].x if k else x0)     # x_{k+1} = P(x_k)
                assert _row_rel(x, xbar_prev, r.n_f) < TOL64, k
            else:
                assert info["alpha"] == pytest.approx(ref[k].alpha, rel=1e-15)
                assert info["beta"] == pytest.approx(ref[k].beta, rel=1e-8)
            assert info["f"] == pytest.approx(ref[k].f, rel=TOL64), k
            gs = m.get_state()
            pr = ref[k].state["p"]
            sc = np.abs(pr).reshape(-1, r.n_f) + np.abs(ref[k].x).reshape(-1, r.n_f)
            assert _row_rel(gs["p"], pr, r.n_f, scale=sc) < TOL64, k
            assert gs["s"] == pytest.approx(ref[k].state["s"], rel=1e-8), k
            assert gs["fallbacks"] == nfall[k]
        # free running from x0: the same branches, the same count
        m.set_x(x0)
        for k in range(K):
            info = m.step()
            assert info["fallback"] == ref[k].fallback, k
        assert info["fallbacks"] == nfall[-1]
        assert _row_rel(m.get_x(), ref[-1].x, r.n_f) < 1e-9


@pytest.mark.parametrize("n_f", [1, 3, 7, 20, 33, 64, 100])
def test_alsncg_various_nf_fp64(tiny, n_f):
    r, _, _ = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 5)
    ref = oracle.alsncg(P, x0, 3)
    with _model(r, n_f=n_f) as m:
        m.set_x(x0)
        for k in range(3):
            m.step()
        assert _row_rel(m.get_x(), ref[-1].x, n_f) < TOL64


def test_exact_line_search_variant(tiny):
    r, P, x0 = tiny
    ref = oracle.alsncg(P, x0, 5, mode="exact")
    with _model(r, ls_mode="exact") as m:
        m.set_x(x0)
        for k in range(5):
            info = m.step()
        assert _row_rel(m.get_x(), ref[-1].x, r.n_f) < 1e-8
        assert info["alpha"] == pytest.approx(ref[-1].alpha, rel=1e-8)


def test_graph_run_equals_steps(tiny):
    r, P, x0 = tiny
    with _model(r) as m:
        m.set_x(x0)
        for _ in range(7):
            m.step(info=False)
        xa = m.get_x()
        m.set_x(x0)
        out = m.run(7, 0.0, check_every=3)
        xb = m.get_x()
    assert out["iters"] == 7
    assert np.array_equal(xa, xb)


def test_determinism(tiny):
    r, _, x0 = tiny
    xs = []
    for _ in range(2):
        with _model(r, precision="mixed") as m:
            m.set_x(x0)
            m.run(5)
            xs.append(m.get_x())
    assert np.array_equal(xs[0], xs[1])


# -- edge cases ------------------------------------------------------------------

def _edge_problem():
    """Empty items, degree-1 rows, heavy rows (>= 2048 ratings) on both sides."""
    rng = np.random.default_rng(0)
    n_u, n_m = 300, 2600
    rows, cols = [], []
    for i in range(n_u):
        if i < 3:
            d = 2300 + 50 * i            # heavy users
        elif i < 10:
            d = 1
        else:
            d = int(rng.integers(2, 40))
        c = rng.choice(n_m - 5, size=d, replace=False)   # last 5 items: empty
        rows.append(np.full(d, i)); cols.append(c)
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    # one heavy item: rated by every user
    extra = np.setdiff1d(np.arange(n_u), rows[cols == 7])
    rows = np.concatenate([rows, extra]); cols = np.concatenate([cols, np.full(extra.size, 7)])
    vals = (np.round(2 * np.clip(rng.normal(3.5, 1, rows.size), 0.5, 5)) / 2).astype(np.float32)
    return n_u, n_m, rows.astype(np.int32), cols.astype(np.int32), vals


@pytest.mark.parametrize("n_f", [5, 40])
def test_edge_cases_fp64(n_f):
    n_u, n_m, rows, cols, vals = _edge_problem()
    P = oracle.build_problem(n_u, n_m, n_f, 0.05, rows, cols, vals)
    x0 = synth.init_factors(n_u, n_m, n_f, 2)
    p = np.random.default_rng(1).normal(size=x0.shape[0])
    with _als()(n_u, n_m, rows, cols, vals, n_f, 0.05) as m:
        m.set_x(x0)
        assert m.loss() == pytest.approx(oracle.loss(P, x0), rel=1e-12)
        g, _ = m.grad()
        gref = oracle.grad(P, x0)
        # a row's gradient is a sum of terms of size |x|^2 (its own
        # regulariser, its ratings): bounded relative to that scale
        assert _rel(g, gref) < 1e-12
        assert _row_rel(g, gref, n_f, scale=np.abs(gref) + np.abs(x0)) < 1e-11
        assert np.allclose(m.linesearch_coeffs(p), oracle.ls_coeffs(P, x0, p), rtol=1e-11)
        ref = oracle.alsncg(P, x0, 4)
        for k in range(4):
            m.step()
        x = m.get_x()
        assert _row_rel(x, ref[-1].x, n_f) < TOL64
        assert np.all(x.reshape(-1, n_f)[n_u + n_m - 5:] == 0.0)   # empty items held at 0


# -- fold-in ------------------------------------------------------------------

def test_foldin_fp64(tiny):
    r, P, x0 = tiny
    ptr, items, vals = synth.foldin_requests(40, r.n_m, 1, 600, seed=5)
    ptr = np.concatenate([ptr, [ptr[-1]]])   # plus one empty request
    M = x0[r.n_u * r.n_f:]
    with _model(r) as m:
        m.set_x(x0)
        u = m.foldin(ptr, items, vals)
    ref = oracle.foldin(r.n_f, r.lam, M, ptr, items, vals.astype(np.float64))
    assert _row_rel(u, ref, r.n_f) < TOL64
    assert np.all(u[-1] == 0)


def test_foldin_rejects_bad_ids(tiny):
    from paper_1508_03110_gb300 import ALSError
    r, _, x0 = tiny
    with _model(r) as m:
        m.set_x(x0)
        with pytest.raises(ALSError, match="EINVAL"):
            m.foldin(np.array([0, 2]), np.array([1, r.n_m]), np.array([3.0, 4.0]))


# -- mixed precision ---------------------------------------------------------------------
# Per-row bound of a mixed-form solve of Eq. (3)/(4) against the exact FP64
# solve u* from the same FP32 inputs, started at the current row u0:
#   |u - u*| <= rho^k |u* - u0| + C kappa(A_i) 2^-24 |u*|
# The first term is what k refinement corrections leave (rho = |I - Ahat^-1 A|;
# the split-BF16 Gram matrix has relative error about 2^-17, so rho <=
# kappa(A_i) 2^-17; the FP32 Gram about n 2^-24); with the default stopping
# rule (a further correction while rho |delta| may exceed 2^-21 of the row)
# at most 1e-6 of the step is left.  The second is the FP32 floor: the
# residual, the factor and the stored row are FP32.  Measured on a GB300 at
# the default refine_steps: at most 1.6e-7 of the step on every row of the
# tiny problem (n_f = 10, 40, 100) and on the sampled rows at full size.

def _kappas(ptr, idx, F, lam, rows):
    """kappa(A_i) of A_i = F_I^T F_I + lam n_i I for the listed rows."""
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        a, b = ptr[i], ptr[i + 1]
        Fi = F[idx[a:b]]
        w = np.linalg.eigvalsh(Fi.T @ Fi + lam * (b - a) * np.eye(F.shape[1]))
        out[t] = w[-1] / max(w[0], 1e-300)
    return out


def _mixed_row_excess(u, ustar, u0, kap, lead, C=4.0):
    """max over rows of |u - u*| / (lead |u* - u0| + C kappa 2^-24 |u*|)
    (< 1 means every row meets the bound; lead may be per row)."""
    err = np.linalg.norm(u - ustar, axis=1)
    bound = lead * np.linalg.norm(ustar - u0, axis=1) + C * kap * 2.0 ** -24 * np.linalg.norm(ustar, axis=1)
    q = np.where(err == 0.0, 0.0, err / np.maximum(bound, 1e-300))
    return float(q.max())


def _half_sweeps_vs_oracle(r, P, x0, x1, n_f):
    """(U rows, exact U, U0, kappa_U, M rows, exact M, M0, kappa_M) of one
    mixed sweep x0 -> x1: the U half against the exact solve from M0, the M
    half against the exact solve from the GPU's U (FP32)."""
    k = r.n_u * n_f
    U0, M0 = x0[:k].reshape(r.n_u, n_f), x0[k:].reshape(r.n_m, n_f)
    U1, M1 = x1[:k].reshape(r.n_u, n_f), x1[k:].reshape(r.n_m, n_f)
    Ustar = oracle.half_sweep(P, 0, M0).reshape(r.n_u, n_f)
    U1f = U1.astype(np.float32).astype(np.float64)
    Mstar = oracle.half_sweep(P, 1, U1f).reshape(r.n_m, n_f)
    ku = _kappas(P.uptr, P.uidx, M0, P.lam, np.arange(r.n_u))
    km = _kappas(P.mptr, P.midx, U1f, P.lam, np.arange(r.n_m))
    return U1, Ustar, U0, ku, M1, Mstar, M0, km


@pytest.mark.parametrize("n_f", [10, 40, 100])
def test_mixed_matches_fp64_run(tiny, n_f):
    """Mixed form: f within 1e-5 of the FP64 GPU run at equal iteration count,
    final train RMSE within 1e-4."""
    r, _, _ = tiny
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7)
    fs = {}
    xs = {}
    for prec in ("fp64", "mixed"):
        with _model(r, n_f=n_f, precision=prec) as m:
            m.set_x(x0)
            fs[prec] = []
            for k in range(30):
                fs[prec].append(m.step()["f"])
            xs[prec] = m.get_x()
    f64, fmx = np.array(fs["fp64"]), np.array(fs["mixed"])
    assert np.all(np.abs(fmx - f64) <= 1e-5 * np.abs(f64)), np.max(np.abs(fmx - f64) / np.abs(f64))

    def rmse(x):
        U = x[:r.n_u * n_f].reshape(r.n_u, n_f); M = x[r.n_u * n_f:].reshape(r.n_m, n_f)
        e = r.vals - np.einsum("ij,ij->i", U[r.rows], M[r.cols])
        return float(np.sqrt(np.mean(e ** 2)))
    assert abs(rmse(xs["mixed"]) - rmse(xs["fp64"])) < 1e-4


@pytest.mark.parametrize("n_f", [10, 40, 100])
def test_mixed_sweep_rows_meet_the_refinement_bound(tiny, n_f):
    """One mixed sweep from FP32 inputs at the default refine_steps (FP32
    Gram for n_f = 10, tensor-core Gram with light rows above): every row
    within 1e-6 of its step plus the FP32 floor."""
    r, _, _ = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7).astype(np.float32).astype(np.float64)
    with _model(r, n_f=n_f, precision="mixed") as m:
        m.set_x(x0)
        m.sweep(1)
        x1 = m.get_x()
    U1, Us, U0, ku, M1, Ms, M0, km = _half_sweeps_vs_oracle(r, P, x0, x1, n_f)
    assert _mixed_row_excess(U1, Us, U0, ku, 1e-6) < 1.0
    assert _mixed_row_excess(M1, Ms, M0, km, 1e-6) < 1.0


def test_mixed_sweep_close_to_oracle(tiny):
    """Three mixed sweeps against three exact ones: the FP32 floor compounds
    over the sweeps, so each row stays within 1e-5 of the oracle's."""
    r, P, x0 = tiny
    with _model(r, precision="mixed") as m:
        m.set_x(x0)
        m.sweep(3)
        x = m.get_x()
    ref = x0
    for _ in range(3):
        ref = oracle.sweep(P, ref)
    assert _rel(x, ref) < 1e-6
    assert _row_rel(x, ref, r.n_f) < 1e-5


# -- tensor-core Gram (mixed, n_f > 32) ------------------------------------------------

@pytest.mark.parametrize("n_f", [48, 100, 128])
def test_tc_sweep_agrees_with_fp32_gram(tiny, n_f):
    """The BF16 tensor-core Gram is the preconditioner of a refinement against
    the FP32 residual: with enough refinement steps the sweep converges to the
    same rows as the FP32-Gram path (and the FP64 oracle)."""
    r, _, _ = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3).astype(np.float32).astype(np.float64)
    ref = oracle.sweep(P, x0)
    out = {}
    for path, refine in (("tc", 1), ("fma", 1), ("tc", 4)):
        with _model(r, n_f=n_f, precision="mixed", gram_path=path, refine_steps=refine) as m:
            m.set_x(x0)
            m.sweep(1)
            out[(path, refine)] = m.get_x()
    for key, lead in ((("fma", 1), None), (("tc", 1), None), (("tc", 4), 1e-6)):
        U1, Us, U0, ku, M1, Ms, M0, km = _half_sweeps_vs_oracle(r, P, x0, out[key], n_f)
        if lead is None:
            # one correction: what is left is rho |step|, rho <= kappa 2^-17
            # (split-BF16 Gram) or n 2^-24 <= kappa 2^-17 here (FP32 Gram)
            lu, lm = ku * 2.0 ** -17, km * 2.0 ** -17
        else:
            lu = lm = lead
        assert _mixed_row_excess(U1, Us, U0, ku, lu) < 1.0, key
        assert _mixed_row_excess(M1, Ms, M0, km, lm) < 1.0, key
    assert _row_rel(out[("tc", 4)], ref, n_f) < 1e-6


def test_tc_foldin_converges(tiny):
    r, _, _ = tiny
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3).astype(np.float32).astype(np.float64)
    ptr, items, vals = synth.foldin_requests(30, r.n_m, 1, 800, seed=9)
    ref = oracle.foldin(n_f, r.lam, x0[r.n_u * n_f:], ptr, items, vals.astype(np.float64))
    with _model(r, n_f=n_f, precision="mixed", gram_path="tc", refine_steps=5) as m:
        m.set_x(x0)
        u = m.foldin(ptr, items, vals)
    # a cold start (u0 = 0): the step is u* itself
    Mf = x0[r.n_u * n_f:].reshape(r.n_m, n_f)
    kap = _kappas(ptr, items, Mf, r.lam, np.arange(len(ptr) - 1))
    assert _mixed_row_excess(u, ref, np.zeros_like(ref), kap, 1e-6) < 1.0
    assert _row_rel(u, ref, n_f) < 1e-6


def test_tc_alsncg_converges(tiny):
    r, _, _ = tiny
    n_f = 64
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3)
    with _model(r, n_f=n_f, precision="mixed", gram_path="tc") as m:
        m.set_x(x0)
        out = m.run(40)
    assert out["gnorm"] < 1e-3 * out["gnorm0"]
    assert out["notspd"] == 0
