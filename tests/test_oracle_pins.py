"""Pins of the FP64 oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage it follows."""
import numpy as np
import pytest

import oracle
import synth


def _small_problem(n_u=40, n_m=25, n_f=4, lam=0.05, dens=0.3, seed=7, min_deg=1):
    rng = np.random.default_rng(seed)
    mask = rng.random((n_u, n_m)) < dens
    for i in range(n_u):                      # every user rates >= min_deg items
        if mask[i].sum() < min_deg:
            mask[i, rng.choice(n_m, min_deg, replace=False)] = True
    for j in range(n_m):
        if mask[:, j].sum() < min_deg:
            mask[rng.choice(n_u, min_deg, replace=False), j] = True
    rows, cols = np.nonzero(mask)
    vals = np.round(2 * np.clip(rng.normal(3.5, 1.0, rows.shape[0]), 0.5, 5)) / 2
    P = oracle.build_problem(n_u, n_m, n_f, lam, rows, cols, vals)
    x0 = synth.init_factors(n_u, n_m, n_f, seed + 100)
    return P, x0


# -- per-row solve -----------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 10, 37, 100])
def test_chol_solve_matches_lapack(n):
    """Eq. (3)/(4) are solved by Cholesky (§V-B); the textbook factorisation
    must agree with LAPACK's general solver on SPD systems."""
    rng = np.random.default_rng(n)
    B = rng.normal(size=(n, 2 * n + 3))
    A = B @ B.T + 0.1 * np.eye(n)
    b = rng.normal(size=n)
    x = oracle.chol_solve(A, b)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref) * np.linalg.cond(A) ** 0.5


def test_chol_rejects_indefinite():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.chol_solve(A, np.ones(2))


def test_user_solve_is_ridge_least_squares():
    """Eq. (3): u_i minimises sum_j (r_ij - u.m_j)^2 + lambda n_ui |u|^2, i.e.
    the stacked least-squares problem [M_I^T; sqrt(lambda n) I] u = [r; 0]."""
    P, x0 = _small_problem()
    M = x0[P.n_u * P.n_f:].reshape(P.n_m, P.n_f)
    U = oracle.half_sweep(P, 0, M).reshape(P.n_u, P.n_f)
    for i in range(P.n_u):
        a, b = P.uptr[i], P.uptr[i + 1]
        MI = M[P.uidx[a:b]]
        n = b - a
        S = np.vstack([MI, np.sqrt(P.lam * n) * np.eye(P.n_f)])
        rhs = np.concatenate([P.uval[a:b], np.zeros(P.n_f)])
        ref = np.linalg.lstsq(S, rhs, rcond=None)[0]
        assert np.allclose(U[i], ref, rtol=1e-11, atol=1e-12)


def test_light_rows_through_their_ratings_matrix():
    """Eq. (3) solved through the n_i x n_i matrix of the row's ratings: for a row with
    n_i < n_f ratings, the solution of Eq. (3) is F^T (F F^T + lambda n_i I)^-1 r,
    and one correction of the mixed form's refinement from any u0,
    u0 + (v - F^T G^-1 F v) / (lambda n_i) with v = F^T (r - F u0) - lambda n_i u0,
    lands on it (Woodbury identity), all in FP64."""
    P, x0 = _small_problem(n_u=40, n_m=25, n_f=12, dens=0.3, seed=3)
    M = x0[P.n_u * P.n_f:].reshape(P.n_m, P.n_f)
    U = oracle.half_sweep(P, 0, M).reshape(P.n_u, P.n_f)
    rng = np.random.default_rng(5)
    light = 0
    for i in range(P.n_u):
        a, b = P.uptr[i], P.uptr[i + 1]
        n = b - a
        if n == 0 or n >= P.n_f:
            continue
        light += 1
        F, r, ln = M[P.uidx[a:b]], P.uval[a:b], P.lam * n
        G = F @ F.T + ln * np.eye(n)
        assert np.allclose(F.T @ np.linalg.solve(G, r), U[i], rtol=1e-10, atol=1e-13)
        u0 = rng.normal(size=P.n_f)
        v = F.T @ (r - F @ u0) - ln * u0
        u1 = u0 + (v - F.T @ np.linalg.solve(G, F @ v)) / ln
        assert np.allclose(u1, U[i], rtol=1e-9, atol=1e-12)
    assert light >= 20


def test_item_solve_is_ridge_least_squares():
    """Eq. (4), the item-side analogue."""
    P, x0 = _small_problem(seed=9)
    U = x0[:P.n_u * P.n_f].reshape(P.n_u, P.n_f)
    M = oracle.half_sweep(P, 1, U).reshape(P.n_m, P.n_f)
    for j in range(P.n_m):
        a, b = P.mptr[j], P.mptr[j + 1]
        UI = U[P.midx[a:b]]
        n = b - a
        S = np.vstack([UI, np.sqrt(P.lam * n) * np.eye(P.n_f)])
        rhs = np.concatenate([P.mval[a:b], np.zeros(P.n_f)])
        ref = np.linalg.lstsq(S, rhs, rcond=None)[0]
        assert np.allclose(M[j], ref, rtol=1e-11, atol=1e-12)


def test_empty_rows_are_held_at_zero():
    """An item nobody rated does not enter f; its solve gives 0, its gradient 0."""
    rows = np.array([0, 0, 1]); cols = np.array([0, 1, 1]); vals = np.array([4.0, 3.0, 5.0])
    P = oracle.build_problem(2, 3, 2, 0.1, rows, cols, vals)
    x = synth.init_factors(2, 3, 2, 5)
    xb = oracle.sweep(P, x)
    assert np.all(xb[(2 + 2) * 2:] == 0.0)
    g = oracle.grad(P, xb)
    assert np.all(g[(2 + 2) * 2:] == 0.0)


# -- half-sweeps and ALS (Algorithm 1) -----------------------------------------

def test_half_sweeps_zero_block_gradient():
    """§III-A: the U half sets dL/du_i = 0 for every i (closed-form normal
    equations); the M half does the same for every m_j."""
    P, x = _small_problem(n_u=60, n_m=30, n_f=5)
    k = P.n_u * P.n_f
    g0 = oracle.grad(P, x)
    xu = x.copy()
    xu[:k] = oracle.half_sweep(P, 0, x[k:])
    gu = oracle.grad(P, xu)
    assert np.linalg.norm(gu[:k]) <= 1e-10 * np.linalg.norm(g0[:k])
    xm = xu.copy()
    xm[k:] = oracle.half_sweep(P, 1, xu[:k])
    gm = oracle.grad(P, xm)
    assert np.linalg.norm(gm[k:]) <= 1e-10 * np.linalg.norm(g0[k:])


def test_als_decreases_f_every_half_sweep():
    """Each half of Algorithm 1 is an exact block minimisation, so f never rises."""
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    x = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    k = P.n_u * P.n_f
    f = oracle.loss(P, x)
    for _ in range(4):
        x = x.copy(); x[:k] = oracle.half_sweep(P, 0, x[k:])
        f1 = oracle.loss(P, x)
        assert f1 <= f * (1 + 1e-13)
        x = x.copy(); x[k:] = oracle.half_sweep(P, 1, x[:k])
        f2 = oracle.loss(P, x)
        assert f2 <= f1 * (1 + 1e-13)
        f = f2


def test_sweep_is_the_two_halves():
    """P(x) = U half from x's M block, then M half from the new U (Algorithm 1)."""
    P, x = _small_problem()
    k = P.n_u * P.n_f
    xb = oracle.sweep(P, x)
    U = oracle.half_sweep(P, 0, x[k:])
    M = oracle.half_sweep(P, 1, U)
    assert np.array_equal(xb, np.concatenate([U, M]))


# -- loss and gradient -----------------------------------------------------------

def test_loss_special_values():
    """Eq. (1) at U = M = 0 is sum r^2; a planted exact fit with lambda = 0 gives 0."""
    P, x = _small_problem(lam=0.3)
    assert oracle.loss(P, np.zeros_like(x)) == pytest.approx(np.sum(P.uval ** 2), rel=1e-14)
    rng = np.random.default_rng(3)
    U = rng.normal(size=(6, 2)); M = rng.normal(size=(5, 2))
    rows, cols = np.meshgrid(np.arange(6), np.arange(5), indexing="ij")
    rows, cols = rows.ravel(), cols.ravel()
    vals = np.einsum("ij,ij->i", U[rows], M[cols])
    Q = oracle.build_problem(6, 5, 2, 0.0, rows, cols, vals)
    assert abs(oracle.loss(Q, np.concatenate([U.ravel(), M.ravel()]))) < 1e-25 + 1e-14 * np.sum(vals ** 2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    """The gradient of §V-C equals central differences of Eq. (1)."""
    P, x = _small_problem(n_u=7, n_m=6, n_f=3, lam=0.2, dens=0.5, seed=seed)
    g = oracle.grad(P, x)
    h = 1e-6
    fd = np.empty_like(x)
    for t in range(x.shape[0]):
        e = np.zeros_like(x); e[t] = h
        fd[t] = (oracle.loss(P, x + e) - oracle.loss(P, x - e)) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g)


# -- line-search polynomial (§V-C) -------------------------------------------------

@pytest.mark.parametrize("seed", [0, 4])
def test_quartic_reproduces_loss(seed):
    """Q(alpha) = f(x + alpha p) for every alpha; c0 = f(x), c1 = g^T p, c4 >= 0."""
    P, x = _small_problem(n_u=50, n_m=30, n_f=6, seed=seed)
    rng = np.random.default_rng(seed + 1)
    p = rng.normal(size=x.shape[0]) * 0.3
    c = oracle.ls_coeffs(P, x, p)
    for a in (-1.0, 0.0, 0.3, 1.0, 2.5):
        f = oracle.loss(P, x + a * p)
        assert oracle.q_eval(c, a) == pytest.approx(f, rel=1e-12)
    assert c[0] == pytest.approx(oracle.loss(P, x), rel=1e-13)
    assert c[1] == pytest.approx(float(oracle.grad(P, x) @ p), rel=1e-11)
    assert c[4] >= 0.0
    # Vandermonde: five samples of f determine the quartic exactly
    al = np.array([-1.0, -0.4, 0.2, 0.7, 1.3])
    V = np.vander(al, 5, increasing=True)
    coef = np.linalg.solve(V, [oracle.loss(P, x + a * p) for a in al])
    assert np.allclose(coef, c, rtol=1e-7, atol=1e-9 * abs(c[0]))


def test_backtracking_armijo_invariants():
    """Algorithm 3 on Q: the accepted alpha passes the sufficient-decrease test,
    alpha / tau did not, and alpha = alpha0 tau^k."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        c = np.array([5.0, -abs(rng.normal()) - 1e-3, rng.normal(), rng.normal(), abs(rng.normal()) + 1e-6])
        ls = oracle.backtracking(c)
        assert ls.ok
        dq = lambda a: oracle.q_eval(c, a) - c[0]
        assert dq(ls.alpha) <= ls.alpha * 0.5 * c[1] * (1 - 1e-12)
        assert ls.alpha == pytest.approx(10.0 * 0.9 ** ls.shrinks, rel=1e-12)
        if ls.shrinks > 0:
            a_prev = ls.alpha / 0.9
            assert dq(a_prev) > a_prev * 0.5 * c[1] * (1 + 1e-12)
    assert not oracle.backtracking(np.array([1.0, 0.5, 1.0, 0.0, 1.0])).ok


def test_exact_step_minimises_quartic():
    rng = np.random.default_rng(1)
    for _ in range(50):
        c = np.array([3.0, -abs(rng.normal()) - 0.1, rng.normal(), rng.normal(), abs(rng.normal()) + 0.05])
        ls = oracle.exact_step(c)
        grid = np.linspace(1e-6, 50, 200001)
        qv = c[0] + grid * (c[1] + grid * (c[2] + grid * (c[3] + grid * c[4])))
        assert oracle.q_eval(c, ls.alpha) <= qv.min() + 1e-9 * abs(qv.min())


# -- Algorithm 2 ---------------------------------------------------------------------

@pytest.mark.parametrize("beta", ["pr", "fr", "hs", "prplus"])
@pytest.mark.parametrize("plain", [False, True])
def test_ncg_wrapper_reproduces_pcg(beta, plain):
    """§III-B: on f = x^T A x / 2 - b^T x with a linear preconditioner
    P(x) = x - B (A x - b) and an exact line search, Algorithm 2 with beta of
    Eq. (8) is preconditioned CG (textbook form, Nocedal & Wright Alg. 5.3).
    So are the Fletcher-Reeves, Hestenes-Stiefel and PR+ forms of beta-bar
    (on a quadratic with exact steps they coincide), and plain NCG
    (gbar = g) is textbook CG (B = I)."""
    n = 12
    rng = np.random.default_rng(5)
    Q = rng.normal(size=(n, n)); A = Q @ Q.T + n * np.eye(n)
    C = rng.normal(size=(n, n)); B = np.linalg.inv(C @ C.T + n * np.eye(n))
    if plain:
        B = np.eye(n)
    b = rng.normal(size=n); x0 = rng.normal(size=n)
    iters = []

    def step(x, p, g):
        return oracle.core.LineSearchResult(float(-(g @ p) / (p @ A @ p)), True, 0, np.inf)

    pre = None if plain else (lambda x: x - B @ (A @ x - b))
    oracle.ncg(x0, lambda x: A @ x - b, pre, step, n,
               on_iter=lambda k, x, g, info: iters.append(x.copy()), beta=beta)
    # textbook PCG
    x = x0.copy(); r = A @ x - b; y = B @ r; p = -y
    ref = []
    for _ in range(n):
        a = (r @ y) / (p @ A @ p)
        x = x + a * p
        r1 = r + a * A @ p
        y1 = B @ r1
        beta = (r1 @ y1) / (r @ y)
        p = -y1 + beta * p
        r, y = r1, y1
        ref.append(x.copy())
    xs = np.linalg.solve(A, b)
    for k in range(n):
        assert np.linalg.norm(iters[k] - ref[k]) <= 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(iters[-1] - xs) <= 1e-10 * np.linalg.norm(xs)


def _dense_minimum(R, n_f, lam):
    """Global minimum of Eq. (1) when every rating is observed:
    f = |R - U^T M|_F^2 + a|U|^2 + b|M|^2 with a = lam n_m, b = lam n_u;
    min over U^T M = Z of a|U|^2 + b|M|^2 is 2 sqrt(ab) |Z|_*, so the optimum
    soft-thresholds the top n_f singular values by s = sqrt(ab)."""
    n_u, n_m = R.shape
    s = np.sqrt(lam * n_m * lam * n_u)
    sig = np.linalg.svd(R, compute_uv=False)
    top, rest = sig[:n_f], sig[n_f:]
    val = np.where(top > s, 2 * s * top - s * s, top ** 2).sum() + (rest ** 2).sum()
    return val


def test_als_and_alsncg_reach_dense_global_minimum():
    """Closed form: on a fully observed 30 x 20 R, both Algorithm 1 and
    Algorithm 2 must reach the global minimum of Eq. (1)."""
    rows, cols, vals = synth.make_dense(30, 20, 3, seed=4)
    P = oracle.build_problem(30, 20, 3, 0.05, rows, cols, vals)
    fstar = _dense_minimum(vals.reshape(30, 20), 3, 0.05)
    x0 = synth.init_factors(30, 20, 3, 8)
    ra = oracle.als(P, x0, 400, keep_x=False, with_grad=False)
    assert ra[-1].f == pytest.approx(fstar, rel=1e-8)
    rn = oracle.alsncg(P, x0, 60, keep_x=False)
    assert rn[-1].f == pytest.approx(fstar, rel=1e-8)
    assert rn[-1].f >= fstar * (1 - 1e-12)


def test_tiny_brute_force_fixed_point():
    """n_f = 1, a 3 x 2 R with one missing rating: the ALS fixed point is the
    minimum found by a grid search over all five unknowns plus a local polish."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    rows = np.array([0, 0, 1, 1, 2]); cols = np.array([0, 1, 0, 1, 0])
    vals = np.array([4.0, 2.0, 3.5, 1.0, 5.0])
    P = oracle.build_problem(3, 2, 1, 0.1, rows, cols, vals)
    g = np.linspace(-3, 3, 25)
    G = np.stack(np.meshgrid(g, g, g, g, g, indexing="ij"), -1).reshape(-1, 5)
    u, m = G[:, :3], G[:, 3:]
    f = np.zeros(G.shape[0])
    for r_, c_, v_ in zip(rows, cols, vals):
        f += (v_ - u[:, r_] * m[:, c_]) ** 2
    nu = np.bincount(rows, minlength=3); nm = np.bincount(cols, minlength=2)
    f += 0.1 * ((nu * u ** 2).sum(1) + (nm * m ** 2).sum(1))
    best = G[np.argmin(f)]
    res = scipy_opt.minimize(lambda x: oracle.loss(P, x), best, jac=lambda x: oracle.grad(P, x),
                             method="BFGS", options=dict(gtol=1e-12, maxiter=500))
    x = np.array([0.5, 0.5, 0.5, 1.0, 1.0])
    for _ in range(2000):
        x = oracle.sweep(P, x)
    assert oracle.loss(P, x) == pytest.approx(res.fun, rel=1e-8)


def test_foldin_equals_user_half_sweep_row():
    """Fold-in is Eq. (3) for a row given from outside R: feeding an existing
    user's ratings gives that user's half-sweep row."""
    P, x = _small_problem(n_u=30, n_m=20, n_f=4)
    k = P.n_u * P.n_f
    U = oracle.half_sweep(P, 0, x[k:]).reshape(P.n_u, P.n_f)
    users = [0, 5, 17]
    ptr = np.concatenate([[0], np.cumsum([P.uptr[i + 1] - P.uptr[i] for i in users])])
    items = np.concatenate([P.uidx[P.uptr[i]:P.uptr[i + 1]] for i in users])
    vals = np.concatenate([P.uval[P.uptr[i]:P.uptr[i + 1]] for i in users])
    out = oracle.foldin(P.n_f, P.lam, x[k:], ptr, items, vals)
    assert np.allclose(out, U[users], rtol=1e-13, atol=1e-14)


def test_alsncg_beats_als_on_tiny():
    """§IV: on the same x_0, ALS-NCG reaches a lower gradient norm than ALS in
    the same number of iterations (the acceleration the paper reports)."""
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    ra = oracle.als(P, x0, 50, keep_x=False)
    rn = oracle.alsncg(P, x0, 50, keep_x=False)
    assert rn[-1].gnorm < ra[-1].gnorm
    assert rn[-1].f <= ra[-1].f * (1 + 1e-9)


def test_thread_count_does_not_change_results():
    r = synth.make_config("tiny")
    P = oracle.build_problem(r.n_u, r.n_m, r.n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    n0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        a = (oracle.loss(P, x0), oracle.grad(P, x0), oracle.sweep(P, x0), oracle.ls_coeffs(P, x0, x0))
        oracle.set_threads(4)
        b = (oracle.loss(P, x0), oracle.grad(P, x0), oracle.sweep(P, x0), oracle.ls_coeffs(P, x0, x0))
    finally:
        oracle.set_threads(n0)
    assert a[0] == b[0]
    for u, v in zip(a[1:], b[1:]):
        assert np.array_equal(u, v)


def test_solve_rows_equals_half_sweep_rows():
    P, x = _small_problem(n_u=30, n_m=20, n_f=4)
    k = P.n_u * P.n_f
    U = oracle.half_sweep(P, 0, x[k:]).reshape(P.n_u, P.n_f)
    M = oracle.half_sweep(P, 1, x[:k]).reshape(P.n_m, P.n_f)
    assert np.array_equal(oracle.solve_rows(P, 0, x[k:], [3, 0, 29]), U[[3, 0, 29]])
    assert np.array_equal(oracle.solve_rows(P, 1, x[:k], [19, 2]), M[[19, 2]])


# -- the fallback / restart branch of Algorithm 2 -------------------------------------
# The paper does not say what Algorithm 2 does when the line search finds no
# step.  The reading taken: x_{k+1} = xbar_k = P(x_k) (the ALS point, already
# computed; it never raises f), and the next direction restarts with
# beta = 0, i.e. p_{k+1} = -gbar_{k+1}.  These pins check that branch against
# quantities recomputed from scratch (sweep, gradient, the ALS driver), never
# against the ncg loop's own bookkeeping.

def _check_fallback_records(P, x0, recs):
    x_prev = np.array(x0, dtype=np.float64)
    for r in recs:
        assert r.fallback
        assert r.alpha == 0.0 and r.beta == 0.0
        xbar_prev = oracle.sweep(P, x_prev)
        assert np.array_equal(r.x, xbar_prev), r.k          # x_{k+1} = P(x_k), exactly
        xbar = oracle.sweep(P, r.x)
        gbar = r.x - xbar
        g = oracle.grad(P, r.x)
        assert np.array_equal(r.state["xbar"], xbar)
        assert np.array_equal(r.state["gbar"], gbar)
        assert np.array_equal(r.state["p"], -gbar)           # restart: p_{k+1} = -gbar_{k+1}
        assert r.state["s"] == float(gbar @ g)               # s_{k+1} = gbar_{k+1} . g_{k+1}
        assert np.array_equal(r.g, g)
        assert r.f <= oracle.loss(P, x_prev) * (1 + 1e-15)  # the ALS point never raises f
        x_prev = r.x


def test_failed_line_search_takes_the_als_point():
    """Algorithm 3 with no admissible step (alpha0 so large that the Armijo
    test fails, and no shrink allowed): every iteration takes the fallback,
    so ALS-NCG must reproduce plain ALS (Algorithm 1) bit for bit."""
    P, x0 = _small_problem(n_u=30, n_m=20, n_f=3, seed=11)
    recs = oracle.alsncg(P, x0, 6, alpha0=1e6, max_shrinks=0)
    _check_fallback_records(P, x0, recs)
    als = oracle.als(P, x0, 6)
    for r, a in zip(recs, als):
        assert np.array_equal(r.x, a.x)
        assert r.f == a.f


def test_non_descent_direction_takes_the_preconditioner_point():
    """c1 = g^T p >= 0 (p not a descent direction): no alpha is tried at all,
    the step is x_{k+1} = xbar_k and the direction restarts.  A preconditioner
    that points uphill, xbar = x + (x - P(x)), makes every p_k = -gbar_k an
    ascent direction."""
    P, x0 = _small_problem(n_u=30, n_m=20, n_f=3, seed=12)
    uphill = lambda x: x + (x - oracle.sweep(P, x))          # noqa: E731
    seen = []

    def step(x, p, g):
        c = oracle.ls_coeffs(P, x, p)
        assert c[1] == pytest.approx(float(g @ p), rel=1e-10)
        assert c[1] > 0.0
        ls = oracle.backtracking(c)
        seen.append(ls)
        return ls

    states = []
    x_prev = np.array(x0)
    out = oracle.ncg(x0, lambda x: oracle.grad(P, x), uphill, step, 4,
                     on_iter=lambda k, x, g, info: states.append((x.copy(), g.copy(), info)))
    assert all(not ls.ok and ls.shrinks == 0 for ls in seen)
    for x, g, info in states:
        assert info["fallback"] and info["beta"] == 0.0
        assert np.array_equal(x, uphill(x_prev))            # x_{k+1} = xbar_k
        gbar = x - uphill(x)
        assert np.array_equal(info["state"]["p"], -gbar)
        assert info["state"]["s"] == float(gbar @ g)
        assert np.array_equal(g, oracle.grad(P, x))
        x_prev = x
    assert np.array_equal(out, x_prev)


def test_fallback_then_resume_restarts_beta():
    """A run where some steps pass and some fall back (at most 2 shrinks):
    after every fallback the next direction is -gbar (beta = 0), after every
    accepted step beta follows Eq. (8) from recomputed vectors."""
    P, x0 = _small_problem(n_u=40, n_m=25, n_f=4, seed=13)
    recs = oracle.alsncg(P, x0, 25, max_shrinks=2)
    kinds = {r.fallback for r in recs}
    assert kinds == {True, False}, "the case must contain both branches"
    g_prev = oracle.grad(P, x0)
    gbar_prev = x0 - oracle.sweep(P, x0)
    p_prev = -gbar_prev
    x_prev = np.array(x0)
    for r in recs:
        if r.fallback:
            assert np.array_equal(r.x, oracle.sweep(P, x_prev))
            assert r.beta == 0.0
        else:
            assert np.allclose(r.x, x_prev + r.alpha * p_prev, rtol=0, atol=1e-14 * np.abs(r.x).max())
        gbar = r.x - oracle.sweep(P, r.x)
        g = oracle.grad(P, r.x)
        beta = 0.0 if r.fallback else float(gbar @ (g - g_prev)) / float(gbar_prev @ g_prev)
        assert r.beta == pytest.approx(beta, rel=1e-12, abs=1e-300)
        p = -gbar + beta * p_prev
        assert np.allclose(r.state["p"], p, rtol=0, atol=1e-12 * np.abs(p).max())
        x_prev, g_prev, gbar_prev, p_prev = r.x, g, gbar, r.state["p"]


# -- the More-Thuente line search on Q (variant; the paper's serial runs, §IV) ----------

def _random_quartics(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        scale = 10.0 ** rng.uniform(-3, 3)
        c = np.array([rng.normal() * scale, -abs(rng.normal()) * scale, rng.normal() * scale,
                      rng.normal() * scale, (abs(rng.normal()) + 0.01) * scale])
        out.append(c)
    return out


def test_more_thuente_meets_strong_wolfe():
    """Every converged step satisfies Q(a) - Q(0) <= ftol a Q'(0) and
    |Q'(a)| <= gtol |Q'(0)|, with the paper's tolerances."""
    n_ok = 0
    for c in _random_quartics(400, 1):
        ls = oracle.more_thuente(c, 1.0, 1e-4, 1e-2)
        assert ls.ok
        a = ls.alpha
        dq = a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])))
        assert dq <= 1e-4 * a * c[1] + 1e-12 * abs(c[1]) * a
        if ls.shrinks < 20:
            assert abs(oracle.q_deriv(c, a)) <= 1e-2 * abs(c[1]) * (1 + 1e-9)
            n_ok += 1
    assert n_ok >= 390


def test_more_thuente_equals_an_independent_implementation():
    """The same published algorithm, implemented independently (scipy's port
    of MINPACK-2's dcsrch, reached through scalar_search_wolfe1), picks the
    same step on random quartics wherever both converge."""
    L = pytest.importorskip("scipy.optimize._linesearch")
    agree = compared = 0
    for c in _random_quartics(400, 2):
        phi = lambda a: a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])))   # noqa: E731
        dphi = lambda a: oracle.q_deriv(c, a)                               # noqa: E731
        ref = L.scalar_search_wolfe1(phi, dphi, phi0=0.0, derphi0=float(c[1]), c1=1e-4, c2=1e-2,
                                     amax=1e15, amin=1e-15, xtol=1e-15)[0]
        ls = oracle.more_thuente(c, 1.0, 1e-4, 1e-2, maxfev=100)
        if ref is None or not ls.ok or ls.shrinks >= 100:
            continue
        compared += 1
        if abs(ls.alpha - ref) <= 1e-8 * abs(ref):
            agree += 1
    assert compared >= 350
    assert agree == compared, (agree, compared)


def test_more_thuente_on_a_quadratic_takes_the_minimiser():
    """On Q with c3 = c4 = 0 (a quadratic), once alpha0 = 1 fails the
    curvature test the cubic/quadratic interpolation is exact, so the search
    lands on the minimiser -c1 / (2 c2)."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        c2 = abs(rng.normal()) + 0.1
        amin = 10.0 ** rng.uniform(-2, 2)
        c = np.array([1.0, -2.0 * c2 * amin, c2, 0.0, 0.0])
        ls = oracle.more_thuente(c, 1.0, 1e-4, 1e-2)
        assert ls.ok
        if abs(amin - 1.0) > 0.02 * amin:
            assert ls.alpha == pytest.approx(amin, rel=1e-10)


@pytest.mark.parametrize("beta", ["pr", "fr", "hs", "prplus"])
def test_beta_forms_on_recomputed_vectors(beta):
    """Each beta-bar form, per iteration of ALS-NCG, from the vectors
    recomputed from scratch (sweep, gradient) rather than the loop's own."""
    P, x0 = _small_problem(n_u=30, n_m=20, n_f=3, seed=21)
    recs = oracle.alsncg(P, x0, 8, beta=beta)
    g, gbar = oracle.grad(P, x0), x0 - oracle.sweep(P, x0)
    p = -gbar
    for r in recs:
        gn, gbn = oracle.grad(P, r.x), r.x - oracle.sweep(P, r.x)
        y = gn - g
        ref = {"pr": gbn @ y / (gbar @ g), "fr": gbn @ gn / (gbar @ g), "hs": gbn @ y / (p @ y),
               "prplus": max(0.0, gbn @ y / (gbar @ g))}[beta]
        if r.fallback:
            ref = 0.0
        assert r.beta == pytest.approx(float(ref), rel=1e-9, abs=1e-300)
        g, gbar, p = gn, gbn, r.state["p"]


def test_plain_ncg_restarts_in_place():
    """Plain NCG (gbar = g): a failed line search keeps x_k and restarts along
    -g_k; an accepted one moves along p.  f never increases."""
    P, x0 = _small_problem(n_u=30, n_m=20, n_f=3, seed=22)
    recs = oracle.alsncg(P, x0, 30, precond="none", max_shrinks=3, alpha0=0.03)
    assert any(r.fallback for r in recs) and not all(r.fallback for r in recs)
    x_prev, f_prev = x0, oracle.loss(P, x0)
    for r in recs:
        g = oracle.grad(P, r.x)
        if r.fallback:
            assert np.array_equal(r.x, x_prev)
            assert np.array_equal(r.state["p"], -g)
        assert np.array_equal(r.state["gbar"], g)
        assert r.f <= f_prev * (1 + 1e-15)
        x_prev, f_prev = r.x, r.f


def test_alsncg_with_more_thuente_reaches_dense_minimum():
    """ALS-NCG with the More-Thuente search (the paper's serial setting:
    alpha0 = 1, ftol 1e-4, gtol 1e-2, 20 evaluations) reaches the closed-form
    global minimum of a fully observed problem."""
    rng = np.random.default_rng(9)
    n_u, n_m, n_f, lam = 30, 20, 3, 0.1
    R = rng.normal(size=(n_u, n_f)) @ rng.normal(size=(n_f, n_m)) + 0.1 * rng.normal(size=(n_u, n_m))
    rows, cols = np.nonzero(np.ones((n_u, n_m)))
    P = oracle.build_problem(n_u, n_m, n_f, lam, rows, cols, R[rows, cols])
    x0 = synth.init_factors(n_u, n_m, n_f, 3)
    recs = oracle.alsncg(P, x0, 300, alpha0=1.0, cc=1e-4, max_shrinks=20, mode="mt", c2=1e-2)
    fstar = _dense_minimum(R, n_f, lam)
    assert recs[-1].f == pytest.approx(fstar, rel=1e-8)


# -- top-t ranking accuracy (§IV) -------------------------------------------------------

def test_ranking_metric_worked_example():
    """The paper's worked example (tests/golden/kendall_tau_example.json):
    p1 = [6,3,1,2,4,5], p2 = [3,4,2,5,6,1], t = 2 take 4 swaps (movie 6 from
    the 5th place to the 1st, movie 3 already 2nd), s_max = 9, q = 5/9."""
    import json
    import os
    from fractions import Fraction
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kendall_tau_example.json")))
    s = oracle.ranking.swaps_to_front(g["p1"][:g["t"]], g["p2"])
    assert s == g["swaps"]
    assert oracle.ranking.s_max(g["n_m"], g["t"]) == g["s_max"]
    assert Fraction(1) - Fraction(s, int(oracle.ranking.s_max(g["n_m"], g["t"]))) == Fraction(g["q"])


def _adjacent_swaps(top, p2):
    """Literal count: bubble each reference item forward one adjacent swap at a time."""
    cur = list(p2)
    n = 0
    for k, a in enumerate(top):
        i = cur.index(a)
        while i > k:
            cur[i - 1], cur[i] = cur[i], cur[i - 1]
            i -= 1
            n += 1
    return n, cur


def test_ranking_swaps_equal_adjacent_swap_counting():
    rng = np.random.default_rng(0)
    for _ in range(300):
        n_m = int(rng.integers(2, 40))
        t = int(rng.integers(1, n_m + 1))
        p1, p2 = rng.permutation(n_m), rng.permutation(n_m)
        n, cur = _adjacent_swaps(list(p1[:t]), list(p2))
        assert oracle.ranking.swaps_to_front(p1[:t], p2) == n
        assert list(cur[:t]) == list(p1[:t])


def test_ranking_identical_and_reversed():
    """q = 1 when p2 equals p1 on the top t; s = s_max when p2 is p1 reversed."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        n_m = int(rng.integers(2, 60))
        t = int(rng.integers(1, n_m + 1))
        p1 = rng.permutation(n_m)
        assert oracle.ranking.swaps_to_front(p1[:t], p1) == 0
        assert oracle.ranking.swaps_to_front(p1[:t], p1[::-1]) == oracle.ranking.s_max(n_m, t)


def test_rank_accuracy_of_factors():
    """From factors: the ranking is by descending u . m (ties by id), the
    reference top-t of the same factors gives q = 1, and q_i equals the
    paper's procedure applied to the two orderings."""
    rng = np.random.default_rng(2)
    U, M = rng.normal(size=(30, 4)), rng.normal(size=(50, 4))
    top = oracle.ranking.topt(U, M, 5)
    for i in range(30):
        assert list(top[i]) == list(np.argsort(-(M @ U[i]), kind="stable")[:5])
    qm, q, s = oracle.ranking.rank_accuracy(U, M, top)
    assert qm == 1.0 and np.all(s == 0)
    U2 = U + 0.3 * rng.normal(size=U.shape)
    qm2, q2, s2 = oracle.ranking.rank_accuracy(U2, M, top)
    for i in range(30):
        n, _ = _adjacent_swaps(list(top[i]), list(np.argsort(-(M @ U2[i]), kind="stable")))
        assert s2[i] == n
    assert 0.0 <= qm2 < 1.0
