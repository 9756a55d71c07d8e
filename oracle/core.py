"""Python half of the FP64 oracle: data preparation, the ctypes binding of
``als_oracle.c``, and the drivers (Algorithms 1, 2, 3) written step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper where it is silent (the same readings the CUDA path
takes):
  * Line search (Algorithm 3) is evaluated on the quartic Q of §V-C.  Its
    sufficient-decrease test is written in difference form,
    Q(a) - Q(0) = c1 a + c2 a^2 + c3 a^3 + c4 a^4 <= a * c * c1,
    with g^T p taken as c1 = Q'(0) from the same pass.  alpha_0 = 10,
    tau = 0.9, c = 0.5 (§V-C), at most 200 shrinks.
  * If c1 >= 0 (p is not a descent direction) or no alpha passes within the
    shrink limit, the step falls back to the ALS point x_{k+1} = xbar_k =
    P(x_k) (already computed) and the next direction restarts with beta = 0.
  * x_0 is given by the caller (the same x_0 for ALS and ALS-NCG).
"""
import ctypes
import dataclasses
import math

import numpy as np

from . import build as _build

_lib = None


class _CProblem(ctypes.Structure):
    _fields_ = [
        ("n_u", ctypes.c_int64), ("n_m", ctypes.c_int64), ("n_f", ctypes.c_int32),
        ("lam", ctypes.c_double),
        ("uptr", ctypes.c_void_p), ("uidx", ctypes.c_void_p), ("uval", ctypes.c_void_p),
        ("mptr", ctypes.c_void_p), ("midx", ctypes.c_void_p), ("mval", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    P = ctypes.POINTER(_CProblem)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_loss.argtypes = [P, vp]; lib.orc_loss.restype = dbl
    lib.orc_grad.argtypes = [P, vp, vp]; lib.orc_grad.restype = None
    lib.orc_half_sweep.argtypes = [P, i32, vp, vp]; lib.orc_half_sweep.restype = i64
    lib.orc_sweep.argtypes = [P, vp, vp]; lib.orc_sweep.restype = i64
    lib.orc_ls_coeffs.argtypes = [P, vp, vp, vp]; lib.orc_ls_coeffs.restype = None
    lib.orc_chol_solve.argtypes = [i32, vp, vp, vp, vp]; lib.orc_chol_solve.restype = i32
    lib.orc_foldin.argtypes = [i32, dbl, i64, vp, vp, vp, vp, vp]; lib.orc_foldin.restype = i64
    lib.orc_solve_rows.argtypes = [P, i32, vp, i64, vp, vp]; lib.orc_solve_rows.restype = i64
    lib.orc_set_threads.argtypes = [i32]; lib.orc_set_threads.restype = None
    lib.orc_get_threads.argtypes = []; lib.orc_get_threads.restype = i32
    _lib = lib
    return lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclasses.dataclass
class Problem:
    """Ratings stored twice (§V-B): by user and by item, each list sorted."""
    n_u: int
    n_m: int
    n_f: int
    lam: float
    uptr: np.ndarray  # int64 [n_u+1]
    uidx: np.ndarray  # int32 [nnz] item ids, ascending within a user
    uval: np.ndarray  # float64 [nnz]
    mptr: np.ndarray  # int64 [n_m+1]
    midx: np.ndarray  # int32 [nnz] user ids, ascending within an item
    mval: np.ndarray  # float64 [nnz]
    _c: _CProblem = None

    @property
    def nnz(self) -> int:
        return int(self.uidx.shape[0])

    @property
    def N(self) -> int:
        """Number of unknowns, n_f (n_u + n_m) (Eq. 5)."""
        return self.n_f * (self.n_u + self.n_m)

    def cstruct(self):
        if self._c is None:
            self._c = _CProblem(self.n_u, self.n_m, self.n_f, self.lam,
                                _ptr(self.uptr), _ptr(self.uidx), _ptr(self.uval),
                                _ptr(self.mptr), _ptr(self.midx), _ptr(self.mval))
        return ctypes.byref(self._c)


def build_problem(n_u, n_m, n_f, lam, rows, cols, vals) -> Problem:
    """Store R by user and R^T by item (§V-B) from COO triplets."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    if rows.size and (rows.min() < 0 or rows.max() >= n_u or cols.min() < 0 or cols.max() >= n_m):
        raise ValueError("rating index out of range")
    o = np.lexsort((cols, rows))
    r_s, c_s = rows[o], cols[o]
    if r_s.size > 1 and np.any((r_s[1:] == r_s[:-1]) & (c_s[1:] == c_s[:-1])):
        raise ValueError("duplicate (user, item) rating")
    uptr = np.zeros(n_u + 1, np.int64)
    np.cumsum(np.bincount(r_s, minlength=n_u), out=uptr[1:])
    o2 = np.lexsort((rows, cols))
    mptr = np.zeros(n_m + 1, np.int64)
    np.cumsum(np.bincount(cols[o2], minlength=n_m), out=mptr[1:])
    return Problem(int(n_u), int(n_m), int(n_f), float(lam),
                   uptr, np.ascontiguousarray(c_s, np.int32), np.ascontiguousarray(vals[o]),
                   mptr, np.ascontiguousarray(rows[o2], np.int32), np.ascontiguousarray(vals[o2]))


def _vec(P: Problem, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    if x.shape[0] != P.N:
        raise ValueError(f"vector has {x.shape[0]} entries, expected {P.N}")
    return x


def loss(P: Problem, x) -> float:
    """Eq. (1)."""
    x = _vec(P, x)
    return float(_load().orc_loss(P.cstruct(), _ptr(x)))


def grad(P: Problem, x) -> np.ndarray:
    """Gradient of Eq. (1) (§III-A, §V-C)."""
    x = _vec(P, x)
    g = np.empty_like(x)
    _load().orc_grad(P.cstruct(), _ptr(x), _ptr(g))
    return g


def half_sweep(P: Problem, side: int, F) -> np.ndarray:
    """side 0: all u_i by Eq. (3) from the M block F; side 1: all m_j by Eq. (4)
    from the U block F.  Returns the solved block."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    n = P.n_u if side == 0 else P.n_m
    out = np.empty(n * P.n_f, np.float64)
    bad = _load().orc_half_sweep(P.cstruct(), int(side), _ptr(F), _ptr(out))
    if bad:
        raise FloatingPointError(f"{bad} rows not positive definite")
    return out


def solve_rows(P: Problem, side: int, F, rows) -> np.ndarray:
    """Eq. (3) (side 0) or Eq. (4) (side 1) for the selected rows only."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.shape[0] * P.n_f, np.float64)
    bad = _load().orc_solve_rows(P.cstruct(), int(side), _ptr(F), rows.shape[0], _ptr(rows), _ptr(out))
    if bad:
        raise FloatingPointError(f"{bad} rows not positive definite")
    return out.reshape(rows.shape[0], P.n_f)


def sweep(P: Problem, x) -> np.ndarray:
    """P(x): one ALS iteration (Algorithm 1 loop body)."""
    x = _vec(P, x)
    xb = np.empty_like(x)
    bad = _load().orc_sweep(P.cstruct(), _ptr(x), _ptr(xb))
    if bad:
        raise FloatingPointError(f"{bad} rows not positive definite")
    return xb


def ls_coeffs(P: Problem, x, p) -> np.ndarray:
    """c_0..c_4 of Q(alpha) = f(x + alpha p) (§V-C)."""
    x, p = _vec(P, x), _vec(P, p)
    c = np.zeros(5, np.float64)
    _load().orc_ls_coeffs(P.cstruct(), _ptr(x), _ptr(p), _ptr(c))
    return c


def chol_solve(A, b) -> np.ndarray:
    """Textbook Cholesky solve of one SPD system."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    n = b.shape[0]
    x = np.empty(n, np.float64)
    L = np.zeros((n, n), np.float64)
    if _load().orc_chol_solve(n, _ptr(A), _ptr(b), _ptr(x), _ptr(L)) != 0:
        raise np.linalg.LinAlgError("matrix not positive definite")
    return x


def foldin(n_f, lam, M, req_ptr, items, vals) -> np.ndarray:
    """Eq. (3) for new users (rows not in R) against a fixed M."""
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(-1)
    req_ptr = np.ascontiguousarray(req_ptr, dtype=np.int64)
    items = np.ascontiguousarray(items, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    nq = req_ptr.shape[0] - 1
    out = np.empty(nq * n_f, np.float64)
    bad = _load().orc_foldin(int(n_f), float(lam), nq, _ptr(req_ptr), _ptr(items),
                             _ptr(vals), _ptr(M), _ptr(out))
    if bad:
        raise FloatingPointError(f"{bad} requests not positive definite")
    return out.reshape(nq, n_f)


# --------------------------------------------------------------------------
# Line search on Q (§V-C, Algorithm 3)
# --------------------------------------------------------------------------

def q_eval(c, alpha) -> float:
    """Q(alpha) = sum_n c_n alpha^n."""
    return float(c[0] + alpha * (c[1] + alpha * (c[2] + alpha * (c[3] + alpha * c[4]))))


@dataclasses.dataclass
class LineSearchResult:
    alpha: float
    ok: bool
    shrinks: int
    margin: float  # relative slack of the deciding test (tie detection)


def backtracking(c, alpha0=10.0, tau=0.9, cc=0.5, max_shrinks=200) -> LineSearchResult:
    """Algorithm 3 on Q: shrink alpha by tau until
    Q(alpha) - Q(0) <= alpha * cc * g^T p, with g^T p = c1."""
    c1 = float(c[1])
    if not (c1 < 0.0):
        return LineSearchResult(0.0, False, 0, float("inf"))
    alpha = float(alpha0)
    margin = float("inf")
    for k in range(max_shrinks + 1):
        dq = alpha * (c[1] + alpha * (c[2] + alpha * (c[3] + alpha * c[4])))
        rhs = alpha * cc * c1
        scale = abs(dq) + abs(rhs)
        margin = min(margin, abs(dq - rhs) / scale if scale > 0 else 0.0)
        if dq <= rhs:
            return LineSearchResult(alpha, True, k, margin)
        alpha *= tau
    return LineSearchResult(0.0, False, max_shrinks, margin)


def exact_step(c) -> LineSearchResult:
    """Variant: the alpha > 0 minimising Q, from the real roots of
    Q'(alpha) = c1 + 2 c2 alpha + 3 c3 alpha^2 + 4 c4 alpha^3."""
    if not (c[1] < 0.0):
        return LineSearchResult(0.0, False, 0, float("inf"))
    roots = np.roots([4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1]])
    cand = [float(r.real) for r in roots if abs(r.imag) <= 1e-12 * max(1.0, abs(r)) and r.real > 0]
    if not cand:
        return LineSearchResult(0.0, False, 0, float("inf"))
    best = min(cand, key=lambda a: q_eval(c, a))
    return LineSearchResult(best, True, 0, float("inf"))


# --------------------------------------------------------------------------
# Variant: the More-Thuente line search (the paper's serial experiments, §IV,
# use it: sufficient-decrease tolerance 1e-4, curvature tolerance 1e-2,
# initial step 1, at most 20 evaluations).  Written from the published
# algorithm (More & Thuente, ACM TOMS 20(3), 1994): trial steps in an
# interval of uncertainty, updated by the cases of its Section 4 (cubic,
# quadratic and secant steps), first on the auxiliary function
# psi(a) = phi(a) - phi(0) - ftol a phi'(0), then on phi itself; the
# extrapolation range [1.1, 4] x the last move when nothing is bracketed.
# phi is Q - c0 (difference form) and phi' = Q', both exact here.
# --------------------------------------------------------------------------

def q_deriv(c, alpha) -> float:
    """Q'(alpha) = c1 + 2 c2 alpha + 3 c3 alpha^2 + 4 c4 alpha^3."""
    return float(c[1] + alpha * (2.0 * c[2] + alpha * (3.0 * c[3] + alpha * 4.0 * c[4])))


def _cubic_step(a, fa, da, b, fb, db):
    """Minimiser of the cubic through (a, fa) and (b, fb) with slopes da, db
    (Nocedal & Wright, Numerical Optimization, eq. 3.59), or None when that
    cubic has no real local minimiser."""
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def _quad_step(a, fa, da, b, fb):
    """Minimiser of the quadratic through (a, fa) with slope da and (b, fb)."""
    return a + 0.5 * da * ((b - a) * (b - a)) / (fa - fb + da * (b - a))


def _secant_step(a, da, b, db):
    """Zero of the line through the slopes (a, da) and (b, db)."""
    return b - db * (b - a) / (db - da)


def _mt_trial(x, fx, dx, y, fy, dy, t, ft, dt, brackt, lo, hi):
    """One trial-step choice and interval update of More & Thuente (§4).
    x: the best step so far, y: the other end, t: the current trial.
    Returns (x, fx, dx, y, fy, dy, t_next, brackt)."""
    same = dt * math.copysign(1.0, dx) > 0.0
    if ft > fx:
        # case 1: a higher value -> the minimiser is bracketed by x and t
        c = _cubic_step(x, fx, dx, t, ft, dt)
        q = _quad_step(x, fx, dx, t, ft)
        if c is None:
            c = q
        nxt = c if abs(c - x) < abs(q - x) else c + 0.5 * (q - c)
        brackt = True
    elif not same:
        # case 2: lower value, slopes of opposite sign -> bracketed by x and t
        c = _cubic_step(x, fx, dx, t, ft, dt)
        sct = _secant_step(x, dx, t, dt)
        if c is None:
            c = sct
        nxt = c if abs(c - t) >= abs(sct - t) else sct
        brackt = True
    elif abs(dt) < abs(dx):
        # case 3: lower value, same slope sign, slope decreasing in size
        c = _cubic_step(x, fx, dx, t, ft, dt)
        beyond = c is not None and (c - t) * (t - x) > 0.0
        if not beyond:
            c = hi if t > x else lo
        sct = _secant_step(x, dx, t, dt)
        if brackt:
            nxt = c if abs(c - t) < abs(sct - t) else sct
            lim = t + 0.66 * (y - t)
            nxt = min(lim, nxt) if t > x else max(lim, nxt)
        else:
            nxt = c if abs(c - t) > abs(sct - t) else sct
            nxt = min(hi, max(lo, nxt))
    else:
        # case 4: lower value, same slope sign, slope not decreasing
        if brackt:
            c = _cubic_step(t, ft, dt, y, fy, dy)
            nxt = c if c is not None else 0.5 * (t + y)
        else:
            nxt = hi if t > x else lo
    # the interval: the end points keep the minimiser between them
    if ft > fx:
        y, fy, dy = t, ft, dt
    else:
        if not same:
            y, fy, dy = x, fx, dx
        x, fx, dx = t, ft, dt
    return x, fx, dx, y, fy, dy, nxt, brackt


def more_thuente(c, alpha0=1.0, ftol=1e-4, gtol=1e-2, xtol=1e-15, stpmin=1e-15, stpmax=1e15,
                 maxfev=20) -> "LineSearchResult":
    """The More-Thuente search for a step satisfying the strong Wolfe
    conditions on Q: Q(a) - Q(0) <= ftol a Q'(0) and |Q'(a)| <= gtol |Q'(0)|.
    `shrinks` holds the number of evaluations.  If no such step is found
    within maxfev evaluations (or the interval collapses), the best step seen
    is taken when it gives sufficient decrease; otherwise the search fails."""
    g0 = float(c[1])
    if not (g0 < 0.0):
        return LineSearchResult(0.0, False, 0, float("inf"))
    phi = lambda a: a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])))   # noqa: E731  Q(a) - c0
    gtest = ftol * g0
    brackt, stage1 = False, True
    width = stpmax - stpmin
    width_prev = 2.0 * width
    x, fx, dx = 0.0, 0.0, g0
    y, fy, dy = 0.0, 0.0, g0
    lo, hi = 0.0, alpha0 + 4.0 * alpha0
    t = min(max(alpha0, stpmin), stpmax)
    best = None
    for nfev in range(1, maxfev + 1):
        ft, dt = phi(t), q_deriv(c, t)
        ftest = t * gtest
        if ft <= ftest and (best is None or ft < best[1]):
            best = (t, ft)
        if stage1 and ft <= ftest and dt >= 0.0:
            stage1 = False
        if ft <= ftest and abs(dt) <= -gtol * g0:
            return LineSearchResult(t, True, nfev, float("inf"))
        if (brackt and (t <= lo or t >= hi)) or (brackt and hi - lo <= xtol * hi) or \
                (t == stpmax and ft <= ftest and dt <= gtest) or (t == stpmin and (ft > ftest or dt >= gtest)):
            break
        if stage1 and ft <= fx and ft > ftest:
            # the auxiliary function psi = phi - a gtest
            x, fxm, dxm, y, fym, dym, t_new, brackt = _mt_trial(
                x, fx - x * gtest, dx - gtest, y, fy - y * gtest, dy - gtest, t, ft - t * gtest, dt - gtest,
                brackt, lo, hi)
            fx, dx = fxm + x * gtest, dxm + gtest
            fy, dy = fym + y * gtest, dym + gtest
        else:
            x, fx, dx, y, fy, dy, t_new, brackt = _mt_trial(x, fx, dx, y, fy, dy, t, ft, dt, brackt, lo, hi)
        if brackt:
            if abs(y - x) >= 0.66 * width_prev:
                t_new = x + 0.5 * (y - x)
            width_prev = width
            width = abs(y - x)
            lo, hi = min(x, y), max(x, y)
        else:
            lo, hi = t_new + 1.1 * (t_new - x), t_new + 4.0 * (t_new - x)
        t_new = min(max(t_new, stpmin), stpmax)
        if (brackt and (t_new <= lo or t_new >= hi)) or (brackt and hi - lo <= xtol * hi):
            t_new = x
        t = t_new
    if best is not None:
        return LineSearchResult(best[0], True, nfev, float("inf"))
    return LineSearchResult(0.0, False, nfev, float("inf"))


# --------------------------------------------------------------------------
# Algorithm 2 (generic) and the ALS / ALS-NCG drivers
# --------------------------------------------------------------------------

BETA_FORMS = ("pr", "fr", "hs", "prplus")


def beta_bar(form, gbar_new, g_new, g, gbar, p):
    """beta-bar_{k+1} in the preconditioned forms (g -> gbar where the
    direction is built, as in Eq. (8)):
      pr     Eq. (8): gbar_{k+1}^T (g_{k+1} - g_k) / gbar_k^T g_k
      fr     Fletcher-Reeves: gbar_{k+1}^T g_{k+1} / gbar_k^T g_k
      hs     Hestenes-Stiefel: gbar_{k+1}^T (g_{k+1} - g_k) / p_k^T (g_{k+1} - g_k)
      prplus max(0, pr)
    On a convex quadratic with an exact line search and a linear
    preconditioner all four equal preconditioned CG's beta.  A zero
    denominator gives 0."""
    y = g_new - g
    if form in ("pr", "prplus"):
        den = float(gbar @ g)
        b = float(gbar_new @ y) / den if den != 0.0 else 0.0
        return max(0.0, b) if form == "prplus" else b
    if form == "fr":
        den = float(gbar @ g)
        return float(gbar_new @ g_new) / den if den != 0.0 else 0.0
    if form == "hs":
        den = float(p @ y)
        return float(gbar_new @ y) / den if den != 0.0 else 0.0
    raise ValueError(f"unknown beta form {form!r}")

@dataclasses.dataclass
class IterRecord:
    k: int
    x: np.ndarray
    f: float
    gnorm: float
    alpha: float = float("nan")
    beta: float = float("nan")
    fallback: bool = False
    shrinks: int = 0
    margin: float = float("inf")
    c: np.ndarray = None
    state: dict = None   # p_k, gbar_k, xbar_k, s_k after this iteration (Algorithm 2)
    g: np.ndarray = None


def ncg(x0, grad_fn, precond_fn, step_fn, iters, on_iter=None, beta="pr"):
    """Algorithm 2 with a general preconditioner P and gradient g:
      gbar_0 = x_0 - P(x_0), p_0 = -gbar_0;
      each k: alpha_k from step_fn, x_{k+1} = x_k + alpha_k p_k,
              gbar_{k+1} = x_{k+1} - P(x_{k+1}),
              beta_{k+1} = gbar_{k+1}^T (g_{k+1} - g_k) / (gbar_k^T g_k)  (Eq. 8,
                           or another form of beta_bar()),
              p_{k+1} = -gbar_{k+1} + beta_{k+1} p_k.
    step_fn(x, p, g) -> LineSearchResult.  A failed step takes the
    preconditioner point xbar_k and restarts the direction (beta = 0).
    precond_fn = None is plain NCG (P = identity in the preconditioned
    gradient: gbar = g); a failed step then keeps x_k and restarts along -g.
    on_iter(k, x, g, info_dict) is called after every iteration."""
    x = np.array(x0, dtype=np.float64, copy=True)
    g = grad_fn(x)
    if precond_fn is None:
        xbar, gbar = x.copy(), g
    else:
        xbar = precond_fn(x)
        gbar = x - xbar
    p = -gbar
    s = float(gbar @ g)
    for k in range(iters):
        ls = step_fn(x, p, g)
        if ls.ok:
            x = x + ls.alpha * p
        else:
            x = xbar.copy()
        g_new = grad_fn(x)
        if precond_fn is None:
            xbar, gbar_new = x.copy(), g_new
        else:
            xbar = precond_fn(x)
            gbar_new = x - xbar
        if ls.ok:
            b = beta_bar(beta, gbar_new, g_new, g, gbar, p)
        else:
            b = 0.0
        p = -gbar_new + b * p
        s = float(gbar_new @ g_new)
        g, gbar = g_new, gbar_new
        beta_k = b
        if on_iter is not None:
            on_iter(k, x, g, dict(alpha=ls.alpha, beta=beta_k, fallback=not ls.ok,
                                  shrinks=ls.shrinks, margin=ls.margin,
                                  state=dict(p=p, gbar=gbar, xbar=xbar, s=s)))
    return x


def alsncg(P: Problem, x0, iters, alpha0=10.0, tau=0.9, cc=0.5, max_shrinks=200,
           mode="backtrack", keep_x=True, beta="pr", precond="als", c2=1e-2):
    """ALS-NCG (Algorithm 2) with P = one ALS sweep and the line search of §V-C.
    Variants: mode "exact" (minimiser of Q) or "mt" (More-Thuente on Q with
    sufficient decrease cc, curvature c2, start alpha0 and at most
    max_shrinks evaluations); beta one of BETA_FORMS; precond "none" is plain
    NCG (gbar = g).  Returns the list of IterRecord, one per iteration (after
    the update)."""
    recs = []
    last_c = {}

    def step(x, p, g):
        c = ls_coeffs(P, x, p)
        last_c["c"] = c
        if mode == "exact":
            return exact_step(c)
        if mode == "mt":
            return more_thuente(c, alpha0, cc, c2, maxfev=max_shrinks)
        return backtracking(c, alpha0, tau, cc, max_shrinks)

    def on_iter(k, x, g, info):
        if not keep_x:
            info = dict(info, state=None)
        recs.append(IterRecord(k=k + 1, x=x.copy() if keep_x else None, f=loss(P, x),
                               gnorm=float(np.linalg.norm(g)), c=last_c.get("c"),
                               g=g.copy() if keep_x else None, **info))

    pre = None if precond == "none" else (lambda x: sweep(P, x))
    ncg(x0, lambda x: grad(P, x), pre, step, iters, on_iter, beta=beta)
    return recs


def als(P: Problem, x0, sweeps, keep_x=True, with_grad=True):
    """Algorithm 1: repeat x <- P(x).  Records f and |g| after every sweep."""
    x = np.array(x0, dtype=np.float64, copy=True)
    recs = []
    for k in range(sweeps):
        x = sweep(P, x)
        gn = float(np.linalg.norm(grad(P, x))) if with_grad else float("nan")
        recs.append(IterRecord(k=k + 1, x=x.copy() if keep_x else None, f=loss(P, x), gnorm=gn))
    return recs
