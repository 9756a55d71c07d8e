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
# Algorithm 2 (generic) and the ALS / ALS-NCG drivers
# --------------------------------------------------------------------------

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


def ncg(x0, grad_fn, precond_fn, step_fn, iters, on_iter=None):
    """Algorithm 2 with a general preconditioner P and gradient g:
      gbar_0 = x_0 - P(x_0), p_0 = -gbar_0;
      each k: alpha_k from step_fn, x_{k+1} = x_k + alpha_k p_k,
              gbar_{k+1} = x_{k+1} - P(x_{k+1}),
              beta_{k+1} = gbar_{k+1}^T (g_{k+1} - g_k) / (gbar_k^T g_k)  (Eq. 8),
              p_{k+1} = -gbar_{k+1} + beta_{k+1} p_k.
    step_fn(x, p, g) -> LineSearchResult.  A failed step takes the
    preconditioner point xbar_k and restarts the direction (beta = 0).
    on_iter(k, x, g, info_dict) is called after every iteration."""
    x = np.array(x0, dtype=np.float64, copy=True)
    g = grad_fn(x)
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
        xbar = precond_fn(x)
        gbar_new = x - xbar
        g_new = grad_fn(x)
        if ls.ok and s != 0.0:
            beta = float(gbar_new @ (g_new - g)) / s
        else:
            beta = 0.0
        p = -gbar_new + beta * p
        s = float(gbar_new @ g_new)
        g, gbar = g_new, gbar_new
        if on_iter is not None:
            on_iter(k, x, g, dict(alpha=ls.alpha, beta=beta, fallback=not ls.ok,
                                  shrinks=ls.shrinks, margin=ls.margin,
                                  state=dict(p=p, gbar=gbar, xbar=xbar, s=s)))
    return x


def alsncg(P: Problem, x0, iters, alpha0=10.0, tau=0.9, cc=0.5, max_shrinks=200,
           mode="backtrack", keep_x=True):
    """ALS-NCG (Algorithm 2) with P = one ALS sweep and the line search of §V-C.
    Returns the list of IterRecord, one per iteration (after the update)."""
    recs = []
    last_c = {}

    def step(x, p, g):
        c = ls_coeffs(P, x, p)
        last_c["c"] = c
        if mode == "exact":
            return exact_step(c)
        return backtracking(c, alpha0, tau, cc, max_shrinks)

    def on_iter(k, x, g, info):
        if not keep_x:
            info = dict(info, state=None)
        recs.append(IterRecord(k=k + 1, x=x.copy() if keep_x else None, f=loss(P, x),
                               gnorm=float(np.linalg.norm(g)), c=last_c.get("c"),
                               g=g.copy() if keep_x else None, **info))

    ncg(x0, lambda x: grad(P, x), lambda x: sweep(P, x), step, iters, on_iter)
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
