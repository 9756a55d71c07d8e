"""Sharded ALS-NCG: the paper's block partitioning and data exchange (§V-A,
§V-B) as a driver over torch.distributed.

Users and items are cut into contiguous blocks, one per rank, balanced by
ratings count (a block boundary lies on a multiple of `grain` rows).  A rank
owns the ratings of its users (by user) and of its items (by item), and its
rows of every vector of Algorithm 2 (x, p, g, gbar, xbar).  Per iteration:

  * line search (§V-C): all-gather the item blocks of x and p (the paper's
    T_m, since n_u >> n_m), per-row Q(alpha) terms of the own users (ratings
    and regulariser) and own items (regulariser), one reduction of five
    scalars, Algorithm 3 on every rank (same scalars, same alpha);
  * P(x) (Algorithm 1 body): all-gather M, solve the own users; all-gather
    the new U, solve the own items;
  * gradient: the own users' rows from the gathered M, the own items' rows
    from the gathered U; one reduction of |g|^2, gbar.g, gbar.(g - g_prev);
  * beta-bar of Eq. (8) and the new direction, locally.

Reductions are fixed-order and independent of the number of ranks: every
per-row FP64 term is summed within fixed row blocks of `grain` rows
(block b = rows [b grain, (b + 1) grain), users then items), the block sums
are gathered and added in block order.  With block boundaries on that grid
the sums -- and so every iterate -- are bit-identical for any number of
ranks.

The per-shard arithmetic is a backend object (`ShardBackend`): the driver
only moves blocks, reduces scalars and runs the scalar steps.  This pool
gives one GPU per run, so no multi-GPU backend is built here; the exchange
and reduction logic is exercised with CPU ranks (gloo) and a backend that
computes each shard's rows on the host.
"""
import numpy as np


def balanced_blocks(deg, world, grain):
    """Cut rows 0 .. n-1 into `world` contiguous blocks of about equal
    weight (ratings + 1 per row), every boundary on a multiple of `grain`
    (except the last, n).  Returns world + 1 boundaries."""
    deg = np.asarray(deg, np.float64)
    n = deg.shape[0]
    w = np.cumsum(deg + 1.0)
    total = w[-1] if n else 0.0
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(w, target))               # first row past the target weight
        i = int(round(i / grain)) * grain
        i = min(max(i, bounds[-1]), n)
        bounds.append(i)
    bounds.append(n)
    return bounds


def block_sums(terms, row0, grain):
    """Sums of per-row terms (rows x k) within the global blocks of `grain`
    rows; the rows start at global row row0 (a multiple of grain).  Each
    block is summed in row order."""
    terms = np.asarray(terms, np.float64)
    n = terms.shape[0]
    if row0 % grain:
        raise ValueError("a shard must start on a block boundary")
    out = []
    for a in range(0, n, grain):
        s = np.zeros(terms.shape[1])
        for i in range(a, min(n, a + grain)):
            s = s + terms[i]
        out.append(s)
    return np.array(out).reshape(-1, terms.shape[1])


class ShardBackend:
    """Per-shard arithmetic of one rank (rows are the rank's own; `F_full`
    is the gathered fixed side).  Every method returns host arrays."""

    def solve(self, side, F_full):                         # Eq. (3) / (4) for the own rows
        raise NotImplementedError

    def grad(self, side, X_own, F_full):                   # own rows of grad f
        raise NotImplementedError

    def q_user_terms(self, XU, PU, XM_full, PM_full):      # own users: 5 Q(alpha) terms per row
        raise NotImplementedError

    def q_item_terms(self, XM, PM):                        # own items: 5 regulariser terms per row
        raise NotImplementedError

    def dots(self, A, B):                                  # per-row dot products of two row blocks
        raise NotImplementedError


class ShardedALSNCG:
    """Algorithm 2 on `world` ranks (see the module docstring).  comm: an
    object with all_gather(array) -> list of arrays, one per rank in rank
    order (e.g. GlooComm).  ls: Algorithm 3 parameters (alpha0, tau, c,
    max_shrinks), the paper's by default; a failed search takes the ALS
    point and restarts the direction, as the single-GPU driver does."""

    def __init__(self, backend, comm, rank, world, n_u, n_m, n_f, lam, ubounds, mbounds, grain,
                 alpha0=10.0, tau=0.9, c=0.5, max_shrinks=200):
        self.be, self.comm, self.rank, self.world = backend, comm, rank, world
        self.n_u, self.n_m, self.n_f, self.lam = n_u, n_m, n_f, lam
        self.ub, self.mb, self.grain = ubounds, mbounds, grain
        self.ls = (alpha0, tau, c, max_shrinks)
        self.u0, self.u1 = ubounds[rank], ubounds[rank + 1]
        self.m0, self.m1 = mbounds[rank], mbounds[rank + 1]
        self.fallbacks = 0

    # -- exchange -----------------------------------------------------------
    def gather_rows(self, own):
        return np.concatenate(self.comm.all_gather(np.ascontiguousarray(own, np.float64)), axis=0)

    def reduce(self, uterms, mterms):
        """Fixed-order totals of per-row terms: own users' and own items'
        rows, summed within global blocks, the blocks added in block order
        (users' blocks, then items')."""
        ub = block_sums(uterms, self.u0, self.grain)
        mb = block_sums(mterms, self.m0, self.grain)
        allu = self.comm.all_gather(ub)
        allm = self.comm.all_gather(mb)
        blocks = [b for part in allu for b in part] + [b for part in allm for b in part]
        tot = np.zeros(np.asarray(uterms).shape[1])
        for b in blocks:
            tot = tot + b
        return tot

    # -- the pieces of Algorithm 2 --------------------------------------------
    def precond(self, XU, XM):
        """P(x): own rows of xbar = (Ubar, Mbar)."""
        Ubar = self.be.solve(0, self.gather_rows(XM))
        Mbar = self.be.solve(1, self.gather_rows(Ubar))
        return Ubar, Mbar

    def gradient(self, XU, XM):
        gU = self.be.grad(0, XU, self.gather_rows(XM))
        gM = self.be.grad(1, XM, self.gather_rows(XU))
        return gU, gM

    def ncg_terms(self, g, gbar, gprev):
        """Per-row |g|^2, gbar.g, gbar.(g - gprev) for both sides."""
        out = []
        for s in range(2):
            d = gprev[s] if gprev is not None else np.zeros_like(g[s])
            out.append(np.stack([self.be.dots(g[s], g[s]), self.be.dots(gbar[s], g[s]),
                                 self.be.dots(gbar[s], g[s] - d)], axis=1))
        return self.reduce(out[0], out[1])

    def q_coeffs(self, X, P):
        ut = self.be.q_user_terms(X[0], P[0], self.gather_rows(X[1]), self.gather_rows(P[1]))
        mt = self.be.q_item_terms(X[1], P[1])
        return self.reduce(ut, mt)

    def step_length(self, c):
        """Algorithm 3 on Q: alpha0, shrink by tau while Q(a) - Q(0) > c a c1
        (difference form); (alpha, ok, shrinks)."""
        alpha0, tau, cc, max_shrinks = self.ls
        if not (c[1] < 0.0):
            return 0.0, False, 0
        a = alpha0
        for k in range(max_shrinks + 1):
            dq = a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])))
            if dq <= a * cc * c[1]:
                return a, True, k
            a *= tau
        return 0.0, False, max_shrinks

    # -- the driver -------------------------------------------------------------
    def run(self, XU, XM, iters, on_iter=None):
        """Algorithm 2 from the own blocks of x_0; returns the own blocks of
        x after `iters` iterations.  on_iter(k, info) gets f, |g|, alpha,
        beta, fallback after each iteration (the same on every rank)."""
        X = [np.array(XU, np.float64), np.array(XM, np.float64)]
        xbar = list(self.precond(*X))
        gbar = [X[s] - xbar[s] for s in range(2)]
        g = list(self.gradient(*X))
        tot = self.ncg_terms(g, gbar, None)
        s_k = tot[1]
        P = [-gbar[0], -gbar[1]]
        for k in range(iters):
            c = self.q_coeffs(X, P)
            alpha, ok, shrinks = self.step_length(c)
            if ok:
                X = [X[s] + alpha * P[s] for s in range(2)]
            else:
                X = [xbar[0].copy(), xbar[1].copy()]
                self.fallbacks += 1
            xbar = list(self.precond(*X))
            gbar_new = [X[s] - xbar[s] for s in range(2)]
            g_new = list(self.gradient(*X))
            tot = self.ncg_terms(g_new, gbar_new, g)
            beta = tot[2] / s_k if (ok and s_k != 0.0) else 0.0
            P = [-gbar_new[s] + beta * P[s] for s in range(2)]
            s_k = tot[1]
            g, gbar = g_new, gbar_new
            if on_iter is not None:
                on_iter(k, dict(gnorm=float(np.sqrt(tot[0])), alpha=alpha, beta=beta, fallback=not ok,
                                shrinks=shrinks, c=c))
        return X[0], X[1]


class GlooComm:
    """all_gather of host arrays over a torch.distributed process group
    (gloo on CPU ranks); arrays may differ in length between ranks."""

    def __init__(self, dist, group=None):
        self.dist, self.group = dist, group

    def all_gather(self, arr):
        import torch
        a = np.ascontiguousarray(arr, np.float64)
        world = self.dist.get_world_size(self.group)
        shape = torch.tensor(list(a.shape) + [0] * (4 - a.ndim) + [a.ndim], dtype=torch.int64)
        shapes = [torch.zeros_like(shape) for _ in range(world)]
        self.dist.all_gather(shapes, shape, group=self.group)
        dims = [tuple(int(v) for v in s[:int(s[4])]) for s in shapes]
        n = max(1, max(int(np.prod(d)) if d else 1 for d in dims))
        buf = torch.zeros(n, dtype=torch.float64)
        flat = torch.from_numpy(a.reshape(-1).copy())
        buf[:flat.numel()] = flat
        outs = [torch.zeros(n, dtype=torch.float64) for _ in range(world)]
        self.dist.all_gather(outs, buf, group=self.group)
        return [o[:int(np.prod(d)) if d else 1].numpy().reshape(d) for o, d in zip(outs, dims)]
