"""Synthetic ratings shaped like the paper's workloads (MovieLens-20M-like
sizes and skew; the dataset itself is not used or reproduced).

Recipe (all draws from numpy PCG64 with the stated seed):
  * degrees: either Zipf rank weights r**-s scaled to nnz, floored at d_min
    and capped at d_max with the surplus redistributed, or (when only the
    range and the mean are given) the midpoint quantiles of a power law
    truncated to [d_min, d_max] whose exponent is solved so that the degrees
    sum to nnz; rounded with the largest-remainder rule, then assigned to ids
    through a random permutation (id is not correlated with degree);
  * item weights: the same two shapes; realised item degrees follow them;
  * positions: each user draws its d_i distinct items with probability
    proportional to the item weights (weighted sampling without replacement,
    done as successive draws with duplicates discarded);
  * values: a rank-k ground truth u*.m* with u*, m* ~ N(0, sigma^2),
    sigma = 1/sqrt(k), plus N(0, 0.5^2) noise, shifted to mean 3.5, clipped to
    [0.5, 5] and rounded to half stars (round-half-even of 2r, then /2).
"""
import dataclasses

import numpy as np


@dataclasses.dataclass
class Ratings:
    name: str
    n_u: int
    n_m: int
    rows: np.ndarray   # int32 user ids
    cols: np.ndarray   # int32 item ids
    vals: np.ndarray   # float32 half-star ratings
    n_f: int
    lam: float

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])


def _pareto_quantiles(n, total, d_min, d_max):
    """Deterministic quantiles of a power law p(d) ~ d^-a truncated to
    [d_min, d_max], at the midpoints (r - 1/2)/n, with the exponent a found by
    bisection so that they sum to ``total``.  Returned in descending order."""
    q = (np.arange(n, dtype=np.float64) + 0.5) / n
    L, H = float(d_min), float(d_max)

    def quant(a):
        if abs(a - 1.0) < 1e-9:
            return L * (H / L) ** q
        b = 1.0 - a
        return (L ** b + q * (H ** b - L ** b)) ** (1.0 / b)

    lo, hi = -6.0, 8.0   # larger a -> more mass near d_min -> smaller sum
    for _ in range(200):
        a = 0.5 * (lo + hi)
        if quant(a).sum() > total:
            lo = a
        else:
            hi = a
    return quant(0.5 * (lo + hi))[::-1].copy()


def rank_degrees(n, total, d_min, d_max, rng, s=None):
    """Integer degrees in [d_min, d_max] summing to ``total``, power law in rank
    (exponent ``s`` if given, else solved), assigned to ids at random."""
    total = int(total)
    if total < n * d_min or total > n * d_max:
        raise ValueError("total outside [n*d_min, n*d_max]")
    r = np.arange(1, n + 1, dtype=np.float64)
    if s is None:
        w = _pareto_quantiles(n, total, d_min, d_max)
    else:
        # Zipf rank weights scaled to the total, floored/capped, surplus
        # redistributed over the entries that are still free.
        w = r ** -s
        w = w * total / w.sum()
        for _ in range(100):
            w = np.clip(w, d_min, d_max)
            free = (w > d_min) & (w < d_max)
            gap = total - w.sum()
            if abs(gap) < 0.5 or not free.any():
                break
            w[free] += gap * w[free] / w[free].sum()
    base = np.floor(w).astype(np.int64)
    base = np.clip(base, d_min, d_max)
    rem = total - int(base.sum())
    frac = w - np.floor(w)
    order = np.argsort(-frac, kind="stable")
    if rem > 0:
        cand = order[base[order] < d_max]
        base[cand[:rem]] += 1
    elif rem < 0:
        cand = order[::-1]
        cand = cand[base[cand] > d_min]
        base[cand[:-rem]] -= 1
    if int(base.sum()) != total:
        raise RuntimeError("degree rounding failed")
    perm = rng.permutation(n)
    out = np.empty(n, np.int64)
    out[perm] = base
    return out


def sample_distinct(deg, weights, rng, draw_rounds=3):
    """For each user i, deg[i] distinct items drawn with probability
    proportional to ``weights`` without replacement.  A few rounds of
    successive draws with duplicates discarded serve most users; users that
    still miss items then take them by exponential keys (Efraimidis and
    Spirakis, 2006) among the items they do not have yet, which continues the
    same successive-sampling distribution.  Returns (rows, cols) grouped by row."""
    deg = np.asarray(deg, np.int64)
    n_u, n_m = deg.shape[0], weights.shape[0]
    if deg.max(initial=0) > n_m:
        raise ValueError("degree larger than the number of items")
    w = np.asarray(weights, np.float64)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    done_u, done_i = [], []
    pu = np.zeros(0, np.int64); pi = np.zeros(0, np.int64); ps = np.zeros(0, np.int64)
    have = np.zeros(n_u, np.int64)
    seq0 = 0
    users = np.nonzero(deg > 0)[0]
    for rnd in range(draw_rounds):
        if users.size == 0:
            break
        k = np.ceil((deg[users] - have[users]) * (1.25 * 2.0 ** rnd)).astype(np.int64) + 8
        u = np.repeat(users, k)
        it = np.minimum(np.searchsorted(cdf, rng.random(u.shape[0]), side="right"), n_m - 1)
        s = seq0 + np.arange(u.shape[0], dtype=np.int64)
        seq0 += u.shape[0]
        U = np.concatenate([pu, u]); I = np.concatenate([pi, it]); S = np.concatenate([ps, s])
        o = np.lexsort((S, U * n_m + I))          # first occurrence of each (user, item)
        key_o = (U * n_m + I)[o]
        first = np.ones(o.shape[0], bool)
        first[1:] = key_o[1:] != key_o[:-1]
        o = o[first]
        U, I, S = U[o], I[o], S[o]
        o = np.lexsort((S, U))                    # per user, in draw order
        U, I, S = U[o], I[o], S[o]
        start = np.zeros(n_u + 1, np.int64)
        np.cumsum(np.bincount(U, minlength=n_u), out=start[1:])
        keep = (np.arange(U.shape[0], dtype=np.int64) - start[U]) < deg[U]
        U, I, S = U[keep], I[keep], S[keep]
        cnt = np.bincount(U, minlength=n_u)
        have[users] = cnt[users]
        full = have[U] == deg[U]
        done_u.append(U[full]); done_i.append(I[full])
        pu, pi, ps = U[~full], I[~full], S[~full]
        users = np.nonzero(have < deg)[0]
    if users.size:
        start = np.zeros(n_u + 1, np.int64)
        np.cumsum(np.bincount(pu, minlength=n_u), out=start[1:])
        for user in users:
            mine = pi[start[user]:start[user + 1]]
            avail = np.ones(n_m, bool)
            avail[mine] = False
            cand = np.nonzero(avail & (w > 0))[0]
            need = int(deg[user] - mine.shape[0])
            keys = np.log(rng.random(cand.shape[0])) / w[cand]
            pick = cand[np.argsort(-keys, kind="stable")[:need]]
            done_u.append(np.full(mine.shape[0] + need, user, np.int64))
            done_i.append(np.concatenate([mine, pick]))
    rows = np.concatenate(done_u) if done_u else np.zeros(0, np.int64)
    cols = np.concatenate(done_i) if done_i else np.zeros(0, np.int64)
    o = np.argsort(rows, kind="stable")
    return rows[o].astype(np.int32), cols[o].astype(np.int32)


def half_star_values(rows, cols, n_u, n_m, rank, rng, noise=0.5, mean=3.5, chunk=1 << 22):
    """Rank-``rank`` ground truth plus Gaussian noise, shifted to ``mean``,
    clipped to [0.5, 5] and rounded to half stars."""
    sig = 1.0 / np.sqrt(rank)
    Ut = rng.normal(0.0, sig, size=(n_u, rank))
    Mt = rng.normal(0.0, sig, size=(n_m, rank))
    r = np.empty(rows.shape[0], np.float64)
    for a in range(0, rows.shape[0], chunk):
        b = min(rows.shape[0], a + chunk)
        r[a:b] = np.einsum("ij,ij->i", Ut[rows[a:b]], Mt[cols[a:b]])
    r += rng.normal(0.0, noise, size=r.shape[0])
    r += mean - r.mean()
    r = np.clip(r, 0.5, 5.0)
    return (np.round(2.0 * r) / 2.0).astype(np.float32)


def make_ratings(name, n_u, n_m, nnz, user_deg, item_w, rank, n_f, lam, seed):
    """user_deg: (d_min, d_max, s or None); item_w: (w_min, w_max, s or None)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    deg = rank_degrees(n_u, nnz, user_deg[0], min(user_deg[1], n_m), rng, user_deg[2])
    r = np.arange(1, n_m + 1, dtype=np.float64)
    if item_w[2] is None:
        w = _pareto_quantiles(n_m, nnz, item_w[0], item_w[1])
    else:
        w = np.clip(item_w[1] * r ** -item_w[2], item_w[0], item_w[1])
    w = w[rng.permutation(n_m)]
    rows, cols = sample_distinct(deg, w, rng)
    vals = half_star_values(rows, cols, n_u, n_m, rank, rng)
    return Ratings(name, n_u, n_m, rows, cols, vals, n_f, lam)


# Workload shapes (sizes, skew, model) -------------------------------------
CONFIGS = {
    # FP64 parity case: 2,000 x 1,000, 1e5 ratings, user degrees Zipf(1.2)
    # floored at 5, item popularity Zipf(1.0); rank-10 truth; n_f 10.
    "tiny": dict(n_u=2000, n_m=1000, nnz=100_000, user_deg=(5, 1000, 1.2),
                 item_w=(1e-9, 1.0, 1.0), rank=10, n_f=10, lam=0.05, seed=1),
    # MovieLens-20M-shaped: 138,493 x 26,744, 2e7 ratings, user degrees power
    # law in [20, 9000] (mean 144.4), item weights power law in [1, 67000];
    # rank-20 truth; n_f 100.
    "ml20m": dict(n_u=138_493, n_m=26_744, nnz=20_000_000, user_deg=(20, 9000, None),
                  item_w=(1.0, 67000.0, None), rank=20, n_f=100, lam=0.05, seed=2),
    # Scaling sweep, first two steps (Zipf(1.1) on both sides, rank-10 truth).
    "scale1e7": dict(n_u=500_000, n_m=50_000, nnz=10_000_000, user_deg=(1, 50_000, 1.1),
                     item_w=(1e-9, 1.0, 1.1), rank=10, n_f=10, lam=0.05, seed=30),
    "scale3e7": dict(n_u=1_000_000, n_m=100_000, nnz=31_600_000, user_deg=(1, 100_000, 1.1),
                     item_w=(1e-9, 1.0, 1.1), rank=10, n_f=50, lam=0.05, seed=31),
}


def make_config(name, **over):
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    return make_ratings(name, cfg["n_u"], cfg["n_m"], cfg["nnz"], cfg["user_deg"], cfg["item_w"],
                        cfg["rank"], cfg["n_f"], cfg["lam"], cfg["seed"])


def make_batch(n_prob, nnz_lo, nnz_hi, dens_lo, dens_hi, seed, rank=10):
    """Independent problems of uneven size: ratings log-uniform in [nnz_lo,
    nnz_hi], density uniform in [dens_lo, dens_hi], 2-8 users per item, Zipf
    degrees (users 1.1, items 1.0), half-star values.  Returns a list of
    (n_u, n_m, rows, cols, vals) with ids local to each problem."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for _ in range(n_prob):
        nnz = int(np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi))))
        dens = rng.uniform(dens_lo, dens_hi)
        ratio = rng.uniform(2.0, 8.0)
        cells = nnz / dens
        n_m = max(4, int(np.sqrt(cells / ratio)))
        n_u = max(4, int(cells / n_m))
        nnz = max(n_u, min(nnz, n_u * n_m // 2))
        deg = rank_degrees(n_u, nnz, 1, n_m, rng, 1.1)
        w = np.arange(1, n_m + 1, dtype=np.float64) ** -1.0
        w = w[rng.permutation(n_m)]
        rows, cols = sample_distinct(deg, w, rng)
        vals = half_star_values(rows, cols, n_u, n_m, rank, rng)
        probs.append((n_u, n_m, rows, cols, vals))
    return probs


C4_NF = (10, 20, 50, 100)


def c4_problems(n_prob=64, nnz_lo=10_000, nnz_hi=10_000_000, seed=4):
    """The batched-uneven workload: n_prob independent problems, ratings
    log-uniform in [nnz_lo, nnz_hi], density in 0.1-5%, n_f assigned round
    robin over C4_NF.  Returns (problems, n_fs)."""
    probs = make_batch(n_prob, nnz_lo, nnz_hi, 0.001, 0.05, seed)
    return probs, [C4_NF[q % len(C4_NF)] for q in range(n_prob)]


def init_factors(n_u, n_m, n_f, seed):
    """x_0 (Eq. 5 layout, n_u rows then n_m rows of n_f): i.i.d. N(0, 1/n_f)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, 1.0 / np.sqrt(n_f), size=(n_u + n_m) * n_f)


def make_dense(n_u, n_m, rank, seed, noise=0.1):
    """A fully observed ratings matrix (every user rates every item)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.normal(size=(n_u, rank)); B = rng.normal(size=(rank, n_m))
    R = A @ B + noise * rng.normal(size=(n_u, n_m)) + 3.0
    rows, cols = np.meshgrid(np.arange(n_u), np.arange(n_m), indexing="ij")
    return rows.reshape(-1).astype(np.int32), cols.reshape(-1).astype(np.int32), R.reshape(-1)


def foldin_requests(n_req, n_m, d_min, d_max, seed, item_s=1.0):
    """New-user requests: log-uniform degree in [d_min, d_max], Zipf items,
    half-star values.  Returns (req_ptr int64, items int32, vals float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    deg = np.floor(np.exp(rng.uniform(np.log(d_min), np.log(d_max + 1), size=n_req))).astype(np.int64)
    deg = np.clip(deg, d_min, min(d_max, n_m))
    w = np.arange(1, n_m + 1, dtype=np.float64) ** -item_s
    w = w[rng.permutation(n_m)]
    rows, cols = sample_distinct(deg, w, rng)
    vals = (np.round(2.0 * np.clip(rng.normal(3.5, 1.0, size=rows.shape[0]), 0.5, 5.0)) / 2.0)
    ptr = np.zeros(n_req + 1, np.int64)
    np.cumsum(deg, out=ptr[1:])
    return ptr, cols.astype(np.int32), vals.astype(np.float32)


# Serial-experiment shapes (the paper's Tables 1-4 ran on MovieLens-20M
# subsets of median users and median movies; these synthetic stand-ins have
# the same shapes, a uniform 5% density and rank-10 half-star values)
TABLE_SHAPES = ((400, 80), (800, 160), (1600, 320), (3200, 640))
TABLE_DENSITY = 0.05


def table_problem(n_u, n_m, seed, density=TABLE_DENSITY, rank=10):
    """Each (user, item) pair is rated with probability `density`; a user or
    item left without ratings gets one at a uniform random partner.  Values:
    rank-`rank` truth plus N(0, 0.5^2) noise, mean 3.5, half stars.  Returns
    (rows, cols, vals)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = rng.random((n_u, n_m)) < density
    for i in np.nonzero(~mask.any(axis=1))[0]:
        mask[i, rng.integers(n_m)] = True
    for j in np.nonzero(~mask.any(axis=0))[0]:
        mask[rng.integers(n_u), j] = True
    rows, cols = np.nonzero(mask)
    vals = half_star_values(rows, cols, n_u, n_m, rank, rng)
    return rows.astype(np.int32), cols.astype(np.int32), vals
