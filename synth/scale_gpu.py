"""Seeded synthetic ratings generated on the GPU, for the scaling sweep
(1e7 .. 1e9 ratings), where generating on the host would take longer than the
runs themselves.  Random numbers and shaping only -- none of the method's
arithmetic lives here.

Recipe (the host generator's, with a GPU sampler):
  * user degrees: Zipf(s) rank weights scaled to nnz, capped at n_m, ids
    permuted (``rank_degrees``, on the host);
  * positions: each user's items drawn with probability proportional to a
    Zipf(s) weight over permuted item ids, by inverse-CDF sampling on the GPU;
    repeated (user, item) pairs are dropped and each user's shortfall is drawn
    again (three rounds); users still short are redrawn exactly by weighted
    sampling without replacement (Gumbel top-k), so every user gets exactly
    its target degree;
  * values: rank-``rank`` truth u* . m* with entries N(0, 1/rank), plus
    N(0, 0.5^2) noise, shifted to mean 3.5, clipped to [0.5, 5], rounded to
    half stars (round half to even).
"""
import numpy as np

from .ratings import rank_degrees

# (n_u, n_m, target ratings) of the scaling steps
SCALE_STEPS = {
    "1e7": (500_000, 50_000, 10_000_000),
    "3e7": (1_000_000, 100_000, 31_600_000),
    "1e8": (2_000_000, 200_000, 100_000_000),
    "3e8": (4_000_000, 500_000, 316_000_000),
    "1e9": (8_000_000, 1_000_000, 1_000_000_000),
}


def make_scale_gpu(n_u, n_m, nnz, seed, s=1.1, rank=10, rounds=3, device="cuda", chunk=1 << 26):
    """Returns (rows int32, cols int32, vals float32) CUDA tensors of distinct
    (user, item) ratings, sorted by user then item."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    deg = rank_degrees(n_u, nnz, 1, n_m, rng, s)
    w = np.arange(1, n_m + 1, dtype=np.float64) ** -s
    w = w[rng.permutation(n_m)]
    cw = torch.tensor(np.cumsum(w) / w.sum(), device=device, dtype=torch.float64)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    users = torch.arange(n_u, device=device, dtype=torch.int64)
    want = torch.tensor(deg, device=device, dtype=torch.int64)

    def draw(counts):
        r = torch.repeat_interleave(users, counts)
        c = torch.empty(r.shape[0], dtype=torch.int64, device=device)
        for a in range(0, r.shape[0], chunk):
            b = min(r.shape[0], a + chunk)
            u = torch.rand(b - a, generator=gen, device=device, dtype=torch.float64)
            c[a:b] = torch.searchsorted(cw, u).clamp_(max=n_m - 1)
        return r * n_m + c

    key = torch.unique(draw(want))
    for _ in range(rounds - 1):
        have = torch.bincount(key // n_m, minlength=n_u)
        short = want - have
        if int(short.sum()) == 0:
            break
        key = torch.unique(torch.cat([key, draw(short.clamp_(min=0))]))
    # users still short (heavy users drawing popular items over and over) are
    # drawn again exactly: weighted sampling without replacement by Gumbel
    # top-k, log w_j - log(-log U_j), the largest d_u scores
    have = torch.bincount(key // n_m, minlength=n_u)
    short = torch.nonzero(have < want).flatten()
    if short.numel() > 0:
        key = key[~torch.isin(key // n_m, short)]
        logw = torch.tensor(np.log(w), device=device, dtype=torch.float64)
        batch = max(1, (1 << 27) // n_m)
        extra = []
        for a in range(0, short.numel(), batch):
            us = short[a:a + batch]
            d = want[us]
            u = torch.rand(us.numel(), n_m, generator=gen, device=device, dtype=torch.float64)
            score = logw - torch.log(-torch.log(u.clamp_(min=1e-300)))
            top = torch.topk(score, int(d.max()), dim=1).indices
            keep = torch.arange(top.shape[1], device=device)[None, :] < d[:, None]
            extra.append((us[:, None] * n_m + top)[keep])
        key = torch.sort(torch.cat([key] + extra)).values
    rows = (key // n_m).to(torch.int32)
    cols = (key % n_m).to(torch.int32)
    del key
    sig = 1.0 / np.sqrt(rank)
    ut = torch.randn(n_u, rank, generator=gen, device=device) * sig
    mt = torch.randn(n_m, rank, generator=gen, device=device) * sig
    vals = torch.empty(rows.shape[0], dtype=torch.float32, device=device)
    total = 0.0
    for a in range(0, rows.shape[0], chunk):
        b = min(rows.shape[0], a + chunk)
        v = (ut[rows[a:b].long()] * mt[cols[a:b].long()]).sum(1)
        v += 0.5 * torch.randn(b - a, generator=gen, device=device)
        vals[a:b] = v
        total += float(v.double().sum())
    vals += 3.5 - total / max(rows.shape[0], 1)
    vals.clamp_(0.5, 5.0)
    vals.mul_(2.0).round_().mul_(0.5)
    return rows, cols, vals
