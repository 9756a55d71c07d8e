"""Top-t ranking accuracy of §IV (the modified Kendall-tau distance of the
serial experiments), written as the paper describes it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A user's ranking lists the items by descending predicted rating u_i . m_j
(FP64 here), ties by ascending item id.  The distance between a reference
ranking p1 and a ranking p2 counts the pairwise swaps needed to bring the
top-t items of p1, one after the other (highest first), to the front of p2:
item a_k moves from its current position to position k, and every position
it passes is one swap.  Normalised: q = 1 - s / s_max with
s_max = (n_m - 1) + ... + (n_m - t) = t (2 n_m - t - 1) / 2, averaged over
the users.
"""
import numpy as np


def ranking(scores) -> np.ndarray:
    """Item ids by descending score, ties by ascending id."""
    scores = np.asarray(scores, np.float64)
    return np.lexsort((np.arange(scores.shape[0]), -scores))


def swaps_to_front(top, p2) -> int:
    """The paper's procedure, step by step: for k = 0 .. t-1, move item
    top[k] from its current position in p2 to position k; the swaps are the
    positions it moves over."""
    cur = list(int(v) for v in p2)
    s = 0
    for k, a in enumerate(int(v) for v in top):
        pos = cur.index(a)
        s += pos - k
        cur.insert(k, cur.pop(pos))
    return s


def s_max(n_m, t) -> float:
    """Largest number of swaps: the lists in opposite order."""
    return t * (2 * n_m - t - 1) / 2.0


def topt(U, M, t) -> np.ndarray:
    """The first t items of every user's ranking (n_u x t)."""
    U = np.asarray(U, np.float64)
    M = np.asarray(M, np.float64)
    return np.stack([ranking(M @ U[i])[:t] for i in range(U.shape[0])]).astype(np.int32)


def rank_accuracy(U, M, top_ref):
    """(mean q, per-user q, per-user s) of the rankings by U, M against the
    reference top-t lists."""
    U = np.asarray(U, np.float64)
    M = np.asarray(M, np.float64)
    top_ref = np.asarray(top_ref)
    t = top_ref.shape[1]
    sm = s_max(M.shape[0], t)
    s = np.array([swaps_to_front(top_ref[i], ranking(M @ U[i])) for i in range(U.shape[0])], np.int64)
    q = 1.0 - s / sm
    return float(q.mean()), q, s
