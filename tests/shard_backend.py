"""A host backend of the sharded driver for CPU-rank tests: each rank's rows
computed by the FP64 oracle from that rank's own ratings and the gathered
fixed side.  Test infrastructure (imports the oracle)."""
import numpy as np

import oracle
from paper_1508_03110_gb300.sharded import ShardBackend


class OracleShard(ShardBackend):
    def __init__(self, n_u, n_m, n_f, lam, rows, cols, vals, ub, mb, rank):
        rows, cols, vals = np.asarray(rows), np.asarray(cols), np.asarray(vals, np.float64)
        self.n_u, self.n_m, self.n_f, self.lam = n_u, n_m, n_f, lam
        self.u0, self.u1 = ub[rank], ub[rank + 1]
        self.m0, self.m1 = mb[rank], mb[rank + 1]
        su = (rows >= self.u0) & (rows < self.u1)       # the own users' ratings (by user)
        sm = (cols >= self.m0) & (cols < self.m1)       # the own items' ratings (by item)
        self.Pu = oracle.build_problem(self.u1 - self.u0, n_m, n_f, lam, rows[su] - self.u0, cols[su], vals[su])
        self.Pm = oracle.build_problem(n_u, self.m1 - self.m0, n_f, lam, rows[sm], cols[sm] - self.m0, vals[sm])
        self.mdeg = np.bincount(cols, minlength=n_m)[self.m0:self.m1].astype(np.float64)

    def solve(self, side, F_full):
        if side == 0:
            return oracle.half_sweep(self.Pu, 0, F_full).reshape(-1, self.n_f)
        return oracle.half_sweep(self.Pm, 1, F_full).reshape(-1, self.n_f)

    def grad(self, side, X_own, F_full):
        if side == 0:
            x = np.concatenate([np.reshape(X_own, -1), np.reshape(F_full, -1)])
            return oracle.grad(self.Pu, x)[: (self.u1 - self.u0) * self.n_f].reshape(-1, self.n_f)
        x = np.concatenate([np.reshape(F_full, -1), np.reshape(X_own, -1)])
        return oracle.grad(self.Pm, x)[self.n_u * self.n_f:].reshape(-1, self.n_f)

    def q_user_terms(self, XU, PU, XM_full, PM_full):
        """Per own user: its ratings' parts of c0..c4 of Q (§V-C) and its
        regulariser lambda n_i |x_i + alpha p_i|^2."""
        P = self.Pu
        out = np.zeros((self.u1 - self.u0, 5))
        for i in range(self.u1 - self.u0):
            a, b = P.uptr[i], P.uptr[i + 1]
            j = P.uidx[a:b]
            e0 = P.uval[a:b] - XM_full[j] @ XU[i]
            al = XM_full[j] @ PU[i] + PM_full[j] @ XU[i]
            be = PM_full[j] @ PU[i]
            n = b - a
            out[i] = [np.sum(e0 * e0) + self.lam * n * (XU[i] @ XU[i]),
                      np.sum(-2.0 * e0 * al) + self.lam * n * 2.0 * (XU[i] @ PU[i]),
                      np.sum(al * al - 2.0 * e0 * be) + self.lam * n * (PU[i] @ PU[i]),
                      np.sum(2.0 * al * be), np.sum(be * be)]
        return out

    def q_item_terms(self, XM, PM):
        d = self.mdeg
        out = np.zeros((XM.shape[0], 5))
        out[:, 0] = self.lam * d * np.einsum("ij,ij->i", XM, XM)
        out[:, 1] = self.lam * d * 2.0 * np.einsum("ij,ij->i", XM, PM)
        out[:, 2] = self.lam * d * np.einsum("ij,ij->i", PM, PM)
        return out

    def dots(self, A, B):
        return np.einsum("ij,ij->i", A, B)
