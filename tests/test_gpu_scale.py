"""Scaling-sweep inputs (Zipf(1.1) on both sides, generated on the GPU) at
1e8 ratings (2e6 users x 2e5 items): the sweep's rows against the oracle's
exact solves of sampled rows -- the heaviest, the lightest and a random set
-- each from that row's own ratings and the same fixed factors (needs a
GB300).  Tolerances as in the full-size ML20M-shaped test: FP64 1e-10 per
row; mixed, from a random start, each row within 1e-6 of its step plus the
FP32 floor 4 kappa(A_i) 2^-24 |u*| (the heaviest item rows, up to 1.2e6
ratings, are split across CTAs and their partial Gram matrices added in
FP64; measured: at most 1e-7 of the step), and f within 1e-5 of the FP64 run
at equal iteration count."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N_U, N_M, NNZ = synth.SCALE_STEPS["1e8"]


@pytest.fixture(scope="module")
def data():
    import torch
    rows, cols, vals = synth.make_scale_gpu(N_U, N_M, NNZ, seed=32)
    du = torch.bincount(rows.long(), minlength=N_U)
    dm = torch.bincount(cols.long(), minlength=N_M)
    rng = np.random.default_rng(5)
    def pick(d):
        o = torch.argsort(d, descending=True).cpu().numpy()
        nz = o[d.cpu().numpy()[o] > 0]
        return np.unique(np.concatenate([nz[:4], nz[-4:], rng.choice(nz, 8, replace=False)]))
    return rows, cols, vals, pick(du), pick(dm)


def _sub(rows, cols, vals, sel, by_user):
    """Ratings of the selected users (or items), with local ids for them."""
    import torch
    key = rows if by_user else cols
    s = torch.tensor(sel, device=key.device, dtype=torch.int32)
    mask = torch.isin(key, s)
    r, c, v = rows[mask].cpu().numpy(), cols[mask].cpu().numpy(), vals[mask].cpu().numpy()
    loc = {int(x): q for q, x in enumerate(sel)}
    if by_user:
        return np.array([loc[int(x)] for x in r], np.int32), c, v
    return r, np.array([loc[int(x)] for x in c], np.int32), v


def _row_rel(a, b, scale=None):
    s = b if scale is None else scale
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(s, axis=1), 1e-300)))


def _kappas(P, side, F, rows):
    ptr, idx = (P.uptr, P.uidx) if side == 0 else (P.mptr, P.midx)
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        Fi = F[idx[ptr[i]:ptr[i + 1]]]
        w = np.linalg.eigvalsh(Fi.T @ Fi + P.lam * (ptr[i + 1] - ptr[i]) * np.eye(F.shape[1]))
        out[t] = w[-1] / max(w[0], 1e-300)
    return out


def _excess(u, ustar, u0, kap, lead=1e-6, C=4.0):
    err = np.linalg.norm(u - ustar, axis=1)
    bound = lead * np.linalg.norm(ustar - u0, axis=1) + C * kap * 2.0 ** -24 * np.linalg.norm(ustar, axis=1)
    return float(np.max(np.where(err == 0.0, 0.0, err / np.maximum(bound, 1e-300))))


@pytest.mark.parametrize("n_f,precision", [(10, "fp64"), (50, "mixed")])
def test_scale_sweep_sampled_rows(data, n_f, precision):
    from paper_1508_03110_gb300 import ALS
    rows, cols, vals, su, sm = data
    lam = 0.05
    x0 = synth.init_factors(N_U, N_M, n_f, 33)
    if precision == "mixed":
        x0 = x0.astype(np.float32).astype(np.float64)
    with ALS(N_U, N_M, rows, cols, vals, n_f, lam, precision=precision) as m:
        m.set_x(x0)
        m.sweep(1)
        x1 = m.get_x()
    U0 = x0[: N_U * n_f].reshape(N_U, n_f)
    M0 = x0[N_U * n_f:].reshape(N_M, n_f)
    U1 = x1[: N_U * n_f].reshape(N_U, n_f)
    M1 = x1[N_U * n_f:].reshape(N_M, n_f)
    r, c, v = _sub(rows, cols, vals, su, True)
    Pu = oracle.build_problem(len(su), N_M, n_f, lam, r, c, v.astype(np.float64))
    ref_u = oracle.solve_rows(Pu, 0, M0.reshape(-1), np.arange(len(su))).reshape(-1, n_f)
    r, c, v = _sub(rows, cols, vals, sm, False)
    Pm = oracle.build_problem(N_U, len(sm), n_f, lam, r, c, v.astype(np.float64))
    U1x = U1 if precision == "fp64" else U1.astype(np.float32).astype(np.float64)
    ref_m = oracle.solve_rows(Pm, 1, U1x.reshape(-1), np.arange(len(sm))).reshape(-1, n_f)
    if precision == "fp64":
        assert _row_rel(U1[su], ref_u) < 1e-10
        assert _row_rel(M1[sm], ref_m) < 1e-10
    else:
        assert _excess(U1[su], ref_u, U0[su], _kappas(Pu, 0, M0, np.arange(len(su)))) < 1.0
        assert _excess(M1[sm], ref_m, M0[sm], _kappas(Pm, 1, U1x, np.arange(len(sm)))) < 1.0


def test_scale_mixed_f_matches_fp64(data):
    from paper_1508_03110_gb300 import ALS
    rows, cols, vals, _, _ = data
    n_f = 50
    x0 = synth.init_factors(N_U, N_M, n_f, 34)
    fs = {}
    for prec in ("fp64", "mixed"):
        with ALS(N_U, N_M, rows, cols, vals, n_f, 0.05, precision=prec) as m:
            m.set_x(x0)
            fs[prec] = np.array([m.step()["f"] for _ in range(3)])
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"])), fs
