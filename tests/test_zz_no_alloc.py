"""The allocation-free line-search entry point (for callers that cannot call
cudaMalloc where they need the coefficients: code running under CUDA-graph
capture, frameworks that own all device memory, allocator-free serving loops)
gives the same Q(alpha) coefficients as the context-based entry point, and
the FP64 oracle's.

Every lane grouping of its kernel runs (n_f = 10, 20, 48, 100: 4, 8, 16 and
32 lanes per row), on a problem with rows of thousands of ratings, empty
rows and single-rating rows, twice in a row (the scratch array is shared
and keeps the last call's contents).

Kept in a file of its own, collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _padded(v, rows, n_f, ld, torch, dtype):
    a = np.zeros((rows, ld), np.float64)
    a[:, :n_f] = np.asarray(v, np.float64).reshape(rows, n_f)
    return torch.tensor(a, dtype=dtype, device="cuda")


def _heavy_problem():
    """Users with 1,000-2,400 ratings, an item rated by every user, single-rating
    users, empty items."""
    rng = np.random.default_rng(0)
    n_u, n_m = 300, 2600
    rows, cols = [], []
    for i in range(n_u):
        d = 2300 + 50 * i if i < 3 else 1000 + 37 * i if i < 6 else 1 if i < 12 else int(rng.integers(2, 40))
        c = rng.choice(n_m - 5, size=d, replace=False)
        rows.append(np.full(d, i)); cols.append(c)
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    extra = np.setdiff1d(np.arange(n_u), rows[cols == 7])
    rows = np.concatenate([rows, extra]); cols = np.concatenate([cols, np.full(extra.size, 7)])
    vals = (np.round(2 * np.clip(rng.normal(3.5, 1, rows.size), 0.5, 5)) / 2).astype(np.float32)
    return n_u, n_m, rows.astype(np.int32), cols.astype(np.int32), vals


def _call(lib, _lib, torch, n_u, n_m, n_f, ld, lam, dev, xd, pd, dt):
    stream = torch.cuda.current_stream()
    c = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.als_linesearch_coeffs_static(n_u, n_m, n_f, ld, lam, dev["uptr"].data_ptr(), dev["uidx"].data_ptr(),
                                          dev["uval"].data_ptr(), dev["mptr"].data_ptr(), xd.data_ptr(),
                                          pd.data_ptr(), dt, c.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    _lib.check(st, "als_linesearch_coeffs_static")
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("n_f", [10, 20, 48, 100])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_context_entry_and_oracle(precision, n_f):
    import torch
    from paper_1508_03110_gb300 import ALS, _lib

    lib = _lib.load()
    n_u, n_m, rows_, cols_, vals_ = _heavy_problem()
    lam = 0.05
    ld = (n_f + 3) // 4 * 4
    rows = n_u + n_m
    x0 = synth.init_factors(n_u, n_m, n_f, 11)
    p = np.random.default_rng(3).normal(size=x0.shape[0]) * 0.1
    if precision == "mixed":      # the FP32 buffers hold the FP32-rounded vectors
        x0 = x0.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    with ALS(n_u, n_m, rows_, cols_, vals_, n_f, lam, precision=precision) as m:
        m.set_x(x0)
        ref = m.linesearch_coeffs(p)
        R = m.ratings()
    P = oracle.build_problem(n_u, n_m, n_f, lam, rows_, cols_, vals_)
    cref = oracle.ls_coeffs(P, x0, p)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    dt = _lib.ALS_DT_F64 if precision == "fp64" else _lib.ALS_DT_F32
    dev = {k: torch.tensor(R[k], device="cuda") for k in ("uptr", "uidx", "uval", "mptr")}
    xd = _padded(x0, rows, n_f, ld, torch, tdt)
    pd = _padded(p, rows, n_f, ld, torch, tdt)
    for call in range(2):
        got = _call(lib, _lib, torch, n_u, n_m, n_f, ld, lam, dev, xd, pd, dt)
        # the same per-rating FP64 terms as the context pass, summed in another order
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * abs(ref[0])), (call, got, ref)
        if precision == "fp64":
            # each coefficient within 1e-10 of the oracle's, relative to itself
            assert np.all(np.abs(got - cref) <= 1e-10 * np.abs(cref)), (call, got, cref)
        else:
            # FP32 products of FP32-rounded inputs (one dot product of n_f terms
            # per rating and vector pair): within 1e-5 of each coefficient
            assert np.all(np.abs(got - cref) <= 1e-5 * np.abs(cref)), (call, (got - cref) / cref)


def test_static_entry_rejects_oversized_problems():
    from paper_1508_03110_gb300 import _lib

    lib = _lib.load()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    st = lib.als_linesearch_coeffs_static(200_000, 100_000, 10, 12, 0.05, dummy, dummy, dummy, dummy,
                                          dummy, dummy, _lib.ALS_DT_F64, dummy, None)
    assert st == _lib.ALS_EINVAL
    assert b"262144" in lib.als_last_error()
