"""The allocation-free line-search entry point (for callers that cannot call
cudaMalloc where they need the coefficients: code running under CUDA-graph
capture, frameworks that own all device memory, allocator-free serving loops)
gives the same Q(alpha) coefficients as the context-based entry point.

Kept in a file of its own, collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _padded(v, rows, n_f, ld, torch, dtype):
    a = np.zeros((rows, ld), np.float64)
    a[:, :n_f] = np.asarray(v, np.float64).reshape(rows, n_f)
    return torch.tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_context_entry(precision):
    import torch
    from paper_1508_03110_gb300 import ALS, _lib

    lib = _lib.load()
    r = synth.make_config("tiny")
    n_f = r.n_f
    ld = (n_f + 3) // 4 * 4
    rows = r.n_u + r.n_m
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 11)
    p = np.random.default_rng(3).normal(size=x0.shape[0]) * 0.1
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision=precision) as m:
        m.set_x(x0)
        ref = m.linesearch_coeffs(p)
        R = m.ratings()
    tdt = torch.float64 if precision == "fp64" else torch.float32
    dt = _lib.ALS_DT_F64 if precision == "fp64" else _lib.ALS_DT_F32
    uptr = torch.tensor(R["uptr"], device="cuda")
    uidx = torch.tensor(R["uidx"], device="cuda")
    uval = torch.tensor(R["uval"], device="cuda")
    mptr = torch.tensor(R["mptr"], device="cuda")
    xd = _padded(x0, rows, n_f, ld, torch, tdt)
    pd = _padded(p, rows, n_f, ld, torch, tdt)
    stream = torch.cuda.current_stream()
    for call in range(2):
        c = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.als_linesearch_coeffs_static(r.n_u, r.n_m, n_f, ld, r.lam, uptr.data_ptr(), uidx.data_ptr(),
                                              uval.data_ptr(), mptr.data_ptr(), xd.data_ptr(), pd.data_ptr(),
                                              dt, c.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        _lib.check(st, "als_linesearch_coeffs_static")
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * abs(ref[0])), (call, got, ref)


def test_static_entry_rejects_oversized_problems():
    from paper_1508_03110_gb300 import _lib

    lib = _lib.load()
    dummy = ctypes.c_void_p(16)
    st = lib.als_linesearch_coeffs_static(200_000, 100_000, 10, 12, 0.05, dummy, dummy, dummy, dummy,
                                          dummy, dummy, _lib.ALS_DT_F64, dummy, None)
    assert st == _lib.ALS_EINVAL
    assert b"262144" in lib.als_last_error()
