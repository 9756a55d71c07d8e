"""Failure detection without a GPU fault: the tensor-core sweep's bounded
device waits are made to run out (a self-test launch issues no MMA, so nothing
ever signals the mbarriers), and the library must report ALS_ETIMEOUT, count
one expiry per row that waited, and leave the context usable (needs a GB300)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_bounded_waits_run_out_and_context_survives():
    from paper_1508_03110_gb300 import ALS, _lib
    r = synth.make_config("tiny")
    n_f = 48
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3)
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    lib = _lib.load()
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc",
             refine_steps=4) as m:
        m.set_x(x0)
        before = m.get_x()
        n = ctypes.c_int64()
        st = lib.als_selftest_wait_expiry(m.ctx, 0.02, ctypes.byref(n))
        assert st == _lib.ALS_ETIMEOUT
        assert n.value == int((np.bincount(r.rows, minlength=r.n_u) > 0).sum())
        assert np.array_equal(m.get_x(), before)          # only scratch was written
        m.sweep(1)                                        # the context still works
        x = m.get_x()
        info = m.step()
    ref = oracle.sweep(P, x0)
    assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.isfinite(info["f"]) and info["notspd"] == 0


def test_wait_selftest_needs_the_tensor_core_path():
    from paper_1508_03110_gb300 import ALS, _lib
    r = synth.make_config("tiny")
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, r.n_f, r.lam) as m:
        assert _lib.load().als_selftest_wait_expiry(m.ctx, 0.02, None) == _lib.ALS_ENOTSUP
