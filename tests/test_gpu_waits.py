"""Failure detection without a GPU fault: the tensor-core sweep's bounded
device waits are made to run out (a self-test launch issues no MMA, so nothing
ever signals the mbarriers), and the library must report ALS_ETIMEOUT, count
one expiry per row that waited, report the recorded expiry once, and run again
once the caller restores a checkpoint or sets new factors (needs a GB300)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _ctx(r, n_f):
    from paper_1508_03110_gb300 import ALS
    return ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc",
               refine_steps=4)


def test_bounded_waits_run_out_and_context_survives():
    from paper_1508_03110_gb300 import ALSError, _lib
    r = synth.make_config("tiny")
    n_f = 48
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3)
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    lib = _lib.load()
    with _ctx(r, n_f) as m:
        m.set_x(x0)
        before = m.get_x()
        n = ctypes.c_int64()
        st = lib.als_selftest_wait_expiry(m.ctx, 0.02, ctypes.byref(n))
        assert st == _lib.ALS_ETIMEOUT
        assert n.value == int((np.bincount(r.rows, minlength=r.n_u) > 0).sum())
        assert np.array_equal(m.get_x(), before)          # only scratch was written
        # the expiry stays recorded: the next call that returns host values
        # reports it once, and it is then cleared
        with pytest.raises(ALSError, match="ETIMEOUT"):
            m.loss()
        assert np.isfinite(m.loss())
        m.sweep(1)                                        # the context still works
        x = m.get_x()
        info = m.step()
    ref = oracle.sweep(P, x0)
    assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.isfinite(info["f"]) and info["notspd"] == 0


def test_expiry_during_iterations_then_restore_checkpoint():
    """An expiry recorded while ALS-NCG runs: the next iteration reports
    ALS_ETIMEOUT; restoring the checkpoint taken before it (als_set_state)
    makes the context run again, and the resumed iterations are bit-identical
    to an uninterrupted run."""
    from paper_1508_03110_gb300 import ALSError, _lib
    r = synth.make_config("tiny")
    n_f = 48
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 4)
    lib = _lib.load()
    with _ctx(r, n_f) as ref:
        ref.set_x(x0)
        for _ in range(4):
            ref.step(info=False)
        x_ref = ref.get_x()
        f_ref = ref.step()["f"]
    with _ctx(r, n_f) as m:
        m.set_x(x0)
        for _ in range(2):
            m.step(info=False)
        st = m.get_state()
        assert lib.als_selftest_wait_expiry(m.ctx, 0.02, None) == _lib.ALS_ETIMEOUT
        with pytest.raises(ALSError, match="ETIMEOUT"):
            m.step()
        m.set_state(st["x"], st["p"], st["g"], st["gbar"], st["xbar"], st["s"], st["gg0"], st["k"],
                    st["fallbacks"])
        for _ in range(2):
            m.step(info=False)
        assert np.array_equal(m.get_x(), x_ref)
        assert m.step()["f"] == f_ref


def test_wait_selftest_needs_the_tensor_core_path():
    from paper_1508_03110_gb300 import ALS, _lib
    r = synth.make_config("tiny")
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, r.n_f, r.lam) as m:
        assert _lib.load().als_selftest_wait_expiry(m.ctx, 0.02, None) == _lib.ALS_ENOTSUP
