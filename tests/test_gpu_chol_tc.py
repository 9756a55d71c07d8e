"""The Cholesky factorisation of the tensor-core sweep in TMEM (launch shape
chol_tc = 1, needs a GB300): the Gram matrix stays in TMEM, each panel of 16
columns is factored on the CUDA cores and the trailing update D -= L21 L21^T
runs as tcgen05 MMAs of the split-BF16 panel.  The factor only
preconditions the refinement against the FP32 residual, so the rows must meet
the same per-row bounds as the shared-memory factorisation's, against the
FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import _half_sweeps_vs_oracle, _mixed_row_excess, _row_rel

pytestmark = pytest.mark.gpu


def _als(r, n_f, **kw):
    from paper_1508_03110_gb300 import ALS
    return ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc", **kw)


@pytest.fixture(scope="module")
def tiny():
    return synth.make_config("tiny")


@pytest.mark.parametrize("n_f", [10, 40, 100, 128])
def test_chol_tc_sweep_rows_meet_the_refinement_bound(tiny, n_f):
    """One sweep at the default refine_steps: every row within 1e-6 of its
    step plus the FP32 floor (n_f = 10: one panel and no MMA; 40 and 100: a
    ragged last panel; 128: all of TMEM's 128 lanes)."""
    r = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 7).astype(np.float32).astype(np.float64)
    with _als(r, n_f) as m:
        m.set_launch(chol_tc=1, dual_max=0)
        assert m.get_launch()["chol_tc"] == 1
        m.set_x(x0)
        m.sweep(1)
        x1 = m.get_x()
    U1, Us, U0, ku, M1, Ms, M0, km = _half_sweeps_vs_oracle(r, P, x0, x1, n_f)
    assert _mixed_row_excess(U1, Us, U0, ku, 1e-6) < 1.0
    assert _mixed_row_excess(M1, Ms, M0, km, 1e-6) < 1.0


@pytest.mark.parametrize("n_f", [48, 100])
def test_chol_tc_one_correction(tiny, n_f):
    """One correction only: what is left is rho |step| with rho = |I -
    Ahat^-1 A|.  The split-BF16 Gram contributes about kappa 2^-17 and the
    split-BF16 trailing updates about as much again, so rho <= kappa 2^-16."""
    r = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3).astype(np.float32).astype(np.float64)
    with _als(r, n_f, refine_steps=1) as m:
        m.set_launch(chol_tc=1, dual_max=0)
        m.set_x(x0)
        m.sweep(1)
        x1 = m.get_x()
    U1, Us, U0, ku, M1, Ms, M0, km = _half_sweeps_vs_oracle(r, P, x0, x1, n_f)
    assert _mixed_row_excess(U1, Us, U0, ku, ku * 2.0 ** -16) < 1.0
    assert _mixed_row_excess(M1, Ms, M0, km, km * 2.0 ** -16) < 1.0


@pytest.mark.parametrize("n_f", [48, 100, 128])
def test_chol_tc_converges_to_the_oracle(tiny, n_f):
    """With four corrections both factorisations reach the FP64 oracle's
    sweep to 1e-6 per row."""
    r = tiny
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3).astype(np.float32).astype(np.float64)
    ref = oracle.sweep(P, x0)
    for ct in (0, 1):
        with _als(r, n_f, refine_steps=4) as m:
            m.set_launch(chol_tc=ct)
            m.set_x(x0)
            m.sweep(1)
            assert _row_rel(m.get_x(), ref, n_f) < 1e-6, ct


def test_chol_tc_alsncg_matches_fp64(tiny):
    """Ten mixed ALS-NCG iterations with the TMEM factorisation: f within 1e-5
    of the FP64 run's at every iteration."""
    from paper_1508_03110_gb300 import ALS
    r = tiny
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 9)
    fs = {}
    for prec in ("fp64", "mixed"):
        with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision=prec) as m:
            if prec == "mixed":
                m.set_launch(chol_tc=1)
            m.set_x(x0)
            fs[prec] = np.array([m.step()["f"] for _ in range(10)])
    assert np.all(np.abs(fs["mixed"] - fs["fp64"]) <= 1e-5 * np.abs(fs["fp64"]))


def test_chol_tc_fullsize_matches_shared_memory_cholesky():
    """ML20M size, the benchmark's launch shapes: two ALS-NCG iterations with
    either factorisation give f within 1e-6 and no factorisation failure."""
    r = synth.make_config("ml20m")
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    fs = {}
    for ct in (0, 1):
        with _als(r, r.n_f) as m:
            m.set_launch(heavy_min=1024, grid_mult=64, split_min=65536, seg_len=4096, dual_max=64, chol_tc=ct)
            m.set_x(x0)
            infos = [m.step() for _ in range(2)]
            fs[ct] = np.array([i["f"] for i in infos])
            assert infos[-1]["notspd"] == 0
    assert np.all(np.abs(fs[1] - fs[0]) <= 1e-6 * np.abs(fs[0]))


def test_chol_tc_foldin_matches_the_oracle(tiny):
    """Fold-in requests (1..800 ratings, cold start u0 = 0) with the TMEM
    factorisation and five corrections: every answer within 1e-6 of the
    oracle's exact solve."""
    from test_gpu_parity import _kappas
    r = tiny
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 3).astype(np.float32).astype(np.float64)
    ptr, items, vals = synth.foldin_requests(30, r.n_m, 1, 800, seed=9)
    ref = oracle.foldin(n_f, r.lam, x0[r.n_u * n_f:], ptr, items, vals.astype(np.float64))
    with _als(r, n_f, refine_steps=5) as m:
        m.set_launch(chol_tc=1, dual_max=0)
        m.set_x(x0)
        u = m.foldin(ptr, items, vals)
    Mf = x0[r.n_u * n_f:].reshape(r.n_m, n_f)
    kap = _kappas(ptr, items, Mf, r.lam, np.arange(len(ptr) - 1))
    assert _mixed_row_excess(u, ref, np.zeros_like(ref), kap, 1e-6) < 1.0
    assert _row_rel(u, ref, n_f) < 1e-6

