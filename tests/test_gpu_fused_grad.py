"""The users' gradient rows written by the mixed tensor-core sweep (needs a
GB300): for every user row the sweep forms the FP32 residual r0 = sum_e f_e
(r_e - f_e . x_i) at the current row, and -2 (r0 - lambda n_i x_i) is that
row of grad f(x); the gradient pass then forms only the rows' FP64 terms."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _als(r, n_f, **kw):
    from paper_1508_03110_gb300 import ALS
    return ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc", **kw)


@pytest.fixture(scope="module")
def tiny():
    return synth.make_config("tiny")


@pytest.mark.parametrize("split,dual_warp", [(False, 1), (True, 1), (False, 0)])
def test_fused_users_gradient_matches_the_gradient_pass(tiny, split, dual_warp):
    """The mixed tensor-core sweep writes the users' gradient rows from its
    first residual; after ALS-NCG steps the state's gradient equals what the
    gradient pass forms at the same x, and the oracle's, row by row to FP32
    rounding: with split rows, and with either light-row kernel."""
    r = tiny
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 21)
    with _als(r, n_f) as m:
        m.set_launch(dual_warp=dual_warp)
        if split:
            m.set_launch(split_min=256, seg_len=64)
        m.set_x(x0)
        for _ in range(3):
            m.step(info=False)
        st = m.get_state()
        g_pass, _ = m.grad()
    gf = st["g"].reshape(-1, n_f)[: r.n_u]
    gp = np.asarray(g_pass).reshape(-1, n_f)[: r.n_u]
    P = oracle.build_problem(r.n_u, r.n_m, n_f, r.lam, r.rows, r.cols, r.vals)
    g_ref = oracle.grad(P, st["x"]).reshape(-1, n_f)[: r.n_u]
    err = np.linalg.norm(gf - gp, axis=1)
    scale = np.maximum(np.linalg.norm(g_ref, axis=1), 1e-3 * np.median(np.linalg.norm(g_ref, axis=1)))
    assert np.max(err / scale) < 1e-4, np.max(err / scale)
    assert np.max(np.linalg.norm(gf - g_ref, axis=1) / scale) < 1e-4
