"""Host logic of bench.py (no GPU): the algorithmic FLOPs of one sweep, counted
per row for the formulation the kernels take (the roofline's numerator)."""
import importlib.util
import os

import numpy as np

import synth


def _bench():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "bench.py")
    spec = importlib.util.spec_from_file_location("bench_host", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _per_row(d, nf, refine, dual_max):
    """Row by row: n_f x n_f Gram, Cholesky, solves and residual; or, for
    0 < d <= min(dual_max, n_f), the d x d matrix F F^T, its Cholesky, and per
    correction F v, F^T z, solves and residual."""
    tot = gram = 0.0
    for di in d.astype(float):
        if di == 0:
            continue
        if di <= min(dual_max, nf):
            tot += nf * di * (di + 1) + di ** 3 / 3 + refine * (4 * nf * di + 2 * di ** 2 + 4 * nf * di)
        else:
            g = di * nf * (nf + 1)
            gram += g
            tot += g + nf ** 3 / 3 + refine * (2 * nf ** 2 + 4 * nf * di)
    return tot, gram


def test_sweep_flops_per_row_formulation():
    b = _bench()
    r = synth.make_config("tiny")
    d = np.concatenate([np.bincount(r.rows, minlength=r.n_u), np.bincount(r.cols, minlength=r.n_m)])
    nf = 100
    for dual_max in (0, 16, 64):
        tot, gram = b.sweep_flops(r, nf, 2, "mixed", dual_max)
        ref_tot, ref_gram = _per_row(d, nf, 2, dual_max)
        assert np.isclose(tot, ref_tot, rtol=1e-12) and np.isclose(gram, ref_gram, rtol=1e-12)
    # light rows cost less in their own formulation, and none of it is on the tensor cores
    t0, g0 = b.sweep_flops(r, nf, 2, "mixed", 0)
    t64, g64 = b.sweep_flops(r, nf, 2, "mixed", 64)
    assert t64 < t0 and g64 < g0
    # the FP64 form has no light rows and no tensor-core part
    t64f, g64f = b.sweep_flops(r, nf, 2, "fp64", 64)
    assert g64f == 0.0
    assert np.isclose(t64f, b.sweep_flops(r, nf, 2, "fp64", 0)[0])
