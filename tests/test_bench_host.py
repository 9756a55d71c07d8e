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


def test_traffic_only_for_captured_sources_and_shapes():
    """`traffic` is the captured per-sweep DRAM bytes over the launches of one
    sweep, and only for the sources and sweep shapes of a capture."""
    b = _bench()
    launch = dict(heavy_min=512, grid_mult=32, sweep_bin_min=0, split_min=2048, seg_len=1024,
                  gram_path=2, dual_max=64, dual_warp=1, tc_chunk=32, chol_tc=1)
    sha = b.kernel_source_sha("k_sweep_tc")
    for gt in (0, 1):
        launch["gather_tma"] = gt
        key = b.shapes_key(launch)
        want = [t[2] for t in b.TRAFFIC["k_sweep_tc"] if t[0] == sha and t[1] == key]
        got = b.traffic_for("k_sweep_tc", 6, launch)
        assert got == (want[0] / 6 if want else None)
        # the passes' shapes do not decide the sweep's launches
        assert b.traffic_for("k_sweep_tc", 6, dict(launch, heavy_min=1024, grid_mult=64)) == got
    assert b.traffic_for("k_sweep_tc", 6, dict(launch, seg_len=512)) is None
    assert b.traffic_for("k_sweep_tc", 0, launch) is None
    assert b.traffic_for("k_sweep_none", 6, launch) is None
