"""The TMA-fed gather of the tensor-core sweep (needs a GB300): the heavy
rows' FP32 factor rows reach shared memory by tile::gather4 TMA copies two
chunks ahead instead of by per-lane cp.async one chunk ahead.  The arithmetic
that follows is the same, so the results must be bit-identical to the
cp.async variant's: one sweep, split-row segments, ALS-NCG iterations, at
the full benchmark size too, and fold-in."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _pair(r, n_f, launch, steps, x0, foldin=None):
    from paper_1508_03110_gb300 import ALS
    out = []
    for g in (0, 1):
        with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc") as m:
            m.set_launch(gather_tma=g, **launch)
            assert m.get_launch()["gather_tma"] == g
            m.set_x(x0)
            m.sweep(1)
            res = [m.get_x()]
            m.set_x(x0)
            for _ in range(steps):
                m.step(info=False)
            res.append(m.get_x())
            if foldin is not None:
                res.append(m.foldin(*foldin))
        out.append(res)
    return out


@pytest.mark.parametrize("n_f", [48, 100, 128])
def test_tma_gather_equals_cp_async(n_f):
    r = synth.make_config("tiny")
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 5)
    req = synth.foldin_requests(60, r.n_m, 1, 900, seed=4)
    a, b = _pair(r, n_f, {}, 4, x0, foldin=req)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_tma_gather_split_rows_equal_cp_async():
    """Forced splitting: every row of at least 256 ratings is cut into
    segments of 64, each gathered by TMA."""
    r = synth.make_config("tiny")
    x0 = synth.init_factors(r.n_u, r.n_m, 100, 6)
    a, b = _pair(r, 100, dict(split_min=256, seg_len=64), 3, x0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_tma_gather_fullsize_equals_cp_async():
    r = synth.make_config("ml20m")
    x0 = synth.init_factors(r.n_u, r.n_m, r.n_f, 11)
    a, b = _pair(r, r.n_f, dict(heavy_min=1024, grid_mult=64, split_min=65536, seg_len=4096, dual_max=64), 2, x0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_chunk_sizes_agree():
    """Rows below 256 ratings gathered in chunks of 16 ratings (7 CTAs per SM)
    or 32: the same Gram matrices (the same MMAs in the same order); the FP32
    residual's compensated sum is grouped per chunk, so the rows agree to the
    refinement's FP32 floor, far inside the mixed form's bound."""
    from paper_1508_03110_gb300 import ALS
    r = synth.make_config("tiny")
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 8)
    out = {}
    for kc in (16, 32):
        with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc") as m:
            m.set_launch(tc_chunk=kc)
            assert m.get_launch()["tc_chunk"] == kc
            m.set_x(x0)
            m.sweep(1)
            out[kc] = m.get_x().reshape(-1, n_f)
    err = np.linalg.norm(out[16] - out[32], axis=1)
    assert np.all(err <= 1e-6 * np.linalg.norm(out[32], axis=1) + 1e-30)
