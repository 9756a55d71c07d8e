"""Per-kernel sweep timing (als_time_sweep, needs a GB300): the classes
partition the rows of both halves, the split rows' tensor-core segments are
timed as a class of their own, and the timed sweep (split part on the
context's stream) writes the same xbar as a sweep with the split part beside
the other rows."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_time_sweep_classes_and_result():
    from paper_1508_03110_gb300 import ALS
    r = synth.make_config("tiny")
    n_f = 100
    x0 = synth.init_factors(r.n_u, r.n_m, n_f, 4)
    with ALS(r.n_u, r.n_m, r.rows, r.cols, r.vals, n_f, r.lam, precision="mixed", gram_path="tc") as m:
        m.set_launch(split_min=256, seg_len=64)
        m.set_x(x0)
        m.step(info=False)
        forked = m.get_state()["xbar"]  # P(x_1), the split part beside the other rows
        ts = m.time_sweep(reps=2)
        timed = m.get_state()["xbar"]   # P(x_1) again, the split part on the context's stream
    assert np.array_equal(forked, timed)
    whole = ("k_sweep_tc_pf", "k_sweep_tc", "k_sweep_dual", "split")
    assert sum(ts[k]["rows"] for k in whole) == r.n_u + r.n_m
    assert sum(ts[k]["ratings"] for k in whole) == 2 * len(r.vals)
    seg = ts["k_sweep_tc_seg"]
    assert seg["launches"] == 2 and seg["rows"] == ts["split"]["rows"] > 0
    assert seg["ratings"] == ts["split"]["ratings"]
    assert 0.0 < seg["ms"] <= ts["split"]["ms"] + 1e-3
    assert ts["sweep_ms"] > 0.0
