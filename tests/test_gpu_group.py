"""Groups of batched contexts with different n_f run together
(als_group_run): each problem follows the oracle's trajectory (FP64), and the
group's result equals running each member alone (needs a GB300)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def probs():
    return synth.make_batch(8, 2_000, 30_000, 0.01, 0.05, seed=12)


def test_group_fp64_matches_oracle_per_problem(probs):
    from paper_1508_03110_gb300 import ALSGroup
    n_fs = [5, 8, 12, 20] * 2
    xs = [synth.init_factors(nu, nm, nf, 40 + q) for q, ((nu, nm, *_r), nf) in enumerate(zip(probs, n_fs))]
    refs = [oracle.alsncg(oracle.build_problem(nu, nm, nf, 0.05, rr, cc, vv), x0, 5)
            for (nu, nm, rr, cc, vv), nf, x0 in zip(probs, n_fs, xs)]
    with ALSGroup(probs, n_fs, 0.05, precision="fp64") as g:
        g.set_x(xs)
        out = g.run(5)
        got = g.get_x()
    assert out["iters"] == 5 and out["kernels"] > 0
    for q in range(len(probs)):
        assert _rel(got[q], refs[q][-1].x) < 1e-9, q


@pytest.mark.parametrize("schedule", ["serial", "concurrent"])
def test_group_equals_members_alone(probs, schedule):
    """One stream for all members or one each: the same factors, bit for bit,
    as each member run on its own."""
    from paper_1508_03110_gb300 import ALSGroup
    n_fs = [10, 20, 50, 100] * 2
    xs = [synth.init_factors(nu, nm, nf, 60 + q) for q, ((nu, nm, *_r), nf) in enumerate(zip(probs, n_fs))]
    with ALSGroup(probs, n_fs, 0.05, precision="mixed", autotune=False, schedule=schedule) as g:
        if schedule == "serial":
            assert len({id(st) for st in g.streams.values()}) == 1
        else:
            assert len({id(st) for st in g.streams.values()}) == len(g.streams)
        g.set_x(xs)
        g.run(12, check_every=4)
        together = g.get_x()
    with ALSGroup(probs, n_fs, 0.05, precision="mixed", autotune=False) as g:
        g.set_x(xs)
        for b in g.batches.values():
            b.run(12, 0.0, check_every=4)
        alone = g.get_x()
    for q in range(len(probs)):
        assert np.array_equal(together[q], alone[q]), q


def test_group_converges_and_rejects_a_repeated_member(probs):
    import ctypes
    from paper_1508_03110_gb300 import ALSError, ALSGroup, _lib
    n_fs = [10, 20, 50, 100] * 2
    xs = [synth.init_factors(nu, nm, nf, 80 + q) for q, ((nu, nm, *_r), nf) in enumerate(zip(probs, n_fs))]
    with ALSGroup(probs, n_fs, 0.05, precision="mixed") as g:
        g.set_x(xs)
        out = g.run(300, rel_tol=1e-4, check_every=10)
        infos = g.infos()
        assert all(i["gnorm"] <= 1e-4 * i["gnorm0"] for i in infos)
        assert out["iters"] < 300
        b = next(iter(g.batches.values()))
        arr = (ctypes.c_void_p * 2)(b.ctx.value, b.ctx.value)
        with pytest.raises(ALSError, match="EINVAL"):
            _lib.check(_lib.load().als_group_run(arr, 2, 1, 0.0, 1, None, None), "als_group_run")
