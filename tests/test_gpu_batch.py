"""Batches: many instances in one persistent launch (through the C ABI).

An instance's arithmetic does not depend on the blocks that run it, so every
instance of a batch must end with exactly the results that parrep_run gives
the same handle alone: the same fixed-point histograms, cycle logs and event
counts, bit for bit.  One instance is also checked against the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1705_06807_gb300 import ParRep, ParRepBatch, configs as K
from paper_1705_06807_gb300.api import ParRepError

pytestmark = pytest.mark.gpu

V10 = K.schlogl_paper(V=10, hist_max=200, split=11)


def _mixed(precision):
    """Schloegl in both threshold modes and toggles, uneven replica counts."""
    out = []
    for i, R in enumerate([1, 33, 64, 200, 77, 5]):
        out.append((ParRep(V10, R, 200, 200, x0=[2 + i], thresh="steps", precision=precision, fv_group=16,
                           T_burn=30.0), 90.0 + 7 * i, 11 + i))
    tg = K.toggle(alpha=20, n=2.5, hist_max=(63, 63))
    for i, R in enumerate([48, 130, 16]):
        out.append((ParRep(tg, R, 0.5, 0.5, x0=[15, 2], precision=precision, fv_group=8, T_burn=5.0),
                    40.0 + 5 * i, 101 + i))
    sc = K.schlogl_classic()
    out.append((ParRep(sc, 96, 1.0, 1.0, x0=[85], precision=precision, T_burn=2.0), 12.0, 7))
    return out


def _result(g):
    pre, post = g.histogram_raw()
    st = g.stats()
    keys = ("events_decorr", "events_dephase", "events_parallel_useful", "cycles", "escapes", "x0", "x_final",
            "T_s")
    return pre, post, g.cycle_log(), {k: st[k] for k in keys}


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    assert a[3] == b[3]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_solo_runs(precision, graph):
    inst = _mixed(precision)
    solo = []
    for g, T, s in inst:
        g.run(T, s)
        solo.append(_result(g))
    b = ParRepBatch([g for g, _, _ in inst], use_graph=graph)
    info = b.run([T for _, T, _ in inst], [s for _, _, s in inst])
    assert b.status() == [0] * len(inst)
    assert info["graph"] == (1 if graph else 0)
    assert info["grid_blocks"] > 0 and info["n_items"] >= len(inst)
    for (g, _, _), r in zip(inst, solo):
        _same(_result(g), r)
    # a second run with other seeds (the graph is replayed) still matches solo runs
    seeds2 = [s + 1000 for _, _, s in inst]
    b.run([T for _, T, _ in inst], seeds2)
    res2 = [_result(g) for g, _, _ in inst]
    for (g, T, _), s2, r in zip(inst, seeds2, res2):
        g.run(T, s2)
        _same(_result(g), r)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_block_shapes_do_not_change_results(precision):
    inst = _mixed(precision)
    shapes = ([(128, 128, "auto"), (64, 64, "auto")] if precision == "f64" else
              [(384, 32, "staged"), (256, 64, "staged"), (384, 128, "staged"), (256, 256, "direct"),
               (128, 128, "direct"), (384, 64, "mixed")])
    ref = None
    for T, RB, layout in shapes:
        b = ParRepBatch([g for g, _, _ in inst], block_threads=T, replicas_per_block=RB, autotune=False,
                        f32_layout=layout)
        info = b.run([T_ for _, T_, _ in inst], [s for _, _, s in inst])
        assert info["block_threads"] == T and info["replicas_per_block"] == RB
        res = [_result(g) for g, _, _ in inst]
        if ref is None:
            ref = res
        else:
            for a, r in zip(res, ref):
                _same(a, r)
        b.close()


def test_batch_mixed_layout_equals_solo_runs():
    """The mixed FP32 batch kernel runs each instance in its own layout --
    one thread per replica from 16384 replicas on, owner + helper warps below
    -- and every instance still ends with its solo run's results."""
    big = ParRep(V10, 20000, 100, 100, x0=[3], thresh="steps", precision="f32", fv_group=32, T_burn=5.0)
    small = ParRep(V10, 40, 200, 200, x0=[2], thresh="steps", precision="f32", fv_group=16, T_burn=5.0)
    tg = ParRep(K.toggle(alpha=20, n=2.5, hist_max=(63, 63)), 17000, 0.5, 0.5, x0=[15, 2], precision="f32",
                T_burn=2.0)
    inst = [(big, 12.0, 5), (small, 60.0, 6), (tg, 6.0, 7)]
    solo = []
    for g, T, sd in inst:
        g.run(T, sd)
        solo.append(_result(g))
    b = ParRepBatch([g for g, _, _ in inst], block_threads=384, replicas_per_block=64, autotune=False,
                    f32_layout="mixed")
    b.run([T for _, T, _ in inst], [sd for _, _, sd in inst])
    assert b.status() == [0, 0, 0]
    assert b.info()["f32_layout"] == "mixed"
    for (g, _, _), r in zip(inst, solo):
        _same(_result(g), r)
    b.close()


def test_batch_layout_choice():
    """The FP32 auto layout is the mixed one, and the chosen layout is
    reported."""
    a = ParRep(V10, 40, 50, 50, x0=[2], thresh="steps", precision="f32")
    b = ParRepBatch([a], autotune=False)
    b.run([5.0], [1])
    assert b.info()["f32_layout"] == "mixed"
    b.close()
    b = ParRepBatch([a], autotune=False, f32_layout="staged")
    b.run([5.0], [1])
    assert b.info()["f32_layout"] == "staged"
    b.close()
    d = ParRep(V10, 40, 50, 50, x0=[2], thresh="steps")
    b = ParRepBatch([d], autotune=False)
    b.run([5.0], [1])
    assert b.info()["f32_layout"] is None
    b.close()


def test_batch_autotuner_tries_shapes_and_keeps_results():
    inst = _mixed("f32")
    b = ParRepBatch([g for g, _, _ in inst], autotune=True)
    info = b.run([T for _, T, _ in inst], [s for _, _, s in inst])
    assert info["tuned_trials"] >= 2
    res = [_result(g) for g, _, _ in inst]
    for (g, T, s), r in zip(inst, res):
        g.run(T, s)
        _same(_result(g), r)


def test_batch_instance_against_oracle():
    """The first Schloegl instance of a batch against the oracle (integers exact)."""
    inst = _mixed("f64")
    b = ParRepBatch([g for g, _, _ in inst])
    b.run([T for _, T, _ in inst], [s for _, _, s in inst])
    g, T, s = inst[3]
    o = O.parrep_run(V10, 200, 200, 200, T, s, [5], thresh="steps", fv_group=16, T_burn=30.0)
    st = g.stats()
    assert st["events_parallel_useful"] == o["events_parallel_useful"]
    assert st["events_dephase"] == o["events_dephase"] and st["escapes"] == o["escapes"]
    assert [c["n_star"] for c in g.cycle_log()] == [c["n_star"] for c in o["cycles"]]
    pre, post = g.histogram_raw()
    # fixed-point sums vs binary64 sums: n * 2^-41 per bin plus summation error
    tol = 4e-12 * (o["events_decorr"] + o["events_parallel_useful"]) + 1e-12 * T
    np.testing.assert_allclose(pre, o["hist_pre"], rtol=1e-12, atol=tol)
    np.testing.assert_allclose(post, o["hist_post"], rtol=1e-12, atol=tol)


def test_batch_reports_a_failing_instance_and_finishes_the_others():
    spec = dict(K.schlogl_classic(), hist_max=120)
    bad = ParRep(spec, 32, 1.0, 1.0, x0=[85])
    good = ParRep(V10, 40, 200, 200, x0=[3], thresh="steps")
    b = ParRepBatch([good, bad], autotune=False)
    rc = b.run_status([60.0, 100.0], [5, 0])
    assert rc == -5
    assert b.status() == [0, -5]
    r = _result(good)
    good.run(60.0, 5)
    _same(_result(good), r)


def test_batch_rejects_bad_arguments():
    a = ParRep(V10, 8, 10, 10, x0=[2], thresh="steps")
    c = ParRep(V10, 8, 10, 10, x0=[2], thresh="steps", precision="f32")
    with pytest.raises(ParRepError):
        ParRepBatch([a, a])
    with pytest.raises(ParRepError):
        ParRepBatch([a, c])
    with pytest.raises(ParRepError):
        ParRepBatch([a], replicas_per_block=48)
    b = ParRepBatch([a])
    with pytest.raises(ParRepError):
        b.run([1e9], [0])
