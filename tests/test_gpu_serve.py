"""Serving: requests through the continuous-batching server (C ABI).

A request's results depend only on the request, so each must equal a solo
parrep_run of a handle with the same network, options and seed, whatever
else runs beside it: statistics and histograms bit for bit (same
fixed-point sums, same normalisation), FIM and RER to 1e-12 relative (the
contraction adds per-bin terms in another order).
"""
import time

import numpy as np
import pytest

from paper_1705_06807_gb300 import ParRep, ParRepServer, configs as K
from paper_1705_06807_gb300.api import ParRepError

pytestmark = pytest.mark.gpu

V10 = K.schlogl_paper(V=10, hist_max=200, split=11)


def _requests():
    cp10 = np.array([V10["c"]] * 2, dtype=float)
    cp10[0, 0] *= 1.1
    cp10[1, 3] *= 0.9
    out = []
    for i, R in enumerate([1, 40, 96, 250]):
        out.append(dict(spec=V10, R=R, tc=200, tp=200, T_end=80.0 + 9 * i, seed=31 + i, x0=[2 + i], thresh="steps",
                        fv_group=16, T_burn=20.0, rer=cp10))
    tg = K.toggle(alpha=20, n=2.5, hist_max=(63, 63))
    for i, R in enumerate([64, 300]):
        out.append(dict(spec=tg, R=R, tc=0.5, tp=0.5, T_end=30.0 + 5 * i, seed=7 + i, x0=[15, 2], thresh="time",
                        fv_group=8, T_burn=5.0, rer=None))
    sc = K.schlogl_classic()
    out.append(dict(spec=sc, R=512, tc=1.0, tp=1.0, T_end=40.0, seed=3, x0=[85], thresh="time", fv_group=32,
                    T_burn=10.0, rer=None))
    return out


def _solo(q, precision):
    g = ParRep(q["spec"], q["R"], q["tc"], q["tp"], x0=q["x0"], thresh=q["thresh"], precision=precision,
               fv_group=q["fv_group"], T_burn=q["T_burn"])
    g.run(q["T_end"], q["seed"])
    rer = g.rer(q["rer"]) if q["rer"] is not None else None
    return g.stats(), g.histogram(), g.fim(), rer


def _submit(srv, q):
    return srv.submit(q["spec"], q["R"], q["tc"], q["tp"], q["T_end"], q["seed"], x0=q["x0"], thresh=q["thresh"],
                      fv_group=q["fv_group"], T_burn=q["T_burn"], rer=q["rer"])


KEYS = ("events_decorr", "events_dephase", "events_parallel_useful", "cycles", "escapes", "x0", "x_final", "T_s")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_served_results_equal_solo_runs(precision):
    reqs = _requests()
    srv = ParRepServer(precision=precision)
    ids = [_submit(srv, q) for q in reqs]  # all in flight together
    res = [srv.result(i) for i in ids]
    for q, r in zip(reqs, res):
        assert r["status"] == 0
        st, hist, fim, rer = _solo(q, precision)
        assert {k: r["stats"][k] for k in KEYS} == {k: st[k] for k in KEYS}
        assert np.array_equal(r["hist"], hist)
        np.testing.assert_allclose(r["fim"], fim, rtol=1e-12, atol=1e-12 * np.abs(fim).max())
        if rer is not None:
            np.testing.assert_allclose(r["rer"], rer, rtol=1e-12, atol=1e-15)
        assert r["latency_s"] > 0.0
    # the same requests again, one at a time: the same results
    for q, r in zip(reqs[:3], res[:3]):
        r2 = srv.result(_submit(srv, q))
        assert np.array_equal(r2["hist"], r["hist"])
        assert {k: r2["stats"][k] for k in KEYS} == {k: r["stats"][k] for k in KEYS}
    s = srv.stats()
    assert s["submitted"] == s["released"] == len(reqs) + 3
    assert s["arena_used"] == 0
    srv.close()


def test_requests_overlap_on_the_device():
    """Short requests submitted while a long one runs finish before it."""
    srv = ParRepServer(precision="f32")
    sc = K.schlogl_classic()
    long_id = srv.submit(sc, 4096, 1.0, 1.0, 3e5, 11, x0=[565], T_burn=0.0)
    time.sleep(0.005)
    short = [srv.submit(V10, 48, 200, 200, 60.0, 100 + i, x0=[3], thresh="steps") for i in range(4)]
    overlapped = 0
    for i in short:
        srv.wait(i)
        if srv.poll(long_id) != 2:
            overlapped += 1
    assert overlapped >= 1
    rs = [srv.result(i) for i in short]
    rl = srv.result(long_id)
    assert all(r["status"] == 0 for r in rs) and rl["status"] == 0
    assert max(r["latency_s"] for r in rs) < rl["latency_s"]
    srv.close()


def test_admission_is_bounded_by_device_memory():
    """A small arena admits a few requests at a time; a finished request
    keeps its memory until its result is read, so results are collected as
    they come; all complete."""
    srv = ParRepServer(precision="f32", arena_bytes=8 << 20)  # about 3.4 MB per request: two at a time
    sc = K.schlogl_classic()
    ids = [srv.submit(sc, 65536, 1.0, 1.0, 30.0, 50 + i, x0=[85], T_burn=0.0) for i in range(6)]
    most, left, t0 = 0, list(ids), time.time()
    while left and time.time() - t0 < 120:
        s = srv.stats()
        most = max(most, s["running"])
        assert s["arena_used"] <= s["arena_bytes"]
        for i in [i for i in left if srv.poll(i) == 2]:
            assert srv.result(i)["status"] == 0
            left.remove(i)
        time.sleep(0.0005)
    assert not left
    assert 1 <= most <= 2
    srv.close()


def test_server_rejects_bad_requests():
    srv = ParRepServer(precision="f64", arena_bytes=8 << 20)
    with pytest.raises(ParRepError):
        srv.submit(V10, 0, 10, 10, 10.0, 1, x0=[2], thresh="steps")
    with pytest.raises(ParRepError):
        srv.submit(V10, 16, 10, 10, 1e9, 1, x0=[2], thresh="steps")
    with pytest.raises(ParRepError):  # can never fit the arena
        srv.submit(K.schlogl_classic(), 1 << 22, 1.0, 1.0, 10.0, 1, x0=[85])
    r = srv.result(srv.submit(V10, 16, 10, 10, 10.0, 1, x0=[2], thresh="steps"))
    assert r["status"] == 0
    srv.close()
