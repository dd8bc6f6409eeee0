"""The genetic switch of Sec. V.B on the CUDA path (binary64 form).

State x0 = 2m + xi, x1 = p, six channels (Table IV with the switching rates
F, G).  Every integer result of a run -- event counts, cycles, escapes, the
cycle log, the final state -- equals the oracle's for the same seed; the
time sums agree to the fixed-point rounding (at most 2^-41 per holding time).
Plain SSA likewise.  The eight-parameter FIM and RER (Appendix A form,
parameters a, b, gamma, k0min, k0max, k1min, k1max, D taken independently)
equal the oracle's per-event sums; batches and served requests give each
instance its solo result; parrep_uq takes the kind.  The pooled histogram of
a small bistable switch matches its exact law, and at the paper's constants
the FIM diagonal matches the exact chain's (Table V).  Only the FP32 form
refuses the kind.
"""
import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from paper_1705_06807_gb300 import ParRep, ParRepBatch, ParRepServer, parrep_ssa, parrep_uq
from paper_1705_06807_gb300.api import ParRepError, parrep_ssa_trace

pytestmark = pytest.mark.gpu

SMALL = [12.0, 5.0, 10.0, 0.2, 20.0, 0.2, 20.0, 25.0]  # bistable: p ~ 0.6 / 46, saddle 12.8


def _spec(c, m_max, p_max, split):
    return dict(kind="genetic", c=list(c), s=[1.0, 1.0, 1.0, 1.0], hist_max=[2 * m_max + 1, p_max],
                regions=[([0, 1], split)])


CASES = [
    ("small_steps", _spec(SMALL, 16, 250, 13), 16, 200, 200, "steps", 300.0, 50.0, 3),
    ("small_time", _spec(SMALL, 16, 250, 13), 40, 2.0, 2.0, "time", 200.0, 20.0, 8),
    ("paper_steps", _spec(E.genetic_paper_params(), 15, 3500, 512), 32, 2000, 2000, "steps", 20.0, 5.0, 5),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name,spec,R,tc,tp,thresh,T,Tb,seed", CASES, ids=[c[0] for c in CASES])
def test_genetic_run_matches_oracle(name, spec, R, tc, tp, thresh, T, Tb, seed, precision):
    """Both precision forms (binary32: six-channel propensities and selection
    in binary32, the oracle's binary32 mode; it runs in the direct layout)."""
    o = O.parrep_run(spec, R, tc, tp, T, seed, [0, 0], thresh=thresh, T_burn=Tb, precision=precision)
    g = ParRep(spec, R, tc, tp, x0=[0, 0], thresh=thresh, T_burn=Tb, precision=precision)
    assert g.run_status(T, seed) == o["status"] == 0
    st = g.stats()
    for k in ("events_decorr", "events_dephase", "events_parallel_useful", "escapes"):
        assert st[k] == o[k], k
    assert st["cycles"] == o["n_cycles"]
    assert st["x0"] == o["x0"] and st["x_final"] == o["x_final"]
    assert st["T_s"] == T == o["T_s"]
    cg, co = g.cycle_log(), o["cycles"]
    assert len(cg) == len(co)
    for a, b in zip(cg, co):
        for k in ("cycle", "W", "ended", "decorr_steps", "dephase_steps", "n_star", "k", "x_tilde"):
            assert a[k] == b[k], (k, a, b)
    pre, post = g.histogram_raw()
    rt = 2.0**-22 if precision == "f32" else 1e-12
    tol = 4e-12 * max(o["events_decorr"] + o["events_parallel_useful"], 1) + 1e-12 * T + (rt * T if precision == "f32" else 0)
    np.testing.assert_allclose(pre, o["hist_pre"], rtol=rt, atol=tol)
    np.testing.assert_allclose(post, o["hist_post"], rtol=rt, atol=tol)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_genetic_plain_ssa_matches_oracle(precision):
    spec = _spec(E.genetic_paper_params(), 15, 3500, 512)
    hg, evg, _ = parrep_ssa(spec, 9, [0, 0], 3.0, 17, precision=precision)
    ho, evo, _ = O.ssa_run(spec, 9, [0, 0], 3.0, 17, precision=precision)
    assert evg == evo
    rt = 2.0**-22 if precision == "f32" else 1e-12
    np.testing.assert_allclose(hg, ho, rtol=rt, atol=4e-12 * evo + 1e-12 * 27.0 + (rt * 27.0 if precision == "f32" else 0))
    J, xs, tau, nj, xf = parrep_ssa_trace(spec, 4, [0, 0], 1e6, 5, 400, precision=precision)
    for t in range(4):
        Jo, xo, to = O.ssa_trace(spec, [0, 0], 5, t, 400, precision=precision)
        assert np.array_equal(J[t], Jo) and np.array_equal(xs[t], xo)


def test_genetic_parrep_matches_exact_law():
    """Algorithm 1 on the small switch (R = 16, n_c = n_p = 1000): pooled
    protein marginal within TV 0.02 of the exact law over about a hundred
    escapes (the oracle's own run of these settings is at 0.005)."""
    mm, pm = 16, 250
    spec = _spec(SMALL, mm, pm, 13)
    Q, pi = E.genetic_stationary(np.array(SMALL), mm, pm, pin=((40 * (mm + 1)) + 1) * 2 + 1)
    xi, m, p = E.genetic_states(mm, pm)
    ex = np.zeros((2 * mm + 2) * (pm + 1))
    ex[(2 * m + xi) * (pm + 1) + p] = pi
    tot, esc = np.zeros(len(ex)), 0
    for seed in range(6):
        g = ParRep(spec, 16, 1000, 1000, x0=[0, 0], thresh="steps")
        g.run(5000.0, 40 + seed)
        pre, post = g.histogram_raw()
        tot += pre + post
        esc += g.stats()["escapes"]
    assert esc > 50
    marg = lambda h: h.reshape(2 * mm + 2, pm + 1).sum(0)
    assert 0.5 * np.abs(marg(tot / tot.sum()) - marg(ex)).sum() < 0.02


def test_genetic_fp32_needs_the_direct_layout():
    """The staged FP32 layout has no six-channel chain: asking for it is
    refused by single runs, servers and batches; the default (auto / mixed)
    layouts and the direct server take the kind."""
    spec = _spec(SMALL, 16, 250, 13)
    g = ParRep(spec, 16, 50, 50, x0=[0, 0], thresh="steps", precision="f32")
    with pytest.raises(ParRepError):
        g.set_options(thresh="steps", precision="f32", f32_layout="staged")
    srv = ParRepServer(precision="f32", arena_bytes=8 << 20, f32_layout="staged")
    with pytest.raises(ParRepError):
        srv.submit(spec, 16, 50, 50, 10.0, 1, x0=[0, 0], thresh="steps")
    srv.close()
    with pytest.raises(ParRepError):
        ParRepBatch([g], f32_layout="staged")
    solo = ParRep(spec, 16, 50, 50, x0=[0, 0], thresh="steps", precision="f32", T_burn=2.0)
    solo.run(10.0, 1)
    for layout in ("direct", "mixed"):
        srv = ParRepServer(precision="f32", arena_bytes=64 << 20, f32_layout=layout)
        r = srv.result(srv.submit(spec, 16, 50, 50, 10.0, 1, x0=[0, 0], thresh="steps", T_burn=2.0),
                       timeout_s=60.0)
        srv.close()
        assert r["status"] == 0 and np.array_equal(r["hist"], solo.histogram())


def _cprime():
    cp = np.array([SMALL] * 3, dtype=float)
    cp[0, 0] *= 1.1   # a
    cp[1, 4] *= 0.8   # k0max
    cp[2, 7] *= 1.05  # D
    return cp


def test_genetic_fim_rer_match_oracle():
    """The eight-parameter FIM and three RERs of a run equal the oracle's
    per-event sums over [T_burn, T_end] (the device contracts the post-burn
    histogram instead; the two agree to the fixed-point rounding)."""
    spec = _spec(SMALL, 16, 250, 13)
    cp = _cprime()
    T, Tb = 200.0, 20.0
    o = O.parrep_run(spec, 40, 2.0, 2.0, T, 8, [0, 0], thresh="time", T_burn=Tb, rer_cprime=cp)
    g = ParRep(spec, 40, 2.0, 2.0, x0=[0, 0], thresh="time", T_burn=Tb)
    assert g.run_status(T, 8) == o["status"] == 0
    assert g.stats()["events_parallel_useful"] == o["events_parallel_useful"]
    F = g.fim()
    Fo = o["fim"] / (T - Tb)
    assert F.shape == (8, 8)
    np.testing.assert_allclose(F, Fo, rtol=1e-7, atol=1e-12 * np.abs(Fo).max())
    R = g.rer(cp)
    np.testing.assert_allclose(R, o["rer"] / (T - Tb), rtol=1e-7, atol=1e-15)
    # I_11 = E[xi]/a (one channel depends on a, linearly)
    h = g.histogram_raw()[1].reshape(2 * 16 + 2, 251)
    p_on = h[1::2].sum() / h.sum()
    assert abs(F[0, 0] - p_on / SMALL[0]) < 1e-9 * F[0, 0]


def _solo(spec, R, tc, tp, thresh, T, Tb, seed, x0):
    g = ParRep(spec, R, tc, tp, x0=x0, thresh=thresh, T_burn=Tb)
    g.run(T, seed)
    return g


def test_genetic_batch_and_serve_equal_solo_runs():
    """Genetic instances beside a Schloegl one in a binary64 batch, and as
    served requests in flight together: each result equals its solo run."""
    V10 = dict(kind="schlogl", c=[3.0, 0.6, 0.25, 2.95], s=[1.0 / 10, 1.0 / 100, 2.0 * 10, 1.0], hist_max=200,
               regions=[([1], 11)])
    sp = _spec(SMALL, 16, 250, 13)
    jobs = [(sp, 24, 1.0, 1.0, "time", 80.0, 10.0, 3, [0, 0]), (sp, 40, 300, 300, "steps", 60.0, 5.0, 4, [1, 30]),
            (V10, 32, 200, 200, "steps", 70.0, 10.0, 5, [3]), (sp, 7, 2.0, 2.0, "time", 50.0, 0.0, 6, [0, 0])]
    solo = [_solo(*j) for j in jobs]
    hs = [ParRep(j[0], j[1], j[2], j[3], x0=j[8], thresh=j[4], T_burn=j[6]) for j in jobs]
    b = ParRepBatch(hs, autotune=False)
    b.run([j[5] for j in jobs], [j[7] for j in jobs])
    assert b.status() == [0] * len(jobs)
    for a, h in zip(solo, hs):
        assert np.array_equal(a.histogram(), h.histogram())
        assert a.stats()["events_parallel_useful"] == h.stats()["events_parallel_useful"]
        np.testing.assert_allclose(h.fim(), a.fim(), rtol=1e-12, atol=1e-14 * np.abs(a.fim()).max())
    srv = ParRepServer(precision="f64")
    ids = [srv.submit(j[0], j[1], j[2], j[3], j[5], j[7], x0=j[8], thresh=j[4], T_burn=j[6],
                      rer=_cprime() if j[0] is sp else None) for j in jobs]
    res = [srv.result(i) for i in ids]
    srv.close()
    for a, r, j in zip(solo, res, jobs):
        assert r["status"] == 0
        assert np.array_equal(r["hist"], a.histogram())
        np.testing.assert_allclose(r["fim"], a.fim(), rtol=1e-12, atol=1e-14 * np.abs(a.fim()).max())
        if j[0] is sp:
            np.testing.assert_allclose(r["rer"], a.rer(_cprime()), rtol=1e-12, atol=1e-15)


def test_genetic_uq_matches_oracle_estimators():
    """parrep_uq over genetic runs: the IAF of the protein count, the mean and
    the eight-parameter FIM with half widths equal the oracle's Sec. IV.B
    estimators applied to the same runs' post-burn histograms and FIMs."""
    from oracle import uq as U

    spec = _spec(SMALL, 16, 250, 13)
    T, Tb = 120.0, 20.0
    hs = [_solo(spec, 24, 1.0, 1.0, "time", T, Tb, 70 + k, [0, 0]) for k in range(6)]
    f = np.tile(np.arange(251.0), 34)  # f = p on bins (2m + xi, p)
    r = parrep_uq(hs, f)
    posts = [h.histogram_raw()[1] for h in hs]
    ref = U.uq(f, posts, [h.fim() for h in hs], T - Tb)
    assert r["fim"].shape == (8, 8)
    np.testing.assert_allclose(r["Y"], ref["Y"], rtol=1e-12)
    np.testing.assert_allclose(r["iaf"], ref["iaf"], rtol=1e-9)
    np.testing.assert_allclose(r["mean_f"], ref["mean_f"], rtol=1e-12)
    np.testing.assert_allclose(r["fim"], ref["fim"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(r["fim_half_width"], ref["fim_half_width"], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(r["bounds"], ref["bounds"], rtol=1e-8)


def test_genetic_paper_constants_fim_against_exact_chain():
    """The paper's switch (Sec. V.B: b = 22.5, a = 2400/b, gamma = 50, D =
    1000, ...) with its Algorithm 1 settings (R = 100, n_c = n_p = 2e4 jumps):
    32 samples to T = 2e4 after a burn-in of 2e3, in one binary64 batch.  The
    mean FIM diagonal lies within 4.5 standard errors (from the spread over
    samples) of the exact chain's, which itself lies inside Table V's half
    widths; parrep_uq returns the same mean."""
    import json
    import os

    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "exact_references.json")))
    exact = np.asarray(ref["genetic_paper"]["fim_diag"])
    spec = _spec(E.genetic_paper_params(), 15, 3500, 512)
    n, T, Tb = 32, 2e4, 2e3
    hs = [ParRep(spec, 100, 20000, 20000, x0=[0, 0], thresh="steps", T_burn=Tb) for _ in range(n)]
    b = ParRepBatch(hs, autotune=False)
    b.run([T] * n, [500 + k for k in range(n)])
    assert b.status() == [0] * n
    Z = np.array([np.diag(h.fim()) for h in hs])
    mean, se = Z.mean(0), Z.std(0, ddof=1) / np.sqrt(n)
    assert np.all(np.abs(mean - exact) <= 4.5 * se + 1e-12 * exact), (mean, exact, se)
    r = parrep_uq(hs, np.tile(np.arange(3501.0), 32))
    np.testing.assert_allclose(np.diag(r["fim"]), mean, rtol=1e-9)
    assert sum(h.stats()["escapes"] for h in hs) > 0
