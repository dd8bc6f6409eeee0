"""The genetic switch of Sec. V.B on the CUDA path (binary64 form).

State x0 = 2m + xi, x1 = p, six channels (Table IV with the switching rates
F, G).  Every integer result of a run -- event counts, cycles, escapes, the
cycle log, the final state -- equals the oracle's for the same seed; the
time sums agree to the fixed-point rounding (at most 2^-41 per holding time).
Plain SSA likewise.  The pooled histogram of a small bistable switch matches
its exact law.  The parts not built for this kind yet (FP32, FIM/RER,
batches, serving, UQ) refuse it with EINVAL.
"""
import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from paper_1705_06807_gb300 import ParRep, ParRepBatch, ParRepServer, parrep_ssa, parrep_uq
from paper_1705_06807_gb300.api import ParRepError

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


@pytest.mark.parametrize("name,spec,R,tc,tp,thresh,T,Tb,seed", CASES, ids=[c[0] for c in CASES])
def test_genetic_run_matches_oracle(name, spec, R, tc, tp, thresh, T, Tb, seed):
    o = O.parrep_run(spec, R, tc, tp, T, seed, [0, 0], thresh=thresh, T_burn=Tb)
    g = ParRep(spec, R, tc, tp, x0=[0, 0], thresh=thresh, T_burn=Tb)
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
    tol = 4e-12 * max(o["events_decorr"] + o["events_parallel_useful"], 1) + 1e-12 * T
    np.testing.assert_allclose(pre, o["hist_pre"], rtol=1e-12, atol=tol)
    np.testing.assert_allclose(post, o["hist_post"], rtol=1e-12, atol=tol)


def test_genetic_plain_ssa_matches_oracle():
    spec = _spec(E.genetic_paper_params(), 15, 3500, 512)
    hg, evg, _ = parrep_ssa(spec, 9, [0, 0], 3.0, 17, precision="f64")
    ho, evo, _ = O.ssa_run(spec, 9, [0, 0], 3.0, 17)
    assert evg == evo
    np.testing.assert_allclose(hg, ho, rtol=1e-12, atol=4e-12 * evo + 1e-12 * 27.0)


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


def test_genetic_parts_not_built_refuse_it():
    spec = _spec(SMALL, 16, 250, 13)
    g = ParRep(spec, 16, 50, 50, x0=[0, 0], thresh="steps", precision="f32")
    with pytest.raises(ParRepError):
        g.run(10.0, 1)
    with pytest.raises(ParRepError):
        parrep_ssa(spec, 1, [0, 0], 1.0, 1, precision="f32")
    g = ParRep(spec, 16, 50, 50, x0=[0, 0], thresh="steps", T_burn=2.0)
    g.run(10.0, 1)
    with pytest.raises(ParRepError):
        g.fim()
    with pytest.raises(ParRepError):
        ParRepBatch([g])
    h = ParRep(spec, 16, 50, 50, x0=[0, 0], thresh="steps", T_burn=2.0)
    h.run(10.0, 2)
    with pytest.raises(ParRepError):
        parrep_uq([g, h], np.arange(34 * 251.0))
    srv = ParRepServer(precision="f64", arena_bytes=8 << 20)
    with pytest.raises(ParRepError):
        srv.submit(spec, 16, 50, 50, 10.0, 1, x0=[0, 0], thresh="steps")
    srv.close()
