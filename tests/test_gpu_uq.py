"""Stationary UQ over independent runs (Sec. IV.B) through parrep_uq.

Parity: the same samples run on the CUDA path (binary64 form) and in the
oracle; the UQ of the device (window integrals Y_k, IAF, mean, FIM mean and
half widths, bounds) against the oracle's estimators on the oracle's own
runs.  The runs agree in every integer; their time sums differ by the
fixed-point rounding (at most 2^-41 per holding time) and by where the
T_burn cut falls, and the tolerances below carry those differences through
each estimator.

Statistics: the paper's Sec. V.A experiment at reduced sample count (V = 25
Schloegl, R = 100, n_c = n_p = 5000, windows [1e5, 2e5]) against the exact
IAF, mean, FIM and sensitivities of the birth-death chain.
"""
import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from oracle import uq as U
from paper_1705_06807_gb300 import ParRep, ParRepBatch, parrep_uq, configs as K
from paper_1705_06807_gb300.api import ParRepError

pytestmark = pytest.mark.gpu

V10 = K.schlogl_paper(V=10, hist_max=200, split=11)
TOG = K.toggle(alpha=20, n=2.5, hist_max=(63, 63))


def _cases(which):
    if which == "schlogl":
        return dict(spec=V10, R=16, tc=200, tp=200, T=300.0, Tb=100.0, x0=[3], thresh="steps",
                    f=np.arange(201.0), seeds=list(range(21, 33)))
    U_, V_ = np.meshgrid(np.arange(64.0), np.arange(64.0), indexing="ij")
    return dict(spec=TOG, R=24, tc=0.5, tp=0.5, T=40.0, Tb=10.0, x0=[15, 2], thresh="time",
                f=(U_ - 0.5 * V_).ravel(), seeds=list(range(5, 13)))


def _per_state_fim(spec):
    """Per-bin FIM rates sum_j lambda_j g_j g_j^T, shape (n_bins, l, l)."""
    c = np.asarray(spec["c"], dtype=float)
    if spec["kind"] == "schlogl":
        xs = np.arange(spec["hist_max"] + 1)
        lam, grad = E.schlogl_props(c, spec["s"], xs), E.schlogl_grad_log(c, xs)
    else:
        h0, h1 = spec["hist_max"]
        U_, V_ = np.meshgrid(np.arange(h0 + 1.0), np.arange(h1 + 1.0), indexing="ij")
        lam, grad = E.toggle_props(c, U_.ravel(), V_.ravel()), E.toggle_grad_log(c, U_.ravel(), V_.ravel())
    return np.einsum("jn,jan,jbn->nab", lam, grad, grad)


@pytest.mark.parametrize("which", ["schlogl", "toggle"])
def test_uq_matches_oracle(which):
    q = _cases(which)
    gpu, orc = [], []
    for s in q["seeds"]:
        g = ParRep(q["spec"], q["R"], q["tc"], q["tp"], x0=q["x0"], thresh=q["thresh"], T_burn=q["Tb"])
        g.run(q["T"], s)
        gpu.append(g)
        o = O.parrep_run(q["spec"], q["R"], q["tc"], q["tp"], q["T"], s, q["x0"], thresh=q["thresh"], T_burn=q["Tb"])
        assert o["status"] == 0
        orc.append(o)
        st = g.stats()
        assert st["events_parallel_useful"] == o["events_parallel_useful"] and st["cycles"] == o["n_cycles"]
    n, w, f = len(q["seeds"]), q["T"] - q["Tb"], q["f"]
    l = gpu[0].L
    rng = np.random.default_rng(1)
    D = rng.normal(size=(5, l))
    r = parrep_uq(gpu, f, directions=D)
    ref = U.uq(f, [o["hist_post"] for o in orc], [o["fim"] / w for o in orc], w, D)
    assert r["n_samples"] == n and r["window"] == w

    # time sums: the fixed-point rounding of every holding time (<= 2^-41 each)
    # and of the T_burn cut; the same bound as the histogram parity
    ev = max(o["events_decorr"] + o["events_parallel_useful"] for o in orc)
    t_sum = 4e-12 * ev + 1e-12 * q["T"]
    tolY = np.abs(f).max() * t_sum
    assert np.all(np.abs(r["Y"] - ref["Y"]) <= tolY + 1e-12 * np.abs(ref["Y"]))
    dev = np.abs(ref["Y"] - ref["Y"].mean()).sum()
    tol_iaf = (4.0 * tolY * dev + n * (2.0 * tolY) ** 2) / (w * (n - 1)) + 1e-10 * ref["iaf"]
    assert abs(r["iaf"] - ref["iaf"]) <= tol_iaf, (r["iaf"], ref["iaf"], tol_iaf)
    assert abs(r["mean_f"] - ref["mean_f"]) <= tolY / w + 1e-12 * abs(ref["mean_f"])

    # FIM: per sample the post-burn time of a bin moves by at most t_sum (cut
    # included), so each Z_k entry moves by at most t_sum max_x |rate| / w
    rates = np.abs(_per_state_fim(q["spec"])).max(axis=0)
    tolZ = t_sum * rates / w + 1e-9 * np.abs(ref["fim"])
    assert np.all(np.abs(r["fim"] - ref["fim"]) <= tolZ + 1e-12)
    tol_hw = 1.96 / np.sqrt(n) * 2.0 * tolZ * np.sqrt(n / (n - 1.0))
    assert np.all(np.abs(r["fim_half_width"] - ref["fim_half_width"]) <= tol_hw + 1e-9 * ref["fim_half_width"] + 1e-12)

    # bounds sqrt(tau v^T I v): relative error at most half the relative errors of tau and of v^T I v
    rel_tau = tol_iaf / ref["iaf"]
    d = np.diag(ref["fim"])
    rel_I = (np.diag(tolZ) + 1e-12) / np.maximum(d, 1e-300)
    unit = U.bounds(ref["iaf"], ref["fim"])
    assert np.all(np.abs(r["bounds"] - unit) <= 0.5 * (rel_tau + rel_I) * unit * 1.01 + 1e-12)
    qv = np.einsum("ka,ab,kb->k", D, ref["fim"], D)
    qtol = np.einsum("ka,ab,kb->k", np.abs(D), tolZ, np.abs(D)) + 1e-12
    rel_q = qtol / np.maximum(qv, 1e-300)
    assert np.all(np.abs(r["direction_bounds"] - ref["bounds"]) <= 0.5 * (rel_tau + rel_q) * ref["bounds"] * 1.01 + 1e-12)

    # the device reduction does not depend on the order of its launch: the same call twice
    r2 = parrep_uq(gpu, f, directions=D)
    assert r2["iaf"] == r["iaf"] and np.array_equal(r2["fim"], r["fim"]) and np.array_equal(r2["Y"], r["Y"])


def test_uq_rejects_bad_samples():
    a = ParRep(V10, 8, 50, 50, x0=[3], thresh="steps", T_burn=20.0)
    b = ParRep(V10, 8, 50, 50, x0=[3], thresh="steps", T_burn=20.0)
    c = ParRep(V10, 8, 50, 50, x0=[3], thresh="steps", T_burn=30.0)
    f = np.arange(201.0)
    a.run(80.0, 1)
    with pytest.raises(ParRepError):   # b has no run
        parrep_uq([a, b], f)
    b.run(80.0, 2)
    c.run(80.0, 3)
    with pytest.raises(ParRepError):   # one sample only
        parrep_uq([a], f)
    with pytest.raises(ParRepError):   # the same handle twice
        parrep_uq([a, a], f)
    with pytest.raises(ParRepError):   # windows differ (T_burn 20 vs 30)
        parrep_uq([a, b, c], f)
    with pytest.raises(ParRepError):   # f of the wrong length
        parrep_uq([a, b], f[:-1])
    t = ParRep(TOG, 8, 0.5, 0.5, x0=[15, 2], T_burn=20.0)
    t.run(80.0, 4)
    with pytest.raises(ParRepError):   # different networks
        parrep_uq([a, t], f)
    r = parrep_uq([a, b], f)
    assert r["n_samples"] == 2 and np.isfinite(r["iaf"]) and r["iaf"] >= 0.0


def test_uq_schlogl_v25_paper_experiment():
    """Sec. V.A's UQ experiment with 128 samples (the paper used 100): the
    FP32 form in one batch; IAF, mean and FIM against the exact chain, and
    the bounds above the exact sensitivities (Table III's comparison)."""
    net = K.schlogl_paper(V=25, hist_max=255)
    N, T, Tb = 128, 2e5, 1e5
    hs = [ParRep(net, 100, 5000, 5000, x0=[4], thresh="steps", precision="f32", T_burn=Tb) for _ in range(N)]
    b = ParRepBatch(hs)
    b.run([T] * N, [4242 + 31 * i for i in range(N)])
    assert b.status() == [0] * N
    x = np.arange(256.0)
    r = parrep_uq(hs, x, directions=np.eye(4))
    b.close()
    pi = E.schlogl_stationary(net["c"], net["s"], 255)
    Q, dQ = E.schlogl_generators(net["c"], net["s"], 255)
    tau = E.iaf_exact(Q, pi, x)
    S = E.stationary_sensitivity(Q, dQ, pi, x)
    F = E.fim_exact(E.schlogl_props(net["c"], net["s"], x), E.schlogl_grad_log(net["c"], x), pi)
    w = T - Tb
    # mean: standard error sqrt(tau / (w N)); IAF: a sample variance of N values
    assert abs(r["mean_f"] - pi @ x) < 4.5 * np.sqrt(tau / (w * N)) + 0.005 * (pi @ x)
    assert abs(r["iaf"] / tau - 1.0) < 4.0 * np.sqrt(2.0 / (N - 1))
    # FIM: within the estimate's own half widths (95%) widened to 4.5 standard
    # errors, plus the 2% ParRep bias allowance of the accuracy tests
    d, hw = np.diag(r["fim"]), np.diag(r["fim_half_width"])
    assert np.all(np.abs(d - np.diag(F)) <= 4.5 * hw / 1.96 + 0.02 * np.diag(F)), (d, np.diag(F))
    assert abs(d[2] - 200.0) < 1e-9
    assert np.allclose(r["direction_bounds"], r["bounds"], rtol=1e-12)
    assert np.all(r["bounds"] >= np.abs(S))
    # the bounds are loose on this multi-scale network, as Sec. V.A observes
    assert np.all(r["bounds"] > 5.0 * np.abs(S))
