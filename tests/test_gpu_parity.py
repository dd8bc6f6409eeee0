"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results -- jump counts, N*, K, X~, the dephased replica states, and
per-trajectory reaction sequences and states of the plain SSA -- must be
identical.

Time sums.  The library rounds each holding time once to 64-bit fixed point
with 2^-40 resolution and sums exactly; the oracle sums binary64 in (stage,
step, replica) order.  For a bin that received n holding times with total h:
  * fixed-point rounding: at most n * 2^-41;
  * the holding time itself: -log(u)/a0 with CUDA's and the C library's log
    may differ by an ulp, so each tau agrees to 2^-51 relative (binary64); in
    the FP32 form the kernel computes -logf(u) * RN(1/a0) against the
    oracle's -logf(u) / a0 -- logf may differ by 1 ulp and the reciprocal
    multiply rounds twice where the division rounds once, so each tau agrees
    to 3 ulp of binary32, below 2^-22 relative;
  * the oracle's binary64 summation: at most n * 2^-53 * h.
So |h_gpu - h_oracle| <= n 2^-41 + (rt + n 2^-53) h, rt = 2^-51 or 2^-22,
with n taken per bin from the oracle's own counts.  The same bound with n =
all contributions so far holds for a clock T_s.  A contribution cut at T_end,
or split at T_burn, is cut at a clock that differs by that clock bound, so
the (at most two) bins that hold a cut may differ by that much more.

The FIM and RER are linear in the post-burn histogram, h -> sum_x r(x) h(x)
with per-state rates r(x) >= 0 (the RER and FIM integrands of Appendix A).  Two cuts move
holding time between bins rather than scaling it: the step that crosses
T_burn is split at a running sum that agrees to rtol * T_burn, and the step
cut at T_end keeps T_end - T_s with T_s agreeing to rtol * T_end.  So in the
FP32 form |dF| <= rtol * |F| + rtol * (T_burn + T_end) / span * max_x r(x),
the maximum over the states either side visited after T_burn.
"""
import numpy as np
import pytest

import oracle as O
from oracle import exact as X
from paper_1705_06807_gb300 import ParRep, configs as K, parrep_philox, parrep_ssa
from paper_1705_06807_gb300.api import ParRepError, parrep_ssa_trace

pytestmark = pytest.mark.gpu


F32_RTOL = 2.0**-22
F64_RTOL = 2.0**-51


def _rt(precision):
    return F32_RTOL if precision == "f32" else F64_RTOL


def _bin_bound(n, h, precision):
    """Per-bin bound on |h_gpu - h_oracle| for n holding times summing to h."""
    n = np.asarray(n, dtype=np.float64)
    return n * 2.0**-41 + (_rt(precision) + n * 2.0**-53) * np.abs(np.asarray(h, dtype=np.float64))


def _clock_bound(n, T, precision):
    """Bound on the difference of two clocks after n contributions summing to T."""
    return n * 2.0**-41 + (_rt(precision) + n * 2.0**-53) * T


def _assert_bins(actual, desired, counts, precision, cut_slack=0.0, max_cut_bins=0):
    """Every bin within its own bound; at most max_cut_bins bins (those that
    hold a cut contribution) may exceed it, by at most cut_slack."""
    actual, desired = np.asarray(actual, dtype=float), np.asarray(desired, dtype=float)
    excess = np.abs(actual - desired) - _bin_bound(counts, desired, precision)
    over = excess > 0
    assert over.sum() <= max_cut_bins, f"{int(over.sum())} bin(s) beyond their bound; worst {excess.max():.3e}"
    if over.any():
        assert excess.max() <= cut_slack, f"cut bin beyond {cut_slack:.3e}: {excess.max():.3e}"


def _assert_close(actual, desired, rtol, atol):
    """|actual - desired| <= rtol |desired| + atol elementwise (atol may be an array)."""
    actual, desired = np.asarray(actual, dtype=float), np.asarray(desired, dtype=float)
    err = np.abs(actual - desired)
    bound = rtol * np.abs(desired) + atol
    bad = err > bound
    assert not bad.any(), f"{int(bad.sum())} element(s) beyond tolerance; worst excess {float((err - bound).max()):.3e}"


def _state_rates(spec, cprime=None):
    """Per-bin FIM rates (n_bins, l, l) and RER rates (k, n_bins) of a network,
    laid out like the histogram (bin = x0 * (hist_max1 + 1) + x1)."""
    c = np.asarray(spec["c"], dtype=float)
    if spec["kind"] == "schlogl":
        xs = np.arange(int(spec["hist_max"][0] if np.ndim(spec["hist_max"]) else spec["hist_max"]) + 1)
        lam = X.schlogl_props(c, spec["s"], xs)
        grad = X.schlogl_grad_log(c, xs)
        props = lambda cc: X.schlogl_props(cc, spec["s"], xs)
    else:
        h0, h1 = spec["hist_max"]
        U, V = np.meshgrid(np.arange(h0 + 1), np.arange(h1 + 1), indexing="ij")
        U, V = U.ravel().astype(float), V.ravel().astype(float)
        lam = X.toggle_props(c, U, V)
        grad = X.toggle_grad_log(c, U, V)
        props = lambda cc: X.toggle_props(cc, U, V)
    fim = np.einsum("jn,jan,jbn->nab", lam, grad, grad)
    rer = []
    for cp in ([] if cprime is None else cprime):
        lp = props(np.asarray(cp, dtype=float))
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(lam > 0, lam * np.log(lam / lp), 0.0) - lam + lp
        rer.append(t.sum(axis=0))
    return fim, np.array(rer)


def run_both(spec, R, tc, tp, T_end, seed, x0, *, thresh="time", precision="f64", fv_group=32, T_burn=0.0,
             x0_uniform_hi=0, block_threads=0, chunk_steps=0, rer=None):
    o = O.parrep_run(spec, R, tc, tp, T_end, seed, x0, thresh=thresh, precision=precision, fv_group=fv_group,
                     T_burn=T_burn, x0_uniform_hi=x0_uniform_hi, rer_cprime=rer, counts=True)
    g = ParRep(spec, R, tc, tp, x0=x0, x0_uniform_hi=x0_uniform_hi, thresh=thresh, precision=precision,
               fv_group=fv_group, T_burn=T_burn, block_threads=block_threads, chunk_steps=chunk_steps)
    g.precision = precision
    rc = g.run_status(T_end, seed)
    return o, g, rc


def assert_parity(o, g, rc, T_end, *, rer=None):
    prec = getattr(g, "precision", "f64")
    rt = F32_RTOL if prec == "f32" else 1e-12
    assert rc == o["status"] == 0, (rc, o["status"])
    st = g.stats()
    assert st["T_s"] == T_end and o["T_s"] == T_end
    assert st["x0"] == o["x0"]
    assert st["x_final"] == o["x_final"]
    assert st["cycles"] == o["n_cycles"]
    assert st["escapes"] == o["escapes"]
    assert st["events_decorr"] == o["events_decorr"]
    assert st["events_dephase"] == o["events_dephase"]
    assert st["events_parallel_useful"] == o["events_parallel_useful"]
    events = o["events_decorr"] + o["events_parallel_useful"]
    cg, co = g.cycle_log(), o["cycles"]
    assert len(cg) == len(co)
    for a, b in zip(cg, co):
        for k in ("cycle", "W", "ended", "decorr_steps", "dephase_steps", "n_star", "k", "x_tilde"):
            assert a[k] == b[k], (k, a, b)
        assert abs(a["T_s"] - b["T_s"]) <= _clock_bound(events, b["T_s"], prec), (a["T_s"], b["T_s"])
    pre, post = g.histogram_raw()
    cut = _clock_bound(events, T_end, prec)
    # pre: the T_burn split; post: the split and the T_end cut
    _assert_bins(pre, o["hist_pre"], o["count_pre"], prec, cut, 1)
    _assert_bins(post, o["hist_post"], o["count_post"], prec, cut, 2)
    h = g.histogram()
    _assert_bins(h * T_end, o["hist_pre"] + o["hist_post"], o["count_pre"] + o["count_post"], prec, 2 * cut, 2)
    span = T_end - g._opt.T_burn
    if span > 0:
        F = g.fim()
        Fo = o["fim"] / span
        frt = max(rt, 1e-9)
        fr, rr = _state_rates(g.spec, rer)
        seen = (post > 0) | (o["hist_post"] > 0)
        cut = frt * (g._opt.T_burn + T_end) / span
        _assert_close(F, Fo, frt, 1e-12 + cut * np.abs(fr[seen]).max(axis=0))
        if rer is not None:
            _assert_close(g.rer(rer), o["rer"] / span, frt, 1e-12 + cut * rr[:, seen].max(axis=1))


# ---------------------------------------------------------------------------
# generator and plain SSA
# ---------------------------------------------------------------------------
def test_philox_device_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    out = parrep_philox(ctr, key)
    ref = np.stack([O.philox(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(out, ref)
    assert list(out[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


SSA_CASES = [(K.schlogl_classic(), [85]), (K.toggle(alpha=20, n=2.5, hist_max=(63, 63)), [15, 2])]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("spec,x0", SSA_CASES)
def test_plain_ssa_trajectories_are_bit_exact(spec, x0, precision):
    """Per trajectory, the reaction index sequence and the integer states of
    the direct method (Sec. II.A) are identical to the oracle's for the same
    Philox stream; each holding time agrees to its 2^-41 fixed-point rounding
    plus the log / reciprocal ulps."""
    n, steps = 40, 600
    J, xs, tau, nj, xf = parrep_ssa_trace(spec, n, x0, 1e6, 23, steps, precision=precision)
    assert np.all(nj == steps)
    for t in range(n):
        Jo, xo, to = O.ssa_trace(spec, x0, 23, t, steps, precision=precision)
        assert np.array_equal(J[t], Jo), t
        assert np.array_equal(xs[t, :, : len(x0)], xo[:, : len(x0)]), t
        assert np.all(np.abs(tau[t] - to) <= 2.0**-41 + _rt(precision) * to), t
        assert tuple(xf[t, : len(x0)]) == tuple(xo[-1, : len(x0)])


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("spec,x0", SSA_CASES)
def test_plain_ssa_matches_oracle(spec, x0, precision):
    """Histograms, jump counts and final states of parrep_ssa against the
    oracle's plain SSA to T_end, with each bin held to its own rounding bound
    (its holding-time count comes from the trajectories' jump records)."""
    T = 3.0 if spec["kind"] == "schlogl" else 40.0
    n = 37
    hg, evg, _ = parrep_ssa(spec, n, x0, T, 11, precision=precision)
    ho, evo, xfo = O.ssa_run(spec, n, x0, T, 11, precision=precision)
    assert evg == evo
    J, xs, tau, nj, xf = parrep_ssa_trace(spec, n, x0, T, 11, 8192, precision=precision)
    assert int(nj.sum()) == evo and np.all(nj < 8192)
    assert np.array_equal(xf[:, : len(x0)], xfo[:, : len(x0)])
    # holding times per bin: the pre-jump states, plus each trajectory's last
    # (truncated) stay at its final state
    ys = spec["hist_max"][1] + 1 if np.ndim(spec["hist_max"]) else 1
    counts = np.zeros(hg.size, dtype=np.int64)
    for t in range(n):
        pre = np.concatenate([[list(x0) + [0] * (2 - len(x0))], xs[t, : nj[t] - 1]]) if nj[t] else np.zeros((0, 2))
        b = (pre[:, 0] * ys + (pre[:, 1] if ys > 1 else 0)).astype(np.int64)
        counts += np.bincount(b, minlength=hg.size)
        counts[xf[t, 0] * ys + (xf[t, 1] if ys > 1 else 0)] += 1
    slack = max(_clock_bound(int(k), T, precision) for k in nj)
    _assert_bins(hg, ho, counts, precision, slack * n, n)
    assert abs(hg.sum() - n * T) <= _clock_bound(evo + n, n * T, precision)


# ---------------------------------------------------------------------------
# full ParRep runs
# ---------------------------------------------------------------------------
V10 = K.schlogl_paper(V=10, hist_max=200, split=11)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("R,G,S", [(48, 16, 32), (64, 32, 256), (33, 8, 7), (1, 32, 64)])
def test_parrep_steps_mode_paper_schlogl(precision, R, G, S):
    """Paper's form of Algorithm 1 (jump-count thresholds), many cycles."""
    cp = np.array([V10["c"]] * 2, dtype=float)
    cp[0, 0] *= 1.1
    cp[1, 3] *= 0.9
    o, g, rc = run_both(V10, R, 300, 300, 300.0, 7 + R, [2], thresh="steps", precision=precision, fv_group=G,
                        T_burn=100.0, chunk_steps=S, rer=cp)
    assert o["escapes"] >= 3
    assert_parity(o, g, rc, 300.0, rer=cp)


@pytest.mark.parametrize("tc", [150, 301, 2000])
def test_parrep_fp32_decorrelation_rounds_in_the_wide_range(tc):
    """The FP32 staged decorrelation where its block-parallel chain takes
    whole windows (states 64 or more from both ends of the range): the classic
    Schloegl network at V = 0.5 (range 0 .. 750, split at 125), whose many
    cycles decorrelate mostly above state 64, with STEPS thresholds whose
    rounds end at various points of a window, against the oracle."""
    spec = K.schlogl_classic(V=0.5)
    o, g, rc = run_both(spec, 64, tc, 300, 200.0, 11 + tc, [150], thresh="steps", precision="f32", T_burn=20.0)
    assert o["n_cycles"] >= 5
    assert_parity(o, g, rc, 200.0)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_parrep_time_mode_classic_schlogl(precision):
    """The rate constants (0.03, 1e-4, 200, 3.5) with time thresholds 1, 1."""
    spec = K.schlogl_classic()
    o, g, rc = run_both(spec, 64, 1.0, 1.0, 60.0, 3, [85], precision=precision, T_burn=20.0, chunk_steps=128)
    assert_parity(o, g, rc, 60.0)


def test_parrep_time_mode_escapes_from_saddle():
    """Start at the saddle so that several escapes happen quickly."""
    spec = K.schlogl_classic()
    o, g, rc = run_both(spec, 96, 0.2, 0.2, 8.0, 5, [250], chunk_steps=64)
    assert o["n_cycles"] >= 2
    assert_parity(o, g, rc, 8.0)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_parrep_toggle(precision):
    spec = K.toggle(alpha=20.0, n=2.5, hist_max=(63, 63))
    cp = np.array([spec["c"]], dtype=float)
    cp[0, 1] = 2.0
    o, g, rc = run_both(spec, 40, 0.5, 0.5, 60.0, 9, [15, 2], precision=precision, T_burn=10.0, chunk_steps=64,
                        rer=cp)
    assert_parity(o, g, rc, 60.0, rer=cp)


def test_parrep_x0_uniform_draw():
    spec = K.schlogl_classic()
    o, g, rc = run_both(spec, 64, 1.0, 1.0, 5.0, 123, [0], x0_uniform_hi=1000)
    assert_parity(o, g, rc, 5.0)


def test_parrep_full_launch_config_first_cycles():
    """The full-size workload (4096 replicas, x0 uniform on [0, 1000], time
    thresholds 1/1) in the benchmark's launch configuration, over the first
    80 time units -- the sample of the long run that the oracle can follow."""
    c = K.C2
    o, g, rc = run_both(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], 80.0, 0, c["x0"],
                        x0_uniform_hi=c["x0_uniform_hi"], T_burn=40.0)
    assert_parity(o, g, rc, 80.0)


def test_parrep_full_launch_config_first_cycles_fp32():
    """The benchmarked form: binary32 propensities with the library's default
    FP32 launch plan for 4096 replicas (32 owner threads + 352 helpers per
    block, 128 blocks, chunks doubling up to about 2048 lockstep steps), x0 uniform
    on [0, 1000], time thresholds 1/1, over the first 3000 time units (four
    escapes, then a parallel step of 4562 lockstep steps cut by T_end),
    against the oracle's binary32 mode."""
    c = K.C2
    o, g, rc = run_both(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], 3000.0, 0, c["x0"],
                        x0_uniform_hi=c["x0_uniform_hi"], T_burn=1500.0, precision="f32")
    st = g.stats()
    assert st["grid_blocks"] == 128 and st["block_threads"] == 384 and 2048 <= st["chunk_steps"] <= 2048 + 128
    assert o["escapes"] >= 3
    assert max(cy["n_star"] for cy in o["cycles"]) > 2048
    assert_parity(o, g, rc, 3000.0)


@pytest.mark.parametrize("T_end", [0.0, 1e-6, 0.01])
def test_parrep_tiny_horizons(T_end):
    spec = K.schlogl_classic()
    o, g, rc = run_both(spec, 64, 1.0, 1.0, T_end, 1, [85])
    assert rc == 0 and o["status"] == 0
    st = g.stats()
    # T_end is taken on the 2^-40 grid of the fixed-point clock
    assert abs(st["T_s"] - T_end) <= 2.0**-41
    assert st["cycles"] == o["n_cycles"]
    assert st["events_decorr"] == o["events_decorr"]
    pre, post = g.histogram_raw()
    np.testing.assert_allclose(pre + post, o["hist_pre"] + o["hist_post"], atol=1e-12)


def test_chunk_and_block_shape_do_not_change_results():
    """The cut is exact, so the chunk length and the block size are invisible:
    all fixed-point sums agree to the last bit."""
    res = []
    # max_blocks = 1: one block takes all three groups of 32 replicas in turn
    for S, B, M in [(5, 32, 0), (64, 128, 0), (512, 64, 0), (64, 32, 1), (37, 32, 2)]:
        g = ParRep(V10, 77, 200, 200, x0=[2], thresh="steps", fv_group=16, T_burn=50.0, chunk_steps=S,
                   block_threads=B, max_blocks=M)
        g.run(150.0, 99)
        pre, post = g.histogram_raw()
        res.append((pre, post, g.cycle_log(), g.stats()["events_parallel_useful"]))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
        assert r[2] == res[0][2] and r[3] == res[0][3]


def test_dephase_bit_exact():
    o_states, steps, _ = O.dephase(V10, 100, [30], 1, 4, 500, 17, thresh="steps", fv_group=8)
    g = ParRep(V10, 100, 10, 500, thresh="steps", fv_group=8)
    s = g.dephase([30], 1, 4, 17)
    assert np.array_equal(s, o_states)


def test_dephase_time_mode_bit_exact():
    spec = K.schlogl_classic()
    o_states, steps, _ = O.dephase(spec, 70, [560], 1, 2, 0.3, 5, fv_group=32)
    g = ParRep(spec, 70, 1.0, 0.3, fv_group=32)
    assert np.array_equal(g.dephase([560], 1, 2, 5), o_states)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_served_requests_match_the_oracle(precision):
    """Requests through the continuous-batching server, several in flight at
    once, checked directly against the oracle's Algorithm 1 (not only
    against solo GPU runs): integers identical, histograms within the
    per-bin bounds, FIM and RER within the contraction bound."""
    from paper_1705_06807_gb300 import ParRepServer

    tg = K.toggle(alpha=20, n=2.5, hist_max=(63, 63))
    cp = np.array([V10["c"]] * 2, dtype=float)
    cp[0, 0] *= 1.1
    cp[1, 3] *= 0.9
    reqs = [dict(spec=V10, R=48, tc=300, tp=300, T_end=200.0, seed=41, x0=[2], thresh="steps", G=16, Tb=50.0, rer=cp),
            dict(spec=tg, R=40, tc=0.5, tp=0.5, T_end=40.0, seed=9, x0=[15, 2], thresh="time", G=32, Tb=10.0,
                 rer=None),
            dict(spec=K.schlogl_classic(), R=256, tc=1.0, tp=1.0, T_end=30.0, seed=5, x0=[250], thresh="time", G=32,
                 Tb=5.0, rer=None)]
    srv = ParRepServer(precision=precision)
    ids = [srv.submit(q["spec"], q["R"], q["tc"], q["tp"], q["T_end"], q["seed"], x0=q["x0"], thresh=q["thresh"],
                      fv_group=q["G"], T_burn=q["Tb"], rer=q["rer"]) for q in reqs]
    res = [srv.result(i) for i in ids]
    srv.close()
    for q, r in zip(reqs, res):
        o = O.parrep_run(q["spec"], q["R"], q["tc"], q["tp"], q["T_end"], q["seed"], q["x0"], thresh=q["thresh"],
                         precision=precision, fv_group=q["G"], T_burn=q["Tb"], rer_cprime=q["rer"], counts=True)
        assert r["status"] == 0 == o["status"]
        st = r["stats"]
        for k, ko in (("cycles", "n_cycles"), ("escapes", "escapes"), ("events_decorr", "events_decorr"),
                      ("events_dephase", "events_dephase"), ("events_parallel_useful", "events_parallel_useful"),
                      ("x_final", "x_final"), ("x0", "x0")):
            assert st[k] == o[ko], (k, st[k], o[ko])
        assert st["T_s"] == q["T_end"]
        events = o["events_decorr"] + o["events_parallel_useful"]
        cut = _clock_bound(events, q["T_end"], precision)
        _assert_bins(r["hist"] * q["T_end"], o["hist_pre"] + o["hist_post"], o["count_pre"] + o["count_post"],
                     precision, 2 * cut, 2)
        span = q["T_end"] - q["Tb"]
        frt = max(_rt(precision), 1e-9)
        fr, rr = _state_rates(q["spec"], q["rer"])
        hp = o["hist_post"]
        seen = hp > 0
        c = frt * (q["Tb"] + q["T_end"]) / span
        _assert_close(r["fim"], o["fim"] / span, frt, 1e-12 + c * np.abs(fr[seen]).max(axis=0))
        if q["rer"] is not None:
            _assert_close(r["rer"], o["rer"] / span, frt, 1e-12 + c * rr[:, seen].max(axis=1))


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_range_error_matches_oracle():
    spec = dict(K.schlogl_classic(), hist_max=120)
    o, g, rc = run_both(spec, 32, 1.0, 1.0, 100.0, 0, [85])
    assert o["status"] == O.OR_ERANGE and rc == -5


def test_invalid_arguments():
    spec = K.schlogl_classic()
    with pytest.raises(ParRepError):
        ParRep(spec, 0, 1.0, 1.0, x0=[85])
    with pytest.raises(ParRepError):
        ParRep(spec, 8, 1.0, 1.0, x0=[5000])
    g = ParRep(spec, 8, 1.0, 1.0, x0=[85])
    assert g.run_status(-1.0, 0) == -1
    assert g.run_status(1e8, 0) == -1
    with pytest.raises(ParRepError):
        g.histogram()  # no completed run
    with pytest.raises(ParRepError):
        g.set_options(fv_group=3)


def test_bounded_wait_times_out_and_context_survives():
    """Fault injection on the host side of the protocol: block 0 leaves at a
    grid barrier, the other blocks' bounded wait expires and the run returns
    ETIMEOUT; the next run on the same context is normal."""
    spec = K.schlogl_classic()
    g = ParRep(spec, 256, 1.0, 1.0, x0=[85], block_threads=64, wait_timeout_s=0.2, debug_stall_barrier=2)
    assert g.run_status(5.0, 1) == -4
    g.set_options(block_threads=64)
    g.run(5.0, 1)
    assert g.stats()["T_s"] == 5.0


@pytest.mark.parametrize("spec,x0", [(V10, [2]), (K.toggle(alpha=20.0, n=2.5, hist_max=(63, 63)), [15, 2])])
def test_fp32_staged_path_is_shape_invariant(spec, x0):
    """The FP32 form stages 32 steps at a time and splits holding times into
    32-bit limbs; none of that may change a bit of the fixed-point sums, the
    cycle log or the event counts across chunk lengths and block sizes."""
    thresh, tc = ("steps", 200) if spec["kind"] == "schlogl" else ("time", 0.5)
    res = []
    for S, B, M in [(32, 64, 0), (256, 256, 0), (1024, 128, 0), (64, 128, 1), (96, 384, 2)]:
        g = ParRep(spec, 77, tc, tc, x0=x0, thresh=thresh, precision="f32", fv_group=16, T_burn=30.0,
                   chunk_steps=S, block_threads=B, max_blocks=M)
        g.run(90.0, 99)
        pre, post = g.histogram_raw()
        res.append((pre, post, g.cycle_log(), g.stats()["events_parallel_useful"]))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
        assert r[2] == res[0][2] and r[3] == res[0][3]


@pytest.mark.parametrize("case", ["v10_steps", "toggle_time", "classic_time"])
def test_fp32_direct_layout_equals_staged(case):
    """The two kernel layouts of the FP32 form -- staged (owner threads fed by
    helper warps) and direct (one thread per replica at high occupancy) --
    take every decision and round every holding time identically: the
    fixed-point sums, the cycle logs and the event counts agree bit for bit,
    and the direct layout matches the oracle's binary32 mode."""
    spec, x0, tc, thresh, T, R = {
        "v10_steps": (V10, [2], 200, "steps", 120.0, 300),
        "toggle_time": (K.toggle(alpha=20.0, n=2.5, hist_max=(63, 63)), [15, 2], 0.5, "time", 60.0, 200),
        "classic_time": (K.schlogl_classic(), [250], 0.3, "time", 12.0, 700),
    }[case]
    out = []
    for layout in ("staged", "direct"):
        g = ParRep(spec, R, tc, tc, x0=x0, thresh=thresh, precision="f32", fv_group=16, T_burn=T / 4,
                   f32_layout=layout)
        g.run(T, 13)
        pre, post = g.histogram_raw()
        out.append((pre, post, g.cycle_log(), g.stats()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    for k in ("events_decorr", "events_dephase", "events_parallel_useful", "escapes", "x_final", "T_s"):
        assert out[0][3][k] == out[1][3][k], k
    o, g, rc = run_both(spec, R, tc, tc, T, 13, x0, thresh=thresh, precision="f32", fv_group=16, T_burn=T / 4)
    g.set_options(thresh=thresh, precision="f32", fv_group=16, T_burn=T / 4, f32_layout="direct")
    g.precision = "f32"
    rc = g.run_status(T, 13)
    assert_parity(o, g, rc, T)


def test_fp32_direct_layout_is_shape_invariant():
    """Block size and the cap on blocks (several groups of replicas per
    block) do not change a bit of the direct layout's results."""
    res = []
    for B, M in [(256, 0), (128, 0), (64, 0), (128, 1), (256, 2)]:
        g = ParRep(V10, 777, 200, 200, x0=[2], thresh="steps", precision="f32", fv_group=32, T_burn=30.0,
                   chunk_steps=96, block_threads=B, max_blocks=M, f32_layout="direct")
        g.run(90.0, 99)
        pre, post = g.histogram_raw()
        res.append((pre, post, g.cycle_log(), g.stats()["events_parallel_useful"]))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
        assert r[2] == res[0][2] and r[3] == res[0][3]


@pytest.mark.parametrize("spec,x0", [(V10, [2]), (K.toggle(alpha=20.0, n=2.5, hist_max=(63, 63)), [15, 2])])
def test_fp32_pipelined_equals_serial_stages(spec, x0):
    """The owner/helper overlap only reorders work between warps: the results
    must equal those of the unpipelined stages bit for bit."""
    thresh, tc = ("steps", 200) if spec["kind"] == "schlogl" else ("time", 0.5)
    out = []
    for serial in (0, 1):
        g = ParRep(spec, 100, tc, tc, x0=x0, thresh=thresh, precision="f32", fv_group=16, T_burn=25.0,
                   serial_stages=serial)
        g.run(80.0, 5)
        pre, post = g.histogram_raw()
        out.append((pre, post, g.cycle_log(), g.stats()["events_parallel_useful"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]


@pytest.mark.parametrize("R,precision,layout,want", [
    (4096, "f32", "staged", 2112),   # 2048 rounded up to whole 96-step sub-chunks
    (8192, "f32", "staged", 1024),   # 2048 x 8192 replica-steps exceed 2^23; 64 owners, 32-step sub-chunks
    (16384, "f32", "direct", 256),
    (65536, "f32", "direct", 128),
    (4096, "f64", "auto", 256),
    (65536, "f64", "auto", 128),
])
def test_default_chunk_length_follows_the_replica_count(R, precision, layout, want):
    """The default chunk between escape votes: 2048 lockstep steps in the FP32
    staged layout and 256 with one thread per replica, halved (down to 128)
    while a chunk would hold more than 2^23 replica-steps."""
    g = ParRep(K.schlogl_classic(), R, 1.0, 1.0, x0=[100], precision=precision, f32_layout=layout)
    assert g.run_status(0.05, 1) == 0
    assert g.stats()["chunk_steps"] == want
