"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results -- jump counts, N*, K, X~, the dephased replica states -- must
be identical.  Time sums: the library keeps them in 64-bit fixed point with
2^-40 resolution (each holding time rounded once, sums exact), the oracle in
binary64 summed in (stage, step, replica) order.  A bin that received n
holding times therefore differs by at most n * 2^-41 from rounding plus the
binary64 summation error (about n * 2^-53 relative); the tolerance used is
atol = 4e-12 * (events in the run) + 1e-12 * T_end, rtol = 1e-12.

In the FP32 form the reaction choice is taken in binary32 on both sides, so
every integer result is still identical.  The holding time differs: the
kernel computes -logf(u) * RN(1/a0), the oracle -logf(u) / a0.  CUDA's and
the C library's logf may differ by 1 ulp, and the reciprocal-multiply rounds
twice where the division rounds once, so each tau agrees to within 3 ulp of
binary32 (relative 3 * 2^-24 < 2^-22); every time sum is bounded by
rtol = 2^-22 on top of the fixed-point term.

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
from paper_1705_06807_gb300.api import ParRepError

pytestmark = pytest.mark.gpu


F32_RTOL = 2.0**-22


def _tol(events, T_end, precision="f64"):
    t = 4e-12 * max(events, 1) + 1e-12 * T_end
    return t + (F32_RTOL * T_end if precision == "f32" else 0.0)


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
                     T_burn=T_burn, x0_uniform_hi=x0_uniform_hi, rer_cprime=rer)
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
    cg, co = g.cycle_log(), o["cycles"]
    assert len(cg) == len(co)
    for a, b in zip(cg, co):
        for k in ("cycle", "W", "ended", "decorr_steps", "dephase_steps", "n_star", "k", "x_tilde"):
            assert a[k] == b[k], (k, a, b)
        assert abs(a["T_s"] - b["T_s"]) <= rt * b["T_s"] + 1e-12 * T_end + 1e-9
    events = o["events_decorr"] + o["events_parallel_useful"]
    pre, post = g.histogram_raw()
    tol = _tol(events, T_end, prec)
    np.testing.assert_allclose(pre, o["hist_pre"], rtol=rt, atol=tol)
    np.testing.assert_allclose(post, o["hist_post"], rtol=rt, atol=tol)
    h = g.histogram()
    np.testing.assert_allclose(h, (o["hist_pre"] + o["hist_post"]) / T_end, rtol=rt, atol=tol / T_end)
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


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("spec,x0", [(K.schlogl_classic(), [85]), (K.toggle(alpha=20, n=2.5, hist_max=(63, 63)), [15, 2])])
def test_plain_ssa_matches_oracle(spec, x0, precision):
    T = 3.0 if spec["kind"] == "schlogl" else 40.0
    hg, evg, _ = parrep_ssa(spec, 37, x0, T, 11, precision=precision)
    ho, evo, _ = O.ssa_run(spec, 37, x0, T, 11, precision=precision)
    assert evg == evo
    rt = F32_RTOL if precision == "f32" else 1e-12
    np.testing.assert_allclose(hg, ho, rtol=rt, atol=_tol(evo, 37 * T, precision))
    assert abs(hg.sum() - 37 * T) < 1e-9 * 37 * T


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
