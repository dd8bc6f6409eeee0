"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here touches the CUDA path.  Each test names the passage or the
textbook fact it checks; the statistical ones use batch means over independent
seeds and fail beyond 4.5 standard errors.
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from paper_1705_06807_gb300 import configs as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _z(samples, target):
    s = np.asarray(samples, dtype=np.float64)
    se = s.std(ddof=1) / np.sqrt(len(s))
    return abs(s.mean() - target) / se


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            out = O.philox(v[0:4], v[4:6])
            assert list(out) == v[6:10]
            n += 1
    assert n == 3


def test_uniform_constructions_are_open_interval_and_exact():
    lo = O.u01_f64(0, 0)
    hi = O.u01_f64(0xFFFFFFFF, 0xFFFFFFFF)
    assert lo == 2.0**-53 and hi == 1.0 - 2.0**-53
    assert O.u01_f32(0) == np.float32(2.0**-24)
    assert O.u01_f32(0xFFFFFFFF) == np.float32(1.0 - 2.0**-24)
    # 52 bits: wa supplies the top 32, wb the next 20
    assert O.u01_f64(1, 0) == (2.0**20 + 0.5) * 2.0**-52
    assert O.u01_f64(0, 1 << 12) == 1.5 * 2.0**-52


# ---------------------------------------------------------------------------
# exact references pinned to the paper's printed values
# ---------------------------------------------------------------------------
def _golden_paper():
    d = {}
    with open(os.path.join(GOLDEN, "paper_schlogl_v25.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v, hw = line.split()[:3]
            d[k] = (float(v), float(hw))
    return d


def test_schlogl_table_reading_reproduces_paper_saddle():
    """Table I with a=1, b=2, c=(3,0.6,0.25,2.95), V=25: the unstable point of
    the rate equation times V is 25.9649 (Fig. 1 caption)."""
    g = _golden_paper()
    n = K.schlogl_paper()
    roots = E.rre_fixed_points(n["c"], n["s"])
    assert len(roots) == 3
    v, hw = g["saddle_population"]
    assert abs(roots[1] - v) <= hw


def test_product_formula_matches_generator_solve():
    """Birth-death product formula against a direct solve of pi Q = 0 (Eq. 1)."""
    n = K.schlogl_paper(hist_max=149)
    x = np.arange(150)
    lam = E.schlogl_props(n["c"], n["s"], x)
    pi1 = E.bd_stationary(lam[0] + lam[2], lam[1] + lam[3])
    Q = E.generator(lam[0] + lam[2], lam[1] + lam[3])
    pi2 = E.stationary_dense(Q)
    assert np.max(np.abs(pi1 - pi2)) < 1e-10
    assert abs(pi1.sum() - 1.0) < 1e-12


def test_exact_fim_reproduces_paper_table():
    """Path-space FIM of Table II from the exact stationary law: I_33 = 200
    exactly (lambda_3 is constant); I_11 and I_44 inside the paper's confidence
    half-widths; I_22 within 3% (the paper's estimate sits 2.6% above the exact
    value, outside its own half-width)."""
    g = _golden_paper()
    n = K.schlogl_paper(hist_max=400)
    x = np.arange(401)
    pi = E.schlogl_stationary(n["c"], n["s"], 400)
    lam = E.schlogl_props(n["c"], n["s"], x)
    F = E.fim_exact(lam, E.schlogl_grad_log(n["c"], x), pi)
    assert np.allclose(F - np.diag(np.diag(F)), 0.0)
    assert abs(F[2, 2] - 200.0) < 1e-10
    for i, key in [(0, "fim_11"), (3, "fim_44")]:
        v, hw = g[key]
        assert abs(F[i, i] - v) <= 2 * hw, (key, F[i, i], v)
    assert abs(F[1, 1] / g["fim_22"][0] - 1.0) < 0.03
    # the grad-lambda form printed in the Sec. IV text would give
    # I_33 = lambda_3 (d lambda_3 / d c_3)^2 = 12.5 * 50^2 = 31250, not 200
    assert abs(lam[2, 0] * n["s"][2] ** 2 - 31250.0) < 1e-9


def test_toggle_cme_reduces_to_independent_poisson():
    """With Hill exponent 0 the production rates are constant alpha/2, so the
    truncated CME must give the product of two Poisson(alpha/(2 delta)) laws."""
    from scipy.stats import poisson

    c = [12.0, 0.0, 1.5, 12.0, 0.0, 1.5]
    pi = E.toggle_stationary(c, 40, 40)
    m = 12.0 / 2.0 / 1.5
    p = poisson.pmf(np.arange(41), m)
    assert np.max(np.abs(pi - np.outer(p, p) / np.outer(p, p).sum())) < 1e-10


def test_toggle_cme_symmetry():
    """The symmetric toggle's law is symmetric under U <-> V.  The two wells
    exchange mass only every ~1e7 time units, so the sparse solve is
    ill-conditioned and holds the symmetry to ~1e-7 relative."""
    pi = E.toggle_stationary(K.toggle()["c"], 100, 100)
    assert np.max(np.abs(pi - pi.T)) < 1e-6 * pi.max()
    U, V = np.meshgrid(np.arange(101), np.arange(101), indexing="ij")
    assert abs(pi[U > V].sum() - pi[U < V].sum()) < 1e-6


# ---------------------------------------------------------------------------
# the oracle's SSA
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ssa_immigration_death_is_poisson(precision):
    """Immigration-death (c1 = c2 = 0): stationary law Poisson(k_in/k_out)."""
    from scipy.stats import poisson

    net = K.immigration_death(20.0, 1.0, hist_max=120)
    means = []
    tot = np.zeros(121)
    for seed in range(16):
        h, ev, _ = O.ssa_run(net, 1, [20], 12500.0, 1000 + seed, precision=precision)
        tot += h
        means.append((h * np.arange(121)).sum() / h.sum())
    p = tot / tot.sum()
    ex = poisson.pmf(np.arange(121), 20.0)
    assert 0.5 * np.abs(p - ex).sum() < 0.01
    assert _z(means, 20.0) < 4.5


def test_ssa_schlogl_bistable_mean_and_well_mass():
    """Schloegl (Table I form) at V = 10: time average of x and the mass of
    {x <= 10} against the exact birth-death law."""
    net = K.schlogl_paper(V=10, hist_max=200, split=11)
    pi = E.schlogl_stationary(net["c"], net["s"], 200)
    x = np.arange(201)
    means, lows = [], []
    for seed in range(16):
        h, ev, _ = O.ssa_run(net, 1, [2], 5000.0, 77 + seed)
        means.append((h * x).sum() / h.sum())
        lows.append(h[:11].sum() / h.sum())
    assert _z(means, (pi * x).sum()) < 4.5
    assert _z(lows, pi[:11].sum()) < 4.5


def test_ssa_toggle_against_cme():
    """Toggle switch with alpha = 10, n = 1 (fast mixing): 2-D time-weighted
    histogram against the truncated CME."""
    net = K.toggle(alpha=10.0, n=1.0, delta=1.0, hist_max=(40, 40))
    pi = E.toggle_stationary(net["c"], 40, 40).ravel()
    tot = np.zeros(41 * 41)
    mU, mV = [], []
    for seed in range(16):
        h, ev, _ = O.ssa_run(net, 1, [5, 5], 10000.0, 5 + seed)
        tot += h
        h = h.reshape(41, 41) / h.sum()
        mU.append((h.sum(1) * np.arange(41)).sum())
        mV.append((h.sum(0) * np.arange(41)).sum())
    p = tot / tot.sum()
    assert 0.5 * np.abs(p - pi).sum() < 0.03
    pi2 = pi.reshape(41, 41)
    assert _z(mU, (pi2.sum(1) * np.arange(41)).sum()) < 4.5
    assert _z(mV, (pi2.sum(0) * np.arange(41)).sum()) < 4.5


def test_ssa_trace_matches_run():
    """The trace and the run draw from the same counters."""
    net = K.schlogl_classic()
    J, xs, tau = O.ssa_trace(net, [85], 9, 0, 500)
    assert set(np.unique(J)) <= {0, 1, 2, 3}
    steps = np.array([1, -1, 1, -1])[J]
    assert np.all(xs[:, 0] == 85 + np.cumsum(steps))
    assert np.all(tau > 0)


# ---------------------------------------------------------------------------
# the parallel step: first-escape lemma (Sec. III.A, results 1 and 2)
# ---------------------------------------------------------------------------
def _tiny_chain():
    net = K.immigration_death(1.0, 1.0, hist_max=40, split=3)  # W = {0, 1, 2}
    x = np.arange(41)
    lam = E.schlogl_props(net["c"], net["s"], x)
    b, d = lam[0] + lam[2], lam[1] + lam[3]
    PW, _ = E.bd_jump_matrix(b[:3], d[:3])
    # the last column of the restricted matrix would leave W; keep the 3x3 block
    nu, lmb = E.qsd_dtmc(PW)
    return net, nu, lmb, b + d


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("R", [1, 7, 32])
def test_first_escape_lemma_tiny_chain(R, precision):
    """With R iid replicas started from the jump-chain QSD, R(N*-1)+K (K
    1-based) is geometric with parameter 1 - lambda, whatever R; the summed
    holding time of the contributions has mean E_nu[1/a0] / (1 - lambda).
    In binary32 one Philox call serves two lockstep steps of a replica: a
    layout that reused a word for both steps would correlate them and bend
    the geometric law of M."""
    net, nu, lmb, a0 = _tiny_chain()
    rng = np.random.default_rng(R)
    M, T = [], []
    trials = 6000
    for t in range(trials):
        st = rng.choice(3, size=R, p=nu)
        states = np.stack([st, np.zeros(R, dtype=int)], axis=1)
        rc, nstar, k, xe, ts = O.parallel_from(net, states, 0, t, 1234 + R, precision=precision)
        assert rc == 0 and xe[0] == 3
        M.append(R * (nstar - 1) + k + 1)
        T.append(ts)
    M = np.array(M)
    mean_geo = 1.0 / (1.0 - lmb)
    assert _z(M, mean_geo) < 4.5
    # distribution: P(M > m) = lambda^m
    for m in [1, 2, 4, 8]:
        p = (M > m).mean()
        se = np.sqrt(lmb**m * (1 - lmb**m) / trials)
        assert abs(p - lmb**m) < 4.5 * se + 1e-12, (m, p, lmb**m)
    et = float(np.sum(nu / a0[:3])) / (1.0 - lmb)
    assert _z(T, et) < 4.5


# ---------------------------------------------------------------------------
# dephasing: Fleming-Viot samples the jump-chain QSD
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("G", [32, 4096])
@pytest.mark.parametrize("n_p", [200, 201])
def test_dephasing_samples_jump_chain_qsd(G, n_p, precision):
    """Fleming-Viot dephasing (Algorithm 1) samples the QSD of the jump chain.
    A birth-death jump chain moves by +-1, so it is bipartite: after n_p
    lockstep jumps from X~ every replica has the parity of X~ + n_p, and the
    two-step chain's QSD on that parity class is the QSD nu restricted to it
    (nu P^2 = lambda^2 nu and P^2 keeps the parity).  In binary32 one Philox
    call serves four dephasing jumps (word i mod 4): reusing a word would
    correlate the jumps and move the sampled law off nu."""
    net = K.immigration_death(5.0, 1.0, hist_max=60, split=8)  # W = {0..7}
    x = np.arange(61)
    lam = E.schlogl_props(net["c"], net["s"], x)
    PW, _ = E.bd_jump_matrix((lam[0] + lam[2])[:8], (lam[1] + lam[3])[:8])
    nu, _ = E.qsd_dtmc(PW)
    target = np.where(np.arange(8) % 2 == n_p % 2, nu, 0.0)
    target /= target.sum()
    cnt = np.zeros(8)
    for cyc in range(4):
        xs, steps, ev = O.dephase(net, 4096, [0], 0, cyc, n_p, 99, thresh="steps", fv_group=G, precision=precision)
        assert steps == n_p and ev == n_p * 4096
        assert xs[:, 0].max() < 8
        cnt += np.bincount(xs[:, 0], minlength=8)[:8]
    p = cnt / cnt.sum()
    assert 0.5 * np.abs(p - target).sum() < 0.03


def test_dephase_steps_time_mode():
    net = K.schlogl_classic()
    a0 = E.schlogl_props(net["c"], net["s"], np.array([85.0])).sum()
    assert O.dephase_steps(net, [85], 1.0) == int(np.ceil(a0))
    assert O.dephase_steps(net, [85], 7.0, thresh="steps") == 7


# ---------------------------------------------------------------------------
# full ParRep (Algorithm 1)
# ---------------------------------------------------------------------------
def test_parrep_clock_and_burn_in_split_are_exact():
    """T_s ends at T_end; the histograms before and after T_burn sum to T_burn
    and T_end - T_burn; the constant channel gives I_33 (T_end - T_burn) s3/c3
    (the I_33 = 200 fact of Table II), and its RER is E[lambda_3] times
    (eps - log(1 + eps)) per unit time."""
    net = K.schlogl_paper(V=10, hist_max=200, split=11)
    eps = 0.1
    cp = np.array([net["c"]] * 2, dtype=float)
    cp[0, 2] *= 1 + eps
    cp[1, 0] *= 1 + eps
    r = O.parrep_run(net, 16, 300, 300, 2000.0, 5, [2], thresh="steps", T_burn=700.0, rer_cprime=cp)
    assert r["status"] == 0
    assert r["T_s"] == 2000.0
    assert abs(r["hist_pre"].sum() - 700.0) < 1e-9
    assert abs(r["hist_post"].sum() - 1300.0) < 1e-9
    F = r["fim"]
    assert abs(F[2, 2] - 1300.0 * net["s"][2] / net["c"][2]) < 1e-8
    assert np.allclose(F - np.diag(np.diag(F)), 0.0)
    A3 = net["c"][2] * net["s"][2]
    assert abs(r["rer"][0] - 1300.0 * A3 * (eps - np.log1p(eps))) < 1e-8
    # channel 1: E[lambda_1] integrated = F_11 c1^2
    assert abs(r["rer"][1] - F[0, 0] * net["c"][0] ** 2 * (eps - np.log1p(eps))) < 1e-6 * abs(r["rer"][1])


@pytest.mark.parametrize("which", ["schlogl", "toggle"])
def test_parrep_fim_rer_are_histogram_contractions(which):
    """The per-jump sums of the RER and FIM integrands (Appendix A) equal the
    post-burn occupation times contracted with
    the closed-form per-state rates (sum_j lambda_j grad log lambda_j^2, and
    sum_j lambda_j log(lambda_j / lambda'_j) - lambda_j + lambda'_j)."""
    if which == "schlogl":
        net = K.schlogl_paper(V=10, hist_max=200, split=11)
        xs = np.arange(201)
        lam = E.schlogl_props(net["c"], net["s"], xs)
        grad = E.schlogl_grad_log(net["c"], xs)
        props = lambda c: E.schlogl_props(c, net["s"], xs)
        run = dict(t_corr=300, t_phase=300, T_end=800.0, x0=[2], thresh="steps")
    else:
        net = K.toggle(alpha=20, n=2.5, hist_max=(63, 63))
        U, V = np.meshgrid(np.arange(64.0), np.arange(64.0), indexing="ij")
        U, V = U.ravel(), V.ravel()
        lam = E.toggle_props(net["c"], U, V)
        grad = E.toggle_grad_log(net["c"], U, V)
        props = lambda c: E.toggle_props(c, U, V)
        run = dict(t_corr=1.0, t_phase=1.0, T_end=60.0, x0=[15, 2], thresh="time")
    cp = np.array([net["c"]] * 2, dtype=float)
    cp[0, 0] *= 1.2
    cp[1, 2] *= 0.7
    r = O.parrep_run(net, 16, run["t_corr"], run["t_phase"], run["T_end"], 9, run["x0"], thresh=run["thresh"],
                     T_burn=20.0, rer_cprime=cp)
    assert r["status"] == 0
    w = r["hist_post"]
    F = E.fim_exact(lam, grad, w)
    assert np.allclose(r["fim"], F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
    for k in range(2):
        Rk = E.rer_exact(lam, props(cp[k]), w)
        assert abs(r["rer"][k] - Rk) <= 1e-12 * abs(Rk)


def test_parrep_without_escapes_is_stationary_poisson():
    """A single region: after decorrelation and dephasing the parallel step
    runs R replicas to T_end; the pooled histogram is Poisson and the FIM of
    the death channel is E[lambda_4]/c4^2 = k_in/k_out^2 (Appendix A)."""
    from scipy.stats import poisson

    net = K.immigration_death(20.0, 2.0, hist_max=80)
    p_tot = np.zeros(81)
    f44 = []
    for seed in range(8):
        r = O.parrep_run(net, 8, 50, 50, 3000.0, 40 + seed, [10], thresh="steps", T_burn=100.0)
        assert r["status"] == 0 and r["escapes"] == 0
        p_tot += r["hist_pre"] + r["hist_post"]
        f44.append(r["fim"][3, 3] / 2900.0)
    p = p_tot / p_tot.sum()
    assert 0.5 * np.abs(p - poisson.pmf(np.arange(81), 10.0)).sum() < 0.01
    assert _z(f44, 20.0 / 4.0) < 4.5


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("thresh,tc", [("steps", 3000), ("time", 4.0)])
def test_parrep_bistable_schlogl_matches_exact(thresh, tc, precision):
    """ParRep on the Schloegl network (Table I form, V = 10) with long
    decorrelation/dephasing: the ergodic mean of x and the mass of the lower
    well against the exact birth-death law (cf. the Sec. V.A comparison with
    the CME), in both precision forms."""
    net = K.schlogl_paper(V=10, hist_max=200, split=11)
    pi = E.schlogl_stationary(net["c"], net["s"], 200)
    x = np.arange(201)
    means, lows, esc = [], [], 0
    for seed in range(12):
        r = O.parrep_run(net, 16, tc, tc, 8000.0, 300 + seed, [2], thresh=thresh, fv_group=16,
                         precision=precision)
        assert r["status"] == 0
        h = r["hist_pre"] + r["hist_post"]
        means.append((h * x).sum() / h.sum())
        lows.append(h[:11].sum() / h.sum())
        esc += r["escapes"]
    assert esc > 100
    assert _z(means, (pi * x).sum()) < 4.5
    assert _z(lows, pi[:11].sum()) < 4.5


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_decorrelation_alone_is_the_exact_chain(precision):
    """With t_corr beyond T_end the run never leaves the decorrelation step
    (Algorithm 1), which simulates X~ with the exact SSA under its own counter
    layout (binary32: one Philox call per two jumps).  Immigration-death then
    has the Poisson(k_in/k_out) law, and every jump's time enters T_s."""
    from scipy.stats import poisson

    net = K.immigration_death(20.0, 2.0, hist_max=80, split=9)
    p_tot = np.zeros(81)
    for seed in range(8):
        r = O.parrep_run(net, 8, 1e6, 5.0, 4000.0, 70 + seed, [10], thresh="time", precision=precision)
        assert r["status"] == 0 and r["n_cycles"] == 1 and r["escapes"] == 0
        assert r["events_parallel_useful"] == 0 and r["events_decorr"] > 0
        p_tot += r["hist_pre"] + r["hist_post"]
    p = p_tot / p_tot.sum()
    assert 0.5 * np.abs(p - poisson.pmf(np.arange(81), 10.0)).sum() < 0.01


def _decorrelated_sojourns(xs, tau, x0, split, t_corr):
    """Brute-force count on an exact SSA trace (pre-jump states, holding times):
    sojourns between two region changes whose time up to their last in-region
    jump (the sojourn minus the exit's holding time) is >= t_corr, i.e. those
    in which a TIME-mode decorrelation would have completed; and the time
    between the first and the last region change."""
    pre = np.concatenate([[x0], xs[:-1, 0]])
    t = np.cumsum(tau)
    ex = np.nonzero((pre >= split) != (xs[:, 0] >= split))[0]
    L = t[ex[1:]] - t[ex[:-1]]
    return int(np.sum(L - tau[ex[1:]] >= t_corr)), t[ex[-1]] - t[ex[0]]


def _schlogl_v10_rates():
    net = K.schlogl_paper(V=10, hist_max=200, split=11)
    lam = E.schlogl_props(net["c"], net["s"], np.arange(201))
    return net, lam[0] + lam[2], lam[1] + lam[3]


@pytest.mark.parametrize("t_corr", [0.1, 1.0])
def test_decorrelated_exit_rate_against_exact_chain_trace(t_corr):
    """bd_decorrelated_exit_rate (the escapes per unit time an exact ParRep
    run has in TIME mode) against the same event counted on exact SSA traces
    of the V = 10 Schloegl chain; at t_corr = 0.1 the exit-on-the-next-jump
    correction is 6% and the pin resolves it."""
    net, b, d = _schlogl_v10_rates()
    exact = E.bd_decorrelated_exit_rate(b, d, 11, t_corr)
    rates = []
    for tr in range(32):
        J, xs, tau = O.ssa_trace(net, [2], 5, tr, 400000)
        c, T = _decorrelated_sojourns(xs, tau, 2, 11, t_corr)
        rates.append(c / T)
    assert _z(rates, exact) < 4.5


def test_decorrelated_exit_rate_limits():
    """t_corr = 0: every sojourn whose first jump stays in its region counts,
    J (2 - p(split-1 -> split) - p(split -> split-1)) with J the stationary
    flux; the rate falls as t_corr grows (fewer sojourns last long enough)."""
    net, b, d = _schlogl_v10_rates()
    pi = E.bd_stationary(b, d)
    J = pi[10] * b[10]
    r0 = J * (2.0 - b[10] / (b[10] + d[10]) - d[11] / (b[11] + d[11]))
    assert abs(E.bd_decorrelated_exit_rate(b, d, 11, 0.0) - r0) < 1e-12 * r0
    rates = [E.bd_decorrelated_exit_rate(b, d, 11, t) for t in (0.5, 1.0, 2.0, 4.0)]
    assert all(a > c for a, c in zip(rates, rates[1:]))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_parrep_escape_rate_is_exact_only_for_long_thresholds(precision):
    """Sec. III.B: ParRep is exact as the decorrelation and dephasing grow.
    With t_corr = t_phase = 4 (TIME mode, R = 16) the parallel-step escapes of
    the V = 10 Schloegl chain come at the exact decorrelated-exit rate; with
    0.25 / 0.25 the dephased replicas are not yet quasi-stationary, the first
    of the R replicas escapes early, and the rate is far too high."""
    net, b, d = _schlogl_v10_rates()
    for tc, ok in ((4.0, True), (0.25, False)):
        exact = E.bd_decorrelated_exit_rate(b, d, 11, tc)
        rates = []
        for seed in range(12):
            r = O.parrep_run(net, 16, tc, tc, 8000.0, 300 + seed, [2], thresh="time", fv_group=16,
                             precision=precision)
            assert r["status"] == 0
            rates.append(r["escapes"] / 8000.0)
        if ok:
            assert _z(rates, exact) < 4.5
        else:
            assert np.mean(rates) > 1.2 * exact and _z(rates, exact) > 6


def test_parrep_cycle_log_is_consistent():
    net = K.schlogl_paper(V=10, hist_max=200, split=11)
    r = O.parrep_run(net, 16, 400, 400, 3000.0, 11, [2], thresh="steps")
    cyc = r["cycles"]
    assert len(cyc) == r["n_cycles"] and cyc[-1]["ended"] == 1
    for a in cyc[:-1]:
        assert a["k"] >= 0 and a["n_star"] >= 1 and a["dephase_steps"] == 400
        # X~ after the cycle is outside the region the cycle ran in
        assert (a["x_tilde"][0] < 11) != (a["W"] == 0)
    ts = [a["T_s"] for a in cyc]
    assert all(b >= a for a, b in zip(ts, ts[1:]))
    assert ts[-1] == 3000.0


def test_parrep_x0_draw_is_uniform():
    net = K.schlogl_classic()
    xs = [O.initial_state(net, s, [0], 1000)[0] for s in range(4000)]
    assert min(xs) >= 0 and max(xs) <= 1000
    assert _z(xs, 500.0) < 4.5


def test_parrep_rejects_bad_input():
    net = K.schlogl_classic()
    assert O.parrep_run(net, 0, 1, 1, 10.0, 0, [85])["status"] == O.OR_EINVAL
    assert O.parrep_run(net, 4, 1, 1, 10.0, 0, [5000])["status"] == O.OR_EINVAL
    small = dict(net, hist_max=120)
    assert O.parrep_run(small, 4, 1, 1, 100.0, 0, [85])["status"] == O.OR_ERANGE


# ---------------------------------------------------------------------------
# stationary sensitivity, IAF and information bounds (Sec. IV.B, Sec. V.A)
# ---------------------------------------------------------------------------
def test_iaf_exact_closed_form_immigration_death():
    """M/M/inf (immigration k_in, death k_out x): Cov(X_0, X_s) =
    (k_in/k_out) exp(-k_out |s|), so tau(x) = 2 k_in / k_out^2."""
    for k_in, k_out in [(5.0, 1.3), (20.0, 2.0)]:
        n = 120
        x = np.arange(n, dtype=float)
        Q = E.generator(np.full(n, k_in), k_out * x)
        pi = E.stationary_dense(Q)
        assert abs(E.iaf_exact(Q, pi, x) / (2.0 * k_in / k_out**2) - 1.0) < 1e-10


def test_iaf_exact_is_the_autocovariance_integral():
    """A random 5-state generator: tau(f) against direct quadrature of
    2 * int_0^inf sum_x pi(x) fbar(x) (exp(sQ) fbar)(x) ds."""
    from scipy.integrate import quad
    from scipy.linalg import expm

    rng = np.random.default_rng(3)
    Q = rng.uniform(0.2, 2.0, size=(5, 5))
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(1))
    pi = E.stationary_dense(Q)
    f = rng.normal(size=5)
    fbar = f - pi @ f
    cov = lambda s: float(pi @ (fbar * (expm(s * Q) @ fbar)))
    ref = 2.0 * quad(cov, 0.0, np.inf, limit=200)[0]
    assert abs(E.iaf_exact(Q, pi, f) / ref - 1.0) < 1e-7


def test_stationary_sensitivity_matches_product_formula_difference():
    """d pi(x)/d c_k from the generator solve against central differences of
    the detailed-balance product formula (V = 25, truncation 255)."""
    net = K.schlogl_paper(V=25, hist_max=255)
    x = np.arange(256.0)
    pi = E.schlogl_stationary(net["c"], net["s"], 255)
    Q, dQ = E.schlogl_generators(net["c"], net["s"], 255)
    S = E.stationary_sensitivity(Q, dQ, pi, x)
    for k in range(4):
        h = 1e-5 * net["c"][k]
        cp, cm = np.array(net["c"]), np.array(net["c"])
        cp[k] += h
        cm[k] -= h
        fd = (E.schlogl_stationary(cp, net["s"], 255) @ x - E.schlogl_stationary(cm, net["s"], 255) @ x) / (2 * h)
        assert abs(S[k] / fd - 1.0) < 1e-6, (k, S[k], fd)


def _half_unit(v, digits=3):
    """Half a unit in the last of the printed significant digits."""
    return 0.5 * 10.0 ** (np.floor(np.log10(abs(v))) - (digits - 1))


def test_exact_sensitivities_and_iaf_against_paper():
    """Table III's CME approximation (truncation [0, 149]) for c1, c3, c4 to
    the printed three digits; the printed c2 entry (+9.10E+02) is garbled,
    the exact value is about -998.  The printed IAF 5.87e5 is a 100-sample
    estimate whose relative standard deviation is sqrt(2/99) = 0.142; the
    exact value lies within it."""
    g = _golden_paper()
    net = K.schlogl_paper(V=25, hist_max=149)
    x = np.arange(150.0)
    pi = E.schlogl_stationary(net["c"], net["s"], 149)
    Q, dQ = E.schlogl_generators(net["c"], net["s"], 149)
    S = E.stationary_sensitivity(Q, dQ, pi, x)
    for k, key in [(0, "cme_sens_c1"), (2, "cme_sens_c3"), (3, "cme_sens_c4")]:
        assert abs(S[k] - g[key][0]) <= _half_unit(g[key][0]), (key, S[k])
    assert -1005.0 < S[1] < -990.0
    tau = E.iaf_exact(Q, pi, x)
    assert abs(tau / g["iaf_x"][0] - 1.0) < np.sqrt(2.0 / 99.0)
    assert 5.62e5 < tau < 5.635e5


def test_bounds_reproduce_table_iii_and_dominate_the_sensitivities():
    """sqrt(tau) sqrt(I_kk) with the printed IAF 5.87e5 and the exact FIM
    diagonal gives Table III's bounds to the printed three digits; with the
    exact tau and FIM the bound dominates |v . grad pi(x)| for every
    direction (Cauchy-Schwarz, the content of the bound)."""
    from oracle import uq as U

    g = _golden_paper()
    net = K.schlogl_paper(V=25, hist_max=255)
    x = np.arange(256.0)
    pi = E.schlogl_stationary(net["c"], net["s"], 255)
    lam = E.schlogl_props(net["c"], net["s"], x)
    F = E.fim_exact(lam, E.schlogl_grad_log(net["c"], x), pi)
    b = U.bounds(g["iaf_x"][0], F)
    for k in range(4):
        v = g["bound_c%d" % (k + 1)][0]
        assert abs(b[k] - v) <= _half_unit(v), (k, b[k])
    Q, dQ = E.schlogl_generators(net["c"], net["s"], 255)
    S = E.stationary_sensitivity(Q, dQ, pi, x)
    tau = E.iaf_exact(Q, pi, x)
    rng = np.random.default_rng(5)
    V = np.vstack([np.eye(4), rng.normal(size=(64, 4))])
    assert np.all(np.abs(V @ S) <= U.bounds(tau, F, V))


def test_uq_estimators_on_oracle_runs_of_immigration_death():
    """The Sec. IV.B estimators over independent oracle runs (one replica, a
    single region, so each run is one SSA path after its start) of
    immigration-death: IAF 2 k_in / k_out^2, mean k_in / k_out and the death
    channel's FIM entry k_in / k_out^2 within their sampling errors."""
    from oracle import uq as U

    k_in, k_out, T_b, T = 5.0, 1.0, 200.0, 420.0
    net = K.immigration_death(k_in, k_out, hist_max=60)
    hs, Z = [], []
    for seed in range(240):
        r = O.parrep_run(net, 1, 10, 10, T, 700 + seed, [5], thresh="steps", T_burn=T_b)
        assert r["status"] == 0
        hs.append(r["hist_post"])
        Z.append(r["fim"] / (T - T_b))
    f = np.arange(61.0)
    out = U.uq(f, hs, Z, T - T_b)
    tau = 2.0 * k_in / k_out**2
    # a sample variance of 240 near-normal values: relative sd sqrt(2/239) = 0.091;
    # the finite window shrinks the mean by 1/(k_out (T - T_b)) = 0.45%
    assert abs(out["iaf"] / tau - 1.0) < 4 * 0.091
    assert abs(out["mean_f"] - k_in / k_out) < 4 * np.sqrt(tau / (T - T_b) / 240)
    assert abs(out["fim"][3, 3] - k_in / k_out**2) < 4 * out["fim_half_width"][3, 3] / 1.96
    assert np.allclose(out["Y"], [h @ f for h in hs])


def test_iaf_exact_on_the_toggle_generator_at_hill_exponent_zero():
    """With Hill exponent 0 the toggle's production rates are the constant
    alpha/2, so U and V are independent M/M/inf chains (production alpha/2,
    degradation delta): tau(U) = alpha/delta^2 and, by independence,
    tau(U - V) = 2 alpha / delta^2 on the two-dimensional generator."""
    alpha, delta, m = 6.0, 1.5, 30
    c = [alpha, 0.0, delta, alpha, 0.0, delta]
    Q = E.toggle_generator(c, m, m).toarray()
    pi = E.toggle_stationary(c, m, m).ravel()
    U, V = np.meshgrid(np.arange(m + 1.0), np.arange(m + 1.0), indexing="ij")
    assert abs(E.iaf_exact(Q, pi, U.ravel()) / (alpha / delta**2) - 1.0) < 1e-9
    assert abs(E.iaf_exact(Q, pi, (U - V).ravel()) / (2.0 * alpha / delta**2) - 1.0) < 1e-9


# ---------------------------------------------------------------------------
# genetic switch of Sec. V.B: exact references pinned to the paper
# ---------------------------------------------------------------------------
def _golden_genetic():
    d = {}
    with open(os.path.join(GOLDEN, "paper_genetic_switch.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v, hw = line.split()[:3]
            d[k] = (float(v), float(hw))
    return d


@pytest.fixture(scope="module")
def genetic_chain():
    c = E.genetic_paper_params()
    Q, pi = E.genetic_stationary(c, 15, 3500)
    return c, Q, pi, E.genetic_states(15, 3500)


def test_genetic_rate_equation_fixed_points_match_paper():
    """The two stable points and the saddle of the rate equations, to the
    four printed decimals (half a unit in the last: 5e-5)."""
    g = _golden_genetic()
    fps = E.genetic_rre_fixed_points(E.genetic_paper_params())
    assert len(fps) == 3
    for (x1, x2), key in zip(fps, ["plus", "saddle", "minus"]):
        for v, k in [(x1, "fp_%s_x1" % key), (x2, "fp_%s_x2" % key)]:
            assert abs(v - g[k][0]) <= 5e-5, (k, v)


def test_genetic_gradients_match_finite_differences():
    c = E.genetic_paper_params()
    rng = np.random.default_rng(2)
    xi = rng.integers(0, 2, 50).astype(float)
    m = rng.integers(0, 10, 50).astype(float)
    p = rng.integers(0, 3000, 50).astype(float)
    G = E.genetic_grad_props(c, xi, m, p)
    for k in range(8):
        h = 1e-6 * c[k]
        cp, cm = c.copy(), c.copy()
        cp[k] += h
        cm[k] -= h
        fd = (E.genetic_props(cp, xi, m, p) - E.genetic_props(cm, xi, m, p)) / (2 * h)
        assert np.allclose(G[:, k], fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max() + 1e-15), k


def test_genetic_generator_without_feedback_is_a_two_state_switch():
    """k0min = k0max = k_on, k1min = k1max = k_off: xi is a two-state chain
    independent of m and p, so P(xi = 1) = k_on/(k_on + k_off), E[m] = a P(xi=1)/gamma,
    E[p] = b E[m] gamma, and tau(xi) = 2 pi_0 pi_1 / (k_on + k_off)."""
    kon, koff = 0.7, 1.9
    c = np.array([6.0, 3.0, 2.0, kon, kon, koff, koff, 100.0])
    Q, pi = E.genetic_stationary(c, 30, 160, pin=0)
    xi, m, p = E.genetic_states(30, 160)
    p1 = kon / (kon + koff)
    assert abs(pi @ xi - p1) < 1e-10
    assert abs(pi @ m - c[0] * p1 / c[2]) < 1e-8
    assert abs(pi @ p - c[1] * c[2] * (pi @ m)) < 1e-6
    assert abs(E.iaf_exact_sparse(Q, pi, xi, pin=0) / (2 * p1 * (1 - p1) / (kon + koff)) - 1.0) < 1e-9


def test_genetic_fim_matches_table_v(genetic_chain):
    """The path-space FIM diagonal E_pi[sum_j (d lambda_j/d c_k)^2 / lambda_j]
    of the exact chain lies within Table V's half widths for all eight
    parameters; entry (1,1) is E[xi]/a in closed form."""
    g = _golden_genetic()
    c, Q, pi, (xi, m, p) = genetic_chain
    assert np.abs(pi @ Q).max() < 1e-12
    lam = E.genetic_props(c, xi, m, p)
    dl = E.genetic_grad_props(c, xi, m, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(lam[:, None, :] > 0, dl**2 / lam[:, None, :], 0.0)
    F = (terms * pi).sum(axis=(0, 2))
    assert abs(F[0] - (pi @ xi) / c[0]) < 1e-15
    for k in range(8):
        v, hw = g["fim_%d%d" % (k + 1, k + 1)]
        assert abs(F[k] - v) <= hw, (k, F[k], v, hw)


def test_genetic_iafs_against_table_vi(genetic_chain):
    """Table VI's IAFs are 100-sample estimates (relative standard deviation
    sqrt(2/99) = 0.142); the exact values lie within one of it, and the IAFs
    of xi and 1 - xi are equal."""
    g = _golden_genetic()
    c, Q, pi, (xi, m, p) = genetic_chain
    t_on = E.iaf_exact_sparse(Q, pi, xi)
    assert abs(E.iaf_exact_sparse(Q, pi, 1.0 - xi) / t_on - 1.0) < 1e-9
    for key, f in [("iaf_active", xi), ("iaf_mrna", m), ("iaf_protein", p)]:
        t = E.iaf_exact_sparse(Q, pi, f)
        assert abs(t / g[key][0] - 1.0) < np.sqrt(2.0 / 99.0), (key, t)


# the genetic switch in the Algorithm 1 oracle (state x[0] = 2 m + xi, x[1] = p)
GEN_SMALL = np.array([12.0, 5.0, 10.0, 0.2, 20.0, 0.2, 20.0, 25.0])  # bistable: p ~ 0.6 / 46, saddle 12.8


def _genetic_spec(c, m_max, p_max, split):
    return dict(kind="genetic", c=list(c), s=[1.0, 1.0, 1.0, 1.0], hist_max=[2 * m_max + 1, p_max],
                regions=[([0, 1], split)])


def _genetic_exact_bins(c, m_max, p_max):
    """Exact law laid out like the oracle's histogram: bin (2 m + xi) * (p_max + 1) + p."""
    Q, pi = E.genetic_stationary(c, m_max, p_max, pin=((min(40, p_max) * (m_max + 1)) + 1) * 2 + 1)
    xi, m, p = E.genetic_states(m_max, p_max)
    out = np.zeros((2 * m_max + 2) * (p_max + 1))
    out[(2 * m + xi) * (p_max + 1) + p] = pi
    return out


def _marginals(h, m_max, p_max):
    h = h.reshape(2 * m_max + 2, p_max + 1)
    return h.sum(0), h[1::2].sum()  # protein marginal, P(xi = 1)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_genetic_ssa_matches_exact_law(precision):
    """The oracle's SSA on a small bistable switch (wells at p ~ 0.6 and 46,
    saddle 12.8): the protein marginal within TV 0.03 of the exact law and
    P(xi = 1) within 4.5 standard errors."""
    mm, pm = 16, 250
    spec = _genetic_spec(GEN_SMALL, mm, pm, 13)
    ex = _genetic_exact_bins(GEN_SMALL, mm, pm)
    tot, on = np.zeros(len(ex)), []
    for seed in range(8):
        h, ev, _ = O.ssa_run(spec, 1, [0, 0], 5000.0, 300 + seed, precision=precision)
        tot += h
        on.append(_marginals(h / h.sum(), mm, pm)[1])
    pm_hat, _ = _marginals(tot / tot.sum(), mm, pm)
    pm_ex, on_ex = _marginals(ex, mm, pm)
    assert 0.5 * np.abs(pm_hat - pm_ex).sum() < 0.03
    assert _z(on, on_ex) < 4.5


def test_genetic_parrep_matches_exact_law():
    """Algorithm 1 on the small switch (R = 16, n_c = n_p = 1000 jumps, regions
    p <= 12 | p >= 13): the pooled protein marginal within TV 0.02 of the
    exact law over about a hundred escapes (with 200-jump thresholds the
    well mass is 1.6% off: ParRep converges as n_c, n_p grow, Sec. III.B)."""
    mm, pm = 16, 250
    spec = _genetic_spec(GEN_SMALL, mm, pm, 13)
    ex = _genetic_exact_bins(GEN_SMALL, mm, pm)
    tot, esc = np.zeros(len(ex)), 0
    for seed in range(6):
        r = O.parrep_run(spec, 16, 1000, 1000, 5000.0, 40 + seed, [0, 0], thresh="steps")
        assert r["status"] == 0
        tot += r["hist_pre"] + r["hist_post"]
        esc += r["escapes"]
    assert esc > 50
    pm_hat, _ = _marginals(tot / tot.sum(), mm, pm)
    pm_ex, _ = _marginals(ex, mm, pm)
    assert 0.5 * np.abs(pm_hat - pm_ex).sum() < 0.02


def test_genetic_parrep_fim_rer_are_histogram_contractions():
    """The per-jump FIM and RER sums of the six-channel network equal the
    post-burn occupation times contracted with the closed-form per-state
    rates sum_j (d lambda_j / d c)^2 / lambda_j and the RER integrand."""
    mm, pm = 16, 250
    spec = _genetic_spec(GEN_SMALL, mm, pm, 13)
    cp = np.array([GEN_SMALL, GEN_SMALL])
    cp[0, 4] *= 1.3
    cp[1, 7] *= 0.8
    r = O.parrep_run(spec, 8, 100, 100, 400.0, 5, [0, 0], thresh="steps", T_burn=50.0, rer_cprime=cp)
    assert r["status"] == 0
    b = np.arange((2 * mm + 2) * (pm + 1))
    x0, p = b // (pm + 1), b % (pm + 1)
    xi, m = x0 & 1, x0 >> 1
    lam = E.genetic_props(GEN_SMALL, xi, m, p)
    dl = E.genetic_grad_props(GEN_SMALL, xi, m, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        rate = np.where(lam[:, None, None, :] > 0, dl[:, :, None, :] * dl[:, None, :, :] / lam[:, None, None, :], 0.0)
    w = r["hist_post"]
    F = np.einsum("jabn,n->ab", rate, w)
    assert np.allclose(r["fim"], F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
    for k in range(2):
        Rk = E.rer_exact(lam, E.genetic_props(cp[k], xi, m, p), w)
        assert abs(r["rer"][k] - Rk) <= 1e-11 * abs(Rk)


def test_stored_exact_references_come_from_the_oracle():
    """tests/golden/exact_references.json (read by bench.py and the GPU
    accuracy tests) is what make_exact_references.py computes from the
    oracle's exact references today."""
    import importlib.util
    import json

    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLDEN, "make_exact_references.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    fresh = mk.compute()
    with open(os.path.join(GOLDEN, "exact_references.json")) as f:
        stored = json.load(f)

    def same(a, b, path):
        if isinstance(a, dict):
            assert set(a) == set(b), path
            for k in a:
                same(a[k], b[k], path + "/" + k)
        elif isinstance(a, list):
            assert np.allclose(a, b, rtol=1e-10, atol=0.0), path
        else:
            assert a == pytest.approx(b, rel=1e-10), path

    same(fresh, stored, "")
    # spot facts: the classic Schloegl lower-well mass and the Table II I_33
    assert stored["schlogl_classic"]["mass_lower"] == pytest.approx(0.22026, abs=1e-5)
    assert stored["schlogl_v25"]["fim_diag"][2] == pytest.approx(200.0, rel=1e-12)
