"""Statistical accuracy of the CUDA path against the exact stationary law.

ParRep (Algorithm 1) on the Schloegl network of Table I with V = 25, whose
stationary law is the detailed-balance product formula of the birth-death
chain, with the settings of Sec. V.A: R = 100 replicas and jump-count
thresholds n_c = n_p = 5000 (the paper finds smaller thresholds not
accurate; with t_corr = t_phase = 1 time unit the QSD is not reached and
the estimate is biased by about 0.17 in total variation, in both forms).
32 independent seeds run as one batch.

Checks: the pooled time-weighted histogram is within total variation 1e-2
of the exact law; bin by bin (batch means over the seeds) at most three of
the ~150 well-populated bins lie beyond 3 standard errors and none beyond
4.5 -- 3 SE per bin is the criterion, read with its multiplicity: with 150
bins an exact sampler puts 0.4 bins beyond 3 SE on average and exceeds 3 of
them with probability 8e-4, while a maximum of 4.5 SE over 150 bins is
exceeded with probability 1e-3; the FIM of the FP32 form is within 1% of
the FP64 form's (Appendix A) and of the exact chain's, compared well by
well; both are near the exact FIM overall.

Error budget: the slowest mode is the hopping between the wells
(correlation time 101 time units), so the pooled run of T = 4e6 time units
has a well-mass standard error of about 2.9e-3; the FIM moves with that mass
by about 0.4%.  Within a well the histogram's shape, and so the well's FIM
average, is known far better, which isolates the precision of the
propensities and the holding times from the rare-event noise.
"""
import numpy as np
import pytest

from oracle import exact as E
from paper_1705_06807_gb300 import ParRep, ParRepBatch, configs as K

pytestmark = pytest.mark.gpu

NET = K.schlogl_paper(V=25)
SPLIT = NET["regions"][0][1]          # W+ = {x <= 25}, W- = {x >= 26}
N_SEEDS, T_EACH, R, NC = 32, 1.25e5, 100, 5000


def _pooled(precision):
    hs = [ParRep(NET, R, NC, NC, x0=[4], thresh="steps", precision=precision) for _ in range(N_SEEDS)]
    b = ParRepBatch(hs)
    b.run([T_EACH] * N_SEEDS, [9001 + 17 * i for i in range(N_SEEDS)])
    assert b.status() == [0] * N_SEEDS
    per = np.array([h.histogram() for h in hs])  # each normalised by its T_s
    fims = np.array([h.fim() for h in hs])       # each a time average over [0, T_s]
    Ts = np.array([h.stats()["T_s"] for h in hs])
    assert np.allclose(Ts, T_EACH)
    esc = sum(h.stats()["escapes"] for h in hs)
    b.close()
    return per, fims, Ts, esc


def _rates():
    """Exact law and per-state FIM diagonal rates lambda_j / c_j^2."""
    x = np.arange(NET["hist_max"] + 1)
    lam = E.schlogl_props(NET["c"], NET["s"], x)
    pi = E.schlogl_stationary(NET["c"], NET["s"], NET["hist_max"])
    r = lam / np.asarray(NET["c"], dtype=float)[:, None] ** 2
    return pi, r


@pytest.fixture(scope="module")
def runs():
    return {p: _pooled(p) for p in ("f64", "f32")}


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_pooled_histogram_within_tv_of_exact_law(runs, precision):
    per, _, Ts, esc = runs[precision]
    pi, _ = _rates()
    assert esc > 1000  # many transitions between the wells
    pooled = (per * Ts[:, None]).sum(0) / Ts.sum()
    tv = 0.5 * np.abs(pooled - pi).sum()
    assert tv <= 1e-2, tv
    # bin by bin: batch means over the independent seeds
    mean = per.mean(0)
    se = per.std(0, ddof=1) / np.sqrt(N_SEEDS)
    big = pi > 1e-3
    z = np.abs(mean[big] - pi[big]) / np.maximum(se[big], 1e-12)
    assert int((z > 3.0).sum()) <= 3, np.sort(z)[-5:]
    assert z.max() < 4.5, (z.max(), np.argmax(z))


def test_fp32_fim_within_one_percent_of_fp64(runs):
    pi, r = _rates()
    F_exact = (r * pi).sum(1)
    well, F, lib = {}, {}, {}
    for p in ("f64", "f32"):
        per, fims, Ts, _ = runs[p]
        h = (per * Ts[:, None]).sum(0) / Ts.sum()
        lib[p] = np.diag((fims * Ts[:, None, None]).sum(0) / Ts.sum())
        F[p] = (r * h).sum(1)
        # the library's FIM is the contraction of its own histogram
        assert np.allclose(lib[p], F[p], rtol=1e-9)
        well[p] = [(r[:, w] * h[w]).sum(1) / h[w].sum() for w in (slice(0, SPLIT), slice(SPLIT, None))]
    well_exact = [(r[:, w] * pi[w]).sum(1) / pi[w].sum() for w in (slice(0, SPLIT), slice(SPLIT, None))]
    for lo_hi in range(2):
        ratio = well["f32"][lo_hi] / well["f64"][lo_hi]
        assert np.all(np.abs(ratio - 1.0) < 0.01), (lo_hi, ratio)
        for p in ("f64", "f32"):
            ratio = well[p][lo_hi] / well_exact[lo_hi]
            assert np.all(np.abs(ratio - 1.0) < 0.01), (p, lo_hi, ratio)
    for p in ("f64", "f32"):
        assert np.all(np.abs(lib[p] / F_exact - 1.0) < 0.02), (p, lib[p] / F_exact)
    # the constant channel's entry is exact in both forms: I_33 = s3 / c3 = 200 (Table II)
    assert abs(lib["f64"][2] - 200.0) < 1e-9 and abs(lib["f32"][2] - 200.0) < 1e-9
