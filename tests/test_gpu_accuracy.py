"""Accuracy of the benchmarked Schloegl workload (4096 replicas, x_0 ~
U{0..1000}, TIME thresholds, T_end = 1e6) against the exact chain.

ParRep is exact only as the decorrelation and dephasing grow (Sec. III.B).
The sharpest test is the parallel-step escape rate: an exact ParRep run has
one escape per sojourn in which a decorrelation of length t_corr completes,
so its escapes per unit time must equal the exact rate of those exits
(computed from the birth-death generator and stored by
tests/golden/make_exact_references.py).  Replicas that are not yet
quasi-stationary when the parallel step starts escape early, and with 4096 of
them the first escape comes far too soon: at t_corr = t_phase = 1 the rate is
about seven times too high; at 12 the rates out of both wells are exact
within 1% (pooled over 1024 runs: TV 0.001 from the exact law).  In between,
the replicas dephased from one point for t_phase lack quasi-stationary mass
near the saddle, and the R-fold first escape amplifies that into lower-well
stays that are 9% (t = 6) and 6% (t = 8) too long.
"""
import numpy as np
import pytest

import bench
from paper_1705_06807_gb300 import configs as K

pytestmark = pytest.mark.gpu


def _runs(t, n, seed0):
    c = bench.workload("schlogl_n4096")
    hists, T, esc, fims, useful, dev_s = bench.accuracy_runs(c, t, n, "f32", seed0)
    return bench.accuracy_summary(hists, T, esc, fims, t)


def test_benchmark_thresholds_are_biased():
    """t_corr = t_phase = 1 (the configuration the headline number is quoted
    on): the escape rate is several times the exact one."""
    r = _runs(1.0, 16, 900_000)
    assert r["escape_rate_ratio"] - 3.0 * r["escape_rate_ratio_se"] > 2.0, r


def test_escape_rates_and_well_mass_are_exact_at_t12():
    """t_corr = t_phase = 12: the escape rate out of each well within 3
    standard errors of the exact decorrelated-exit rate, the lower-well mass
    within 3 standard errors of 0.22026 and the FIM diagonal within 3 standard
    errors of the exact one (the constant channel's entry exactly)."""
    c = bench.workload("schlogl_n4096")
    byr = []
    hists, T, esc, fims, useful, dev_s = bench.accuracy_runs(c, 12.0, 64, "f32", 910_000, by_region=byr)
    r = bench.accuracy_summary(hists, T, esc, fims, 12.0, esc_by_region=byr)
    assert abs(r["escape_rate_ratio"] - 1.0) < 3.0 * r["escape_rate_ratio_se"], r
    for w in ("lower", "upper"):
        assert abs(r[f"escape_rate_ratio_{w}"] - 1.0) < 3.0 * r[f"escape_rate_ratio_{w}_se"], r
    assert abs(r["well_mass"] - r["well_mass_exact"]) < 3.0 * r["well_mass_se"], r
    for e, se in zip(r["fim_diag_rel_error"], r["fim_diag_rel_se"]):
        # I_33 = E[lambda_3]/c3^2 is a constant channel: exact in every run
        assert abs(e) < (3.0 * se if se > 1e-12 else 1e-12), r
