"""Stationary uncertainty quantification from independent ParRep runs --
TEST INFRASTRUCTURE ONLY (imported by tests/ alone).

Sec. IV.B estimates the two factors of the stationary information bound
S_{f,v} <= sqrt(tau(f)) sqrt(v^T I_H v) from N independent samples that each
ran to T after a burn-in T_b:

* the IAF tau(f): Y_k is the integral of f over [T_b, T] of sample k; the
  estimator is sum_k (Y_k - Ybar)^2 / ((T - T_b) (N - 1));
* the stationary mean pi(f) as the mean of Y_k / (T - T_b);
* the path-space FIM I_H: the mean of the samples' ergodic averages Z_k, with
  a normal 95% half-width 1.96 sd(Z) / sqrt(N) per entry (the half widths of
  Table II);
* the bounds: sqrt(tau) sqrt(v^T I_H v) for each direction v (unit vectors
  give the per-parameter bounds of Table III).

Here a sample's occupation times come from the oracle's post-burn histogram
(time spent in each state during [T_b, T]), so Y_k = sum_x f(x) h_k(x).
"""
from __future__ import annotations

import numpy as np


def integral_of(f, hist_post):
    """Y = integral of f over the post-burn window = sum_x f(x) h(x)."""
    return float(np.sum(np.asarray(f, dtype=np.float64) * np.asarray(hist_post, dtype=np.float64)))


def iaf_estimate(Y, window):
    """Sec. IV.B: sample variance of the window integrals over the window length."""
    Y = np.asarray(Y, dtype=np.float64)
    n = len(Y)
    ybar = Y.sum() / n
    return float(np.sum((Y - ybar) ** 2) / (window * (n - 1)))


def fim_estimate(Z):
    """Mean of the per-sample ergodic FIM averages and the 95% half-widths."""
    Z = np.asarray(Z, dtype=np.float64)
    n = Z.shape[0]
    mean = Z.sum(axis=0) / n
    sd = np.sqrt(np.sum((Z - mean) ** 2, axis=0) / (n - 1))
    return mean, 1.96 * sd / np.sqrt(n)


def bounds(tau, fim, directions=None):
    """sqrt(tau) sqrt(v^T I v) for each row v of directions (default: the
    unit vectors, one bound per parameter)."""
    I = np.asarray(fim, dtype=np.float64)
    V = np.eye(I.shape[0]) if directions is None else np.atleast_2d(np.asarray(directions, dtype=np.float64))
    q = np.einsum("ka,ab,kb->k", V, I, V)
    return np.sqrt(tau) * np.sqrt(np.maximum(q, 0.0))


def uq(f, hist_posts, fims, window, directions=None):
    """All of the above from N samples' post-burn histograms (time units) and
    per-sample FIM ergodic averages."""
    Y = np.array([integral_of(f, h) for h in hist_posts])
    tau = iaf_estimate(Y, window)
    mean = float(Y.sum() / len(Y) / window)
    fim, half = fim_estimate(fims)
    return dict(Y=Y, iaf=tau, mean_f=mean, fim=fim, fim_half_width=half, bounds=bounds(tau, fim, directions))
