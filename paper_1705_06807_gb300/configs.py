"""Network specifications and seeded synthetic workloads.

Plain data only: rate constants, region tests, histogram ranges and seeded
draws of instance parameters.  Nothing here computes any part of the method,
so both the CUDA path and the CPU oracle can be fed from it.

A network spec is a dict:
  kind      "schlogl" (1 species, 4 channels), "toggle" (2 species, 4 channels)
            or "genetic" (state x0 = 2m + xi, x1 = p; 6 channels)
  c         rate constants.  Schloegl: (c1, c2, c3, c4) with
            lambda_j = c_j * s_j * h_j(x), h = (x(x-1), x(x-1)(x-2), 1, x).
            Toggle: (aU, nU, dU, aV, nV, dV) with production aU/(1+V^nU) of U,
            aV/(1+U^nV) of V, degradation dU*U and dV*V.
            Genetic switch: (a, b, gamma, k0min, k0max, k1min, k1max, D).
  s         Schloegl fixed factors s_j (combinatorial factors or volume scaling)
  hist_max  largest state kept per species (states must stay in [0, hist_max])
  regions   list of (a, b): region(x) = first i with a . x < b, else len(regions)
"""
from __future__ import annotations

import numpy as np


def schlogl_classic(V: float = 1.0, hist_max: int = 1500, split: int = 250) -> dict:
    """Schloegl network with k = (0.03, 1e-4, 200, 3.5) and combinatorial
    factors: lambda = (k1 x(x-1)/2, k2 x(x-1)(x-2)/6, k3, k4 x).  Wells near
    x = 85 and 565, saddle near 250; regions x < split and x >= split.  V
    rescales the rates as in the volume scaling of Table I (k1/V, k2/V^2,
    k3 V, k4), the region split and the histogram range."""
    return dict(kind="schlogl", c=[0.03, 1e-4, 200.0, 3.5],
                s=[0.5 / V, 1.0 / (6.0 * V * V), V, 1.0],
                hist_max=int(round(hist_max * V)), regions=[([1], int(round(split * V)))])


def schlogl_paper(V: float = 25.0, hist_max: int = 255, split: int = 26) -> dict:
    """Schloegl network of Table I with a = 1, b = 2, c = (3, 0.6, 0.25, 2.95):
    lambda = (c1 a x(x-1)/V, c2 x(x-1)(x-2)/V^2, c3 b V, c4 x).  With V = 25
    the saddle is at 25.9649, so W+ = {x <= 25} and W- = {x >= 26}."""
    a, b = 1.0, 2.0
    return dict(kind="schlogl", c=[3.0, 0.6, 0.25, 2.95], s=[a / V, 1.0 / (V * V), b * V, 1.0],
                hist_max=hist_max, regions=[([1], split)])


def immigration_death(k_in: float, k_out: float, hist_max: int = 200, split: int = 10**9) -> dict:
    """Schloegl form with c1 = c2 = 0: immigration at rate k_in, death k_out x.
    Its stationary law is Poisson(k_in / k_out)."""
    return dict(kind="schlogl", c=[0.0, 0.0, k_in, k_out], s=[1.0, 1.0, 1.0, 1.0],
                hist_max=hist_max, regions=[([1], split)])


def genetic_switch(c=None, m_max: int = 15, p_max: int = 3500, split: int = 512) -> dict:
    """Genetic switch of Sec. V.B (Table IV): DNA state xi, mRNA m, protein
    p, stored as x0 = 2m + xi and x1 = p.  Default constants are the paper's
    (b = 22.5, a = 2400/b, gamma = 50, k0min = k1min = 24/b, k0max = k1max =
    2400/b, D = 1000); regions p < split and p >= split (the paper's line
    through the saddle at p = 511.2865)."""
    if c is None:
        b = 22.5
        c = [2400.0 / b, b, 50.0, 24.0 / b, 2400.0 / b, 24.0 / b, 2400.0 / b, 1000.0]
    return dict(kind="genetic", c=[float(v) for v in c], s=[1.0, 1.0, 1.0, 1.0], hist_max=[2 * m_max + 1, p_max],
                regions=[([0, 1], split)])


def toggle(alpha: float = 50.0, n: float = 2.5, delta: float = 1.0, hist_max=(127, 127)) -> dict:
    """Symmetric two-species toggle switch: production alpha/(1+V^n) of U and
    alpha/(1+U^n) of V, degradation delta U and delta V.  Regions U > V
    (region 0: -U + V < 0) and U <= V (region 1)."""
    return dict(kind="toggle", c=[alpha, n, delta, alpha, n, delta], s=[1.0, 1.0, 1.0, 1.0],
                hist_max=list(hist_max), regions=[([-1, 1], 0)])


# ---------------------------------------------------------------------------
# the headline workloads
# ---------------------------------------------------------------------------
C1 = dict(name="schlogl_n64_T1e4", network=schlogl_classic(), n_replicas=64, t_corr=1.0, t_phase=1.0,
          T_end=1e4, x0=[85], seed=0, precision="f64", thresh="time")
C2 = dict(name="schlogl_n4096_T1e6_fim", network=schlogl_classic(), n_replicas=4096, t_corr=1.0,
          t_phase=1.0, T_end=1e6, x0=[0], x0_uniform_hi=1000, seed=0, precision="f64", thresh="time",
          T_burn=5e5)
C3 = dict(name="toggle_n16384_T1e5", network=toggle(), n_replicas=16384, t_corr=1.0, t_phase=1.0,
          T_end=1e5, x0=[49, 0], seed=0, precision="f32", thresh="time")


def batch_instances(n: int = 256, seed: int = 0, T_end: float = 1e4, n_min: int = 64, n_max: int = 65536):
    """Seeded instance list for the batched workload: half Schloegl with the
    system size V drawn from {0.5, 1, 2, 4, 8}, half toggles with the Hill
    exponent uniform in [2, 3] and production uniform in [30, 80]; replica
    counts log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        R = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        if i % 2 == 0:
            V = float(rng.choice([0.5, 1.0, 2.0, 4.0, 8.0]))
            net = schlogl_classic(V=V)
            x0 = [int(round(85 * V))]
        else:
            hill = float(rng.uniform(2.0, 3.0))
            alpha = float(rng.uniform(30.0, 80.0))
            # alpha + 10 sd of Poisson(alpha) + 20: no excursion reaches it
            hm = int(max(63, np.ceil(alpha + 10.0 * np.sqrt(alpha) + 20.0)))
            net = toggle(alpha=alpha, n=hill, hist_max=(hm, hm))
            x0 = [int(alpha), 0]
        out.append(dict(network=net, n_replicas=R, t_corr=1.0, t_phase=1.0, T_end=T_end, x0=x0,
                        seed=int(rng.integers(0, 2**63)), precision="f32", thresh="time"))
    return out


def serve_requests(rate: float = 200.0, seconds: float = 60.0, seed: int = 0, n_min: int = 64, n_max: int = 65536,
                   T_min: float = 1e3, T_max: float = 1e5):
    """Seeded request stream for the serving workload: Poisson arrivals at
    `rate` per second for `seconds`; each request a Schloegl or toggle
    instance (50/50, parameters drawn as in batch_instances), replica count
    log-uniform in [n_min, n_max], T_end log-uniform in [T_min, T_max].
    Returns a list of (arrival time in seconds, instance dict)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= seconds:
            break
        R = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        T_end = float(np.exp(rng.uniform(np.log(T_min), np.log(T_max))))
        if rng.random() < 0.5:
            V = float(rng.choice([0.5, 1.0, 2.0, 4.0, 8.0]))
            net = schlogl_classic(V=V)
            x0 = [int(round(85 * V))]
        else:
            hill = float(rng.uniform(2.0, 3.0))
            alpha = float(rng.uniform(30.0, 80.0))
            hm = int(max(63, np.ceil(alpha + 10.0 * np.sqrt(alpha) + 20.0)))
            net = toggle(alpha=alpha, n=hill, hist_max=(hm, hm))
            x0 = [int(alpha), 0]
        out.append((t, dict(network=net, n_replicas=R, t_corr=1.0, t_phase=1.0, T_end=T_end, x0=x0,
                            seed=int(rng.integers(0, 2**63)), thresh="time")))
    return out
