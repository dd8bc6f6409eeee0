"""Writes exact_references.json: exact values of the truncated chains that
bench.py and the GPU tests compare their estimates with.

Every number comes from the oracle's exact references (oracle/exact.py) and
nothing else:
  * schlogl_classic (k = 0.03, 1e-4, 200, 3.5 with factors 1/2, 1/6, 1, 1;
    regions x < 250 | x >= 250; truncated at 1500): the stationary law by the
    product formula, the lower-well mass, the mean, the diagonal of the
    path-space FIM (Appendix A form), and the rate of the escapes that follow
    a completed TIME-mode decorrelation for the listed t_corr (in all, and
    out of the lower and the upper region);
  * schlogl_v25 (Table I, a = 1, b = 2, c = (3, 0.6, 0.25, 2.95), V = 25,
    truncated at 255): the stationary law, the mean of x, its IAF, the
    stationary sensitivities of pi(x) and the FIM diagonal (Sec. V.A);
  * genetic_paper (Sec. V.B at the paper's constants, m <= 15, p <= 3500):
    the FIM diagonal over the eight parameters and the mean protein count.

  python tests/golden/make_exact_references.py      # rewrites the file
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact as E  # noqa: E402
from paper_1705_06807_gb300 import configs as K  # noqa: E402

PATH = os.path.join(HERE, "exact_references.json")
T_CORR = [0.5, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0, 12.0, 16.0]


def compute():
    out = {}
    net = K.schlogl_classic()
    hm = net["hist_max"]
    x = np.arange(hm + 1.0)
    lam = E.schlogl_props(net["c"], net["s"], x)
    b, d = lam[0] + lam[2], lam[1] + lam[3]
    pi = E.schlogl_stationary(net["c"], net["s"], hm)
    split = net["regions"][0][1]
    F = E.fim_exact(lam, E.schlogl_grad_log(net["c"], x), pi)
    out["schlogl_classic"] = {
        "hist_max": hm, "split": split, "pi": pi.tolist(), "mass_lower": float(pi[:split].sum()),
        "mean": float(pi @ x), "fim_diag": np.diag(F).tolist(),
        "decorrelated_exit_rate": {f"{t:g}": E.bd_decorrelated_exit_rate(b, d, split, t) for t in T_CORR},
        "decorrelated_exit_rates_lower_upper": {f"{t:g}": list(E.bd_decorrelated_exit_rates(b, d, split, t))
                                                for t in T_CORR},
    }
    net = K.schlogl_paper(V=25, hist_max=255)
    x = np.arange(256.0)
    pi = E.schlogl_stationary(net["c"], net["s"], 255)
    Q, dQ = E.schlogl_generators(net["c"], net["s"], 255)
    F = E.fim_exact(E.schlogl_props(net["c"], net["s"], x), E.schlogl_grad_log(net["c"], x), pi)
    out["schlogl_v25"] = {
        "hist_max": 255, "pi": pi.tolist(), "mean": float(pi @ x), "iaf_x": float(E.iaf_exact(Q, pi, x)),
        "sensitivity_x": [float(v) for v in E.stationary_sensitivity(Q, dQ, pi, x)], "fim_diag": np.diag(F).tolist(),
    }
    # the genetic switch of Sec. V.B at the paper's constants, truncated to
    # m <= 15, p <= 3500: the path-space FIM diagonal E_pi[sum_j (d lambda_j /
    # d c_k)^2 / lambda_j] (Table V), the parameters taken independently
    c = E.genetic_paper_params()
    Q, pi = E.genetic_stationary(c, 15, 3500)
    xi, m, p = E.genetic_states(15, 3500)
    lam = E.genetic_props(c, xi, m, p)
    dl = E.genetic_grad_props(c, xi, m, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(lam[:, None, :] > 0, dl**2 / lam[:, None, :], 0.0)
    out["genetic_paper"] = {"m_max": 15, "p_max": 3500, "fim_diag": (terms * pi).sum(axis=(0, 2)).tolist(),
                            "mean_p": float(pi @ p)}
    return out


if __name__ == "__main__":
    with open(PATH, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print(PATH)
