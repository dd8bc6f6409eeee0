"""Exact references for the ParRep oracle -- TEST INFRASTRUCTURE ONLY.

Each function is a plain definition written out in numpy/scipy:

* ``schlogl_props`` -- the Schloegl propensities of Table I (Sec. V.A) in the
  form lambda_j = c_j s_j h_j(x), h = (x(x-1), x(x-1)(x-2), 1, x).
* ``bd_stationary`` -- the stationary law of a birth-death chain by the
  detailed-balance product formula pi(x+1)/pi(x) = b(x)/d(x+1), truncated.
* ``generator`` / ``stationary_dense`` -- the generator Q of Eq. (1) and the
  solution of pi Q = 0 (a check on the product formula).
* ``toggle_stationary`` -- the truncated chemical master equation (Eq. 2) at
  steady state for the two-species toggle switch, solved with scipy.sparse.
* ``qsd_dtmc`` / ``qsd_ctmc`` -- quasi-stationary distributions in a set W
  (Sec. III.A): principal left eigenvectors of the jump-chain matrix or of Q
  restricted to W.
* ``bd_mfpt`` -- mean first passage time of a birth-death chain (textbook sum).
* ``bd_decorrelated_exit_rate`` -- the stationary rate of the exits that
  follow a completed TIME-mode decorrelation (Algorithm 1): the rate at which
  an exact ParRep run should see parallel-step escapes.
* ``fim_exact`` / ``rer_exact`` -- the path-space FIM (Appendix A form
  E_pi sum_j lambda_j grad log lambda_j grad log lambda_j^T) and the relative
  entropy rate E_pi sum_j [lambda_j log(lambda_j/lambda'_j) - lambda_j + lambda'_j].
* ``rre_fixed_points`` -- the real roots of the Schloegl rate equation (Sec. V.A).
* ``iaf_exact`` -- the integrated autocovariance of f (Sec. IV.B; the
  appendix's integral of Cov_f over the real line) from the Poisson equation
  Q g = -fbar.
* ``stationary_sensitivity`` -- d pi(f)/d c_k by differentiating pi Q = 0
  (the CME linear system behind Table III's approximated sensitivities).
* ``genetic_*`` -- the genetic switch of Sec. V.B (Table IV with the
  switching rates F, G): propensities and their parameter derivatives, the
  truncated three-dimensional generator, its stationary law and IAFs (sparse
  solves), and the equilibria of the rescaled rate equations.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# propensities (plain formulas, vectorised over states)
# ---------------------------------------------------------------------------
def schlogl_props(c, s, x):
    x = np.asarray(x, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    h = np.stack([x * (x - 1.0), x * (x - 1.0) * (x - 2.0), np.ones_like(x), x])
    return (c * s)[:, None] * h  # (4, len(x))


def toggle_props(c, U, V):
    aU, nU, dU, aV, nV, dV = [float(v) for v in c]
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    return np.stack([aU / (1.0 + V ** nU), aV / (1.0 + U ** nV), dU * U, dV * V])


def toggle_grad_log(c, U, V):
    """d log lambda_j / d c_k, shape (4, 6, n)."""
    aU, nU, dU, aV, nV, dV = [float(v) for v in c]
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    g = np.zeros((4, 6) + U.shape)
    g[0, 0] = 1.0 / aU
    with np.errstate(divide="ignore", invalid="ignore"):
        pV = V ** nU
        g[0, 1] = np.where(V > 0, -pV * np.log(np.where(V > 0, V, 1.0)) / (1.0 + pV), 0.0)
        pU = U ** nV
        g[1, 4] = np.where(U > 0, -pU * np.log(np.where(U > 0, U, 1.0)) / (1.0 + pU), 0.0)
    g[1, 3] = 1.0 / aV
    g[2, 2] = 1.0 / dU
    g[3, 5] = 1.0 / dV
    return g


# ---------------------------------------------------------------------------
# birth-death chains
# ---------------------------------------------------------------------------
def bd_stationary(birth, death):
    """pi on {0..n-1} for birth rates b(x) (x -> x+1) and death rates d(x)
    (x -> x-1), by pi(x+1)/pi(x) = b(x)/d(x+1), computed in log space."""
    b = np.asarray(birth, dtype=np.float64)
    d = np.asarray(death, dtype=np.float64)
    logr = np.log(b[:-1]) - np.log(d[1:])
    logpi = np.concatenate([[0.0], np.cumsum(logr)])
    logpi -= logpi.max()
    pi = np.exp(logpi)
    return pi / pi.sum()


def schlogl_stationary(c, s, xmax):
    x = np.arange(xmax + 1)
    lam = schlogl_props(c, s, x)
    return bd_stationary(lam[0] + lam[2], lam[1] + lam[3])


def generator(rates_up, rates_down):
    """Dense generator Q (Eq. 1) of a birth-death chain truncated to n states
    (births out of the last state and deaths out of state 0 are dropped)."""
    up = np.asarray(rates_up, dtype=np.float64)
    dn = np.asarray(rates_down, dtype=np.float64)
    n = len(up)
    Q = np.zeros((n, n))
    for x in range(n):
        if x + 1 < n:
            Q[x, x + 1] = up[x]
        if x - 1 >= 0:
            Q[x, x - 1] = dn[x]
        Q[x, x] = -Q[x].sum()
    return Q


def stationary_dense(Q):
    """Solves pi Q = 0, sum pi = 1 by a dense least-squares solve."""
    n = Q.shape[0]
    A = np.vstack([Q.T, np.ones((1, n))])
    rhs = np.zeros(n + 1)
    rhs[-1] = 1.0
    pi, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return pi


def bd_mfpt(birth, death, x_from, x_to):
    """Mean first passage time from x_from up to x_to > x_from of a birth-death
    chain reflecting at 0: sum_{y=x_from}^{x_to-1} 1/(b(y) pi(y)) * sum_{z<=y} pi(z)
    with pi the (unnormalised) product-form weights."""
    b = np.asarray(birth, dtype=np.float64)
    d = np.asarray(death, dtype=np.float64)
    n = x_to + 1
    logr = np.log(b[: n - 1]) - np.log(d[1:n])
    logw = np.concatenate([[0.0], np.cumsum(logr)])
    t = 0.0
    for y in range(x_from, x_to):
        # sum_{z<=y} w(z) / (b(y) w(y))
        t += np.sum(np.exp(logw[: y + 1] - logw[y])) / b[y]
    return t


def bd_mfpt_down(birth, death, x_from, x_to, xmax):
    """Mean first passage time from x_from down to x_to < x_from, truncated at xmax."""
    b = np.asarray(birth, dtype=np.float64)[::-1][: xmax + 1]
    d = np.asarray(death, dtype=np.float64)[::-1][: xmax + 1]
    # reflect: state y -> xmax - y, births become deaths
    return bd_mfpt(d, b, xmax - x_from, xmax - x_to)


def bd_decorrelated_exit_rate(birth, death, split, t_corr):
    """Escapes per unit time that follow a completed decorrelation step (the
    sum of the two regions' terms of bd_decorrelated_exit_rates)."""
    lo, hi = bd_decorrelated_exit_rates(birth, death, split, t_corr)
    return lo + hi


def bd_decorrelated_exit_rates(birth, death, split, t_corr):
    """Escapes per unit time that follow a completed decorrelation step, out of
    W- and out of W+ separately: (J S-(t), J S+(t)) in the notation below.

    Birth-death chain on {0..n-1}, regions W- = {x < split} and W+ = {x >=
    split}.  In the TIME form of Algorithm 1's decorrelation the in-W time is
    the sum of the holding times of the jumps that stayed in W since the chain
    entered W, and the step ends at the first such jump with in-W time >=
    t_corr; the dephasing and parallel steps then produce the one exit that
    ends this sojourn.  So an exact ParRep run has one parallel-step escape per
    sojourn whose first jump at or after t_corr stays in W.

    A sojourn in W+ starts at `split` (entered from split-1) and one in W- at
    split-1.  By detailed balance both entries happen at the stationary flux
    J = pi(split-1) b(split-1) = pi(split) d(split), and sojourns are i.i.d.
    given their entry state, so the rate is J (S-(t) + S+(t)) with
        S_W(t) = sum_x P_entry(X_t = x, no exit by t) (1 - p_exit(x)),
    P = exp(t Q_W) (Q restricted to W, exits killed) and p_exit(x) the
    probability that the next jump from x leaves W.

    Q_W is reversible with respect to pi on W, so D^(1/2) Q_W D^(-1/2) (D =
    diag pi) is the symmetric tridiagonal matrix with diagonal -a0(x) and
    off-diagonal sqrt(b(x) d(x+1)); exp(t Q_W) comes from its eigenpairs,
    which stays exact for the stiff generators (rates up to 1e5) where a
    Krylov or Pade exponential is slow."""
    from scipy.linalg import eigh_tridiagonal

    b = np.asarray(birth, dtype=np.float64).copy()
    d = np.asarray(death, dtype=np.float64).copy()
    n = len(b)
    b[-1] = 0.0  # truncation: no births out of the last state
    d[0] = 0.0
    pi = bd_stationary(b, d)
    J = pi[split - 1] * b[split - 1]
    terms = []
    for lo, hi, entry in ((0, split - 1, split - 1), (split, n - 1, split)):
        xs = np.arange(lo, hi + 1)
        a0 = b[xs] + d[xs]  # every jump leaves the state (exits are killed)
        out = np.zeros(len(xs))  # rate of the jump that leaves W
        if entry == split - 1:
            out[-1] = b[split - 1]
        else:
            out[0] = d[split]
        p_stay = np.where(a0 > 0, 1.0 - out / np.where(a0 > 0, a0, 1.0), 0.0)
        w = pi[xs] / pi[xs].sum()
        lam, V = eigh_tridiagonal(-a0, np.sqrt(b[xs][:-1] * d[xs][1:]))
        e = entry - lo
        coef = V.T @ (np.sqrt(w) * p_stay)
        terms.append(J * float(np.sum(V[e] * np.exp(lam * float(t_corr)) * coef) / np.sqrt(w[e])))
    return terms[0], terms[1]


# ---------------------------------------------------------------------------
# two-species toggle switch: truncated CME at steady state
# ---------------------------------------------------------------------------
def toggle_generator(c, Umax, Vmax):
    nU, nV = Umax + 1, Vmax + 1
    U, V = np.meshgrid(np.arange(nU), np.arange(nV), indexing="ij")
    U = U.ravel()
    V = V.ravel()
    lam = toggle_props(c, U, V)
    idx = U * nV + V
    rows, cols, vals = [], [], []
    moves = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    out = np.zeros(len(idx))
    for j, (du, dv) in enumerate(moves):
        U2, V2 = U + du, V + dv
        ok = (U2 >= 0) & (U2 <= Umax) & (V2 >= 0) & (V2 <= Vmax)
        rows.append(idx[ok])
        cols.append((U2 * nV + V2)[ok])
        vals.append(lam[j][ok])
        out += np.where(ok, lam[j], 0.0)
    rows.append(idx)
    cols.append(idx)
    vals.append(-out)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(len(idx), len(idx)))


def toggle_stationary(c, Umax, Vmax):
    """Stationary law on [0,Umax] x [0,Vmax] (truncated CME, reflecting edges),
    returned as an array of shape (Umax+1, Vmax+1)."""
    Q = toggle_generator(c, Umax, Vmax)
    n = Q.shape[0]
    QT = Q.T.tocsr()

    def solve(row):
        # pi Q = 0 with the equation of state `row` replaced by sum(pi) = 1
        A = QT.tolil()
        A[row, :] = np.ones(n)
        rhs = np.zeros(n)
        rhs[row] = 1.0
        return spla.spsolve(A.tocsc(), rhs)

    pi = solve(0)
    pi = solve(int(np.argmax(pi)))  # a well-conditioned normalisation row
    pi = np.maximum(pi, 0.0)
    pi /= pi.sum()
    return pi.reshape(Umax + 1, Vmax + 1)


# ---------------------------------------------------------------------------
# quasi-stationary distributions (Sec. III.A)
# ---------------------------------------------------------------------------
def qsd_dtmc(P_W):
    """QSD of a DTMC in W: principal left eigenvector of the sub-stochastic
    jump matrix restricted to W.  Returns (nu, lambda) with P(N > n) = lambda^n."""
    w, vl = np.linalg.eig(P_W.T)
    i = int(np.argmax(w.real))
    nu = np.abs(vl[:, i].real)
    return nu / nu.sum(), float(w[i].real)


def qsd_ctmc(Q_W):
    """QSD of a CTMC in W: principal left eigenvector of Q restricted to W."""
    w, vl = np.linalg.eig(Q_W.T)
    i = int(np.argmax(w.real))
    nu = np.abs(vl[:, i].real)
    return nu / nu.sum(), float(w[i].real)


def bd_jump_matrix(birth, death):
    """Jump (embedded) chain of a birth-death chain on {0..n-1}."""
    b = np.asarray(birth, dtype=np.float64)
    d = np.asarray(death, dtype=np.float64)
    n = len(b)
    P = np.zeros((n, n + 2))  # columns: -1 .. n (off-range moves kept as exits)
    a0 = b + d
    for x in range(n):
        P[x, x + 2] = b[x] / a0[x]
        P[x, x] = d[x] / a0[x]
    return P[:, 1:-1], P


# ---------------------------------------------------------------------------
# path-space FIM and relative entropy rate (Appendix A)
# ---------------------------------------------------------------------------
def fim_exact(lam, grad, weights):
    """sum_x w(x) sum_j lambda_j(x) g_j(x) g_j(x)^T; lam (m, n), grad (m, l, n)."""
    return np.einsum("n,jn,jan,jbn->ab", weights, lam, grad, grad)


def rer_exact(lam, lam_p, weights):
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(lam > 0, lam * np.log(lam / lam_p), 0.0) - lam + lam_p
    return float(np.sum(weights * t.sum(axis=0)))


def schlogl_grad_log(c, x):
    n = len(np.atleast_1d(x))
    g = np.zeros((4, 4, n))
    for j in range(4):
        g[j, j] = 1.0 / c[j]
    return g


def rre_fixed_points(c, s, V=1.0):
    """Real non-negative roots of d x/dt = A1 x^2 - A2 x^3 + A3 - A4 x (the
    large-population limit of Table I written in population units)."""
    A = np.asarray(c, dtype=np.float64) * np.asarray(s, dtype=np.float64)
    r = np.roots([-A[1], A[0], -A[3], A[2]])
    r = np.sort(r[np.abs(r.imag) < 1e-9].real)
    return r[r >= 0]


# ---------------------------------------------------------------------------
# stationary sensitivity and the integrated autocovariance (Sec. IV.B and the
# appendix that derives the information bounds)
# ---------------------------------------------------------------------------
def schlogl_generators(c, s, xmax):
    """Truncated Schloegl generator Q on {0..xmax} (births out of xmax and
    deaths out of 0 dropped) and its derivatives dQ/dc_k, k = 0..3.  Channels
    0 and 2 move x up, 1 and 3 down; lambda_j is linear in c_j, so dQ/dc_k is
    the generator of channel k alone with rates s_k h_k(x)."""
    x = np.arange(xmax + 1)
    lam = schlogl_props(c, s, x)
    Q = generator(lam[0] + lam[2], lam[1] + lam[3])
    one = schlogl_props(np.ones(4), s, x)  # s_k h_k(x) = d lambda_k / d c_k
    zero = np.zeros(xmax + 1)
    dQ = []
    for k in range(4):
        up = one[k] if k in (0, 2) else zero
        dn = one[k] if k in (1, 3) else zero
        dQ.append(generator(up, dn))
    return Q, dQ


def _bordered_solve(A, rhs, border):
    """Solves A y + mu * 1 = rhs, border . y = 0 (A singular with null space
    the constants); returns y."""
    n = A.shape[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A
    M[:n, n] = 1.0
    M[n, :n] = border
    y = np.linalg.solve(M, np.concatenate([rhs, [0.0]]))
    return y[:n]


def iaf_exact(Q, pi, f):
    """Integrated autocovariance of f along the stationary chain,
    tau(f) = integral over the real line of Cov_pi(f(X_0), f(X_s)) ds
    = 2 sum_x pi(x) fbar(x) g(x), where fbar = f - pi(f) and
    g = integral_0^inf exp(sQ) fbar ds solves the Poisson equation
    Q g = -fbar with pi . g = 0."""
    Q = np.asarray(Q, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    fbar = np.asarray(f, dtype=np.float64) - float(pi @ np.asarray(f, dtype=np.float64))
    g = _bordered_solve(Q, -fbar, pi)
    return 2.0 * float(np.sum(pi * fbar * g))


def stationary_sensitivity(Q, dQ, pi, f):
    """d pi(f) / d c_k for each generator derivative dQ_k: differentiating
    pi Q = 0 and sum pi = 1 gives Q^T dpi = -dQ_k^T pi with sum dpi = 0."""
    Q = np.asarray(Q, dtype=np.float64)
    pi = np.asarray(pi, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    out = []
    for dQk in dQ:
        dpi = _bordered_solve(Q.T, -(np.asarray(dQk).T @ pi), np.ones(len(pi)))
        out.append(float(dpi @ f))
    return np.array(out)


# ---------------------------------------------------------------------------
# genetic switch with positive feedback (Sec. V.B): DNA state xi in {0, 1},
# mRNA m, protein p; six channels (Table IV and the switching rates F, G)
# ---------------------------------------------------------------------------
GENETIC_PARAMS = ("a", "b", "gamma", "k0min", "k0max", "k1min", "k1max", "D")


def genetic_paper_params():
    """Sec. V.B's values: b = 22.5, a = 2400/b, gamma = 50, k0min = k1min =
    24/b, k0max = k1max = 2400/b, D = 1000, in the order of GENETIC_PARAMS."""
    b = 22.5
    return np.array([2400.0 / b, b, 50.0, 24.0 / b, 2400.0 / b, 24.0 / b, 2400.0 / b, 1000.0])


def genetic_props(c, xi, m, p):
    """Propensities of the six channels, shape (6, n): transcription a xi,
    mRNA decay gamma m, translation gamma b m, protein decay p, activation
    F(p) (1 - xi), deactivation G(p) xi, with h = p^2/(p^2 + D^2),
    F = k0min + (k0max - k0min) h and G = k1max - (k1max - k1min) h."""
    a, b, g, k0n, k0x, k1n, k1x, D = [float(v) for v in c]
    xi, m, p = (np.asarray(v, dtype=np.float64) for v in (xi, m, p))
    h = p * p / (p * p + D * D)
    F = k0n + (k0x - k0n) * h
    G = k1x - (k1x - k1n) * h
    return np.stack([a * xi, g * m, g * b * m, p, F * (1.0 - xi), G * xi])


def genetic_grad_props(c, xi, m, p):
    """d lambda_j / d c_k, shape (6, 8, n), the parameters taken independent."""
    a, b, g, k0n, k0x, k1n, k1x, D = [float(v) for v in c]
    xi, m, p = (np.asarray(v, dtype=np.float64) for v in (xi, m, p))
    h = p * p / (p * p + D * D)
    dh_dD = -2.0 * p * p * D / (p * p + D * D) ** 2
    out = np.zeros((6, 8) + xi.shape)
    out[0, 0] = xi
    out[1, 2] = m
    out[2, 1] = g * m
    out[2, 2] = b * m
    out[4, 3] = (1.0 - h) * (1.0 - xi)
    out[4, 4] = h * (1.0 - xi)
    out[4, 7] = (k0x - k0n) * dh_dD * (1.0 - xi)
    out[5, 5] = h * xi
    out[5, 6] = (1.0 - h) * xi
    out[5, 7] = -(k1x - k1n) * dh_dD * xi
    return out


def genetic_states(m_max, p_max):
    """All (xi, m, p) of the truncated space, flattened in (p, m, xi) order."""
    p, m, xi = np.meshgrid(np.arange(p_max + 1), np.arange(m_max + 1), np.arange(2), indexing="ij")
    return xi.ravel(), m.ravel(), p.ravel()


def genetic_generator(c, m_max, p_max):
    """Sparse generator of the chain on {0,1} x [0, m_max] x [0, p_max]
    (moves that would leave the box are dropped)."""
    xi, m, p = genetic_states(m_max, p_max)
    lam = genetic_props(c, xi, m, p)
    nm = m_max + 1
    idx = (p * nm + m) * 2 + xi
    moves = [(0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 0, 0), (-1, 0, 0)]
    rows, cols, vals = [], [], []
    out = np.zeros(len(idx))
    for j, (dxi, dm, dp) in enumerate(moves):
        xi2, m2, p2 = xi + dxi, m + dm, p + dp
        ok = (xi2 >= 0) & (xi2 <= 1) & (m2 >= 0) & (m2 <= m_max) & (p2 >= 0) & (p2 <= p_max) & (lam[j] > 0)
        rows.append(idx[ok])
        cols.append(((p2 * nm + m2) * 2 + xi2)[ok])
        vals.append(lam[j][ok])
        out += np.where(ok, lam[j], 0.0)
    rows.append(idx)
    cols.append(idx)
    vals.append(-out)
    n = len(idx)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def _solve_pinned(A, rhs, r):
    """Solves A y = rhs with equation r replaced by y(r) = rhs[r] (sparse LU)."""
    A = A.tolil(copy=True)
    A.rows[r] = [r]
    A.data[r] = [1.0]
    return spla.splu(A.tocsc()).solve(rhs)


def genetic_stationary(c, m_max, p_max, pin=None):
    """pi Q = 0, sum pi = 1 on the truncated box: Q^T w = 0 with the equation
    of state `pin` (default: a state near the upper well) replaced by
    w(pin) = 1, then pi = w / sum w."""
    Q = genetic_generator(c, m_max, p_max)
    n = Q.shape[0]
    r = ((min(1840, p_max) * (m_max + 1)) + min(2, m_max)) * 2 + 1 if pin is None else pin
    rhs = np.zeros(n)
    rhs[r] = 1.0
    w = _solve_pinned(Q.T, rhs, r)
    w = np.maximum(w, 0.0)
    return Q, w / w.sum()


def iaf_exact_sparse(Q, pi, f, pin=None):
    """iaf_exact for a sparse generator: Q g = -fbar with the equation of
    state `pin` replaced by g(pin) = 0 (it follows from the others, since
    pi . Q g = 0 = -pi . fbar); the constant left free in g does not change
    sum pi fbar g."""
    f = np.asarray(f, dtype=np.float64)
    fbar = f - float(pi @ f)
    r = int(np.argmax(pi)) if pin is None else pin
    rhs = -fbar.copy()
    rhs[r] = 0.0
    g = _solve_pinned(Q, rhs, r)
    return 2.0 * float(np.sum(pi * fbar * g))


def genetic_rre_fixed_points(c):
    """Equilibria of the rescaled rate equations of Sec. V.B:
    dX1/dt = a F/(F+G) - gamma X1, dX2/dt = gamma b X1 - X2.  At rest
    X1 = X2/(gamma b) and a F(X2)/(F(X2)+G(X2)) = X2/b; the roots in X2 are
    bracketed on a fine grid and refined by bisection."""
    a, b, g, k0n, k0x, k1n, k1x, D = [float(v) for v in c]

    def r(X2):
        h = X2 * X2 / (X2 * X2 + D * D)
        F = k0n + (k0x - k0n) * h
        G = k1x - (k1x - k1n) * h
        return a * F / (F + G) - X2 / b

    grid = np.linspace(0.0, 4.0 * a * b, 400001)
    val = r(grid)
    roots = []
    for i in np.nonzero(np.sign(val[:-1]) != np.sign(val[1:]))[0]:
        lo, hi = grid[i], grid[i + 1]
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if np.sign(r(mid)) == np.sign(r(lo)):
                lo = mid
            else:
                hi = mid
        X2 = 0.5 * (lo + hi)
        roots.append((X2 / (g * b), X2))
    return roots
