"""The binary32 direct-method choice of a +-1 chain by integer thresholds.

The FP32 Schloegl chain of the library decides a step by comparing the
23-bit index k of the uniform u = (k + 1/2) 2^-23 with three per-state
thresholds (K0, K1, D): the chain goes up iff k < K0 or 0 <= k - K1 < D.  The
reading behind it: RN(u a0) does not decrease with k, so every comparison
"c_j <= RN(u a0)" of the direct method (Sec. II) flips at one index, found by
bisection; and the rounding case (no cumulative sum above the target) takes
the last channel with positive propensity.  These tests check that reading
exhaustively -- all 2^23 indices -- against the binary32 direct method as the
oracle's binary32 mode takes it, for states across the Schloegl range.  No GPU.
"""
import numpy as np
import pytest

from paper_1705_06807_gb300 import configs as K

F32 = np.float32
KS = np.arange(1 << 23, dtype=np.int64)
U = ((KS.astype(F32) + F32(0.5)) * F32(2.0 ** -23)).astype(F32)


def _props(spec, x):
    """Binary32 Schloegl propensities in the oracle's operation order."""
    c, s = spec["c"], spec["s"]
    xf = F32(x)
    h1 = F32(xf * F32(xf - F32(1.0)))
    h2 = F32(h1 * F32(xf - F32(2.0)))
    return [F32(F32(c[0] * s[0]) * h1), F32(F32(c[1] * s[1]) * h2), F32(c[2] * s[2]), F32(F32(c[3] * s[3]) * xf)]


def _direct_up(lam):
    """Up (channel 0 or 2) for every index: the first j with c_j > t, else the
    last channel with positive propensity -- left-to-right binary32 sums."""
    c0 = lam[0]
    c1 = F32(c0 + lam[1])
    c2 = F32(c1 + lam[2])
    a0 = F32(c2 + lam[3])
    t = (U * a0).astype(F32)
    J = (c0 <= t).astype(np.int64) + (c1 <= t) + (c2 <= t) + (a0 <= t)
    last = 3 if lam[3] > 0 else 2 if lam[2] > 0 else 1 if lam[1] > 0 else 0
    J = np.where(J == 4, last, J)
    return (J == 0) | (J == 2)


def _first_k_at_least(a0, c):
    lo, hi = 0, 1 << 23
    while lo < hi:
        mid = (lo + hi) // 2
        if F32(F32(F32(mid) + F32(0.5)) * F32(2.0 ** -23)) * a0 >= c:
            hi = mid
        else:
            lo = mid + 1
    return lo


def _threshold_up(lam):
    c0 = lam[0]
    c1 = F32(c0 + lam[1])
    c2 = F32(c1 + lam[2])
    a0 = F32(c2 + lam[3])
    K0, K1, K2 = (_first_k_at_least(a0, c) for c in (c0, c1, c2))
    last = 3 if lam[3] > 0 else 2 if lam[2] > 0 else 1 if lam[1] > 0 else 0
    D = (1 << 23) - K1 if last % 2 == 0 else K2 - K1
    return (KS < K0) | ((KS - K1 >= 0) & (KS - K1 < D))


@pytest.mark.parametrize("V", [1.0, 0.5])
def test_thresholds_reproduce_the_binary32_choice_for_every_index(V):
    spec = K.schlogl_classic(V=V)
    hm = spec["hist_max"]
    states = sorted({0, 1, 2, 3, 85, 250, 251, 565, hm - 1, hm} | set(range(5, hm, max(1, hm // 12))))
    flips = 0
    for x in states:
        lam = _props(spec, x)
        want = _direct_up(lam)
        got = _threshold_up(lam)
        assert np.array_equal(want, got), f"state {x}: {np.flatnonzero(want != got)[:5]}"
        flips += int(np.count_nonzero(want[1:] != want[:-1]))
    # the up set is at most two intervals: at most three flips per state
    assert 0 < flips <= 3 * len(states)


def test_rounding_rule_states():
    """x = 0: only the constant birth channel has a positive propensity, so
    a0 equals the last nonzero cumulative sum and every index goes up; the
    threshold encoding must give the same for all 2^23 indices."""
    spec = K.schlogl_classic()
    lam = _props(spec, 0)
    assert lam[0] == 0 and lam[1] == 0 and lam[3] == 0 and lam[2] > 0
    assert _direct_up(lam).all() and _threshold_up(lam).all()
