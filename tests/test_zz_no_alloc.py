"""parrep_ssa_noalloc: the plain-SSA entry point for callers that cannot
allocate device memory (a framework that owns the whole memory pool, or a
loop where cudaMalloc/cudaFree would synchronise the device).  It keeps its
scratch in a fixed array inside the library; its results must equal those of
parrep_ssa, call after call (the array is shared and must be cleared).

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_1705_06807_gb300 import _lib as L
from paper_1705_06807_gb300 import configs as K
from paper_1705_06807_gb300.api import ParRepError, parrep_ssa, parrep_ssa_noalloc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("spec,x0,T", [(K.schlogl_classic(), [85], 3.0),
                                        (K.toggle(alpha=20, n=2.5, hist_max=(63, 63)), [15, 2], 40.0)])
def test_noalloc_matches_allocating_entry_point_twice(spec, x0, T, precision):
    import torch

    ref, ev_ref, _ = parrep_ssa(spec, 53, x0, T, 21, precision=precision)
    # the same kernel sums the same fixed-point holding times: the normalised
    # histograms are identical, not merely close
    for call in range(2):
        out = torch.full((ref.size,), -1.0, dtype=torch.float64, device="cuda")
        ev = parrep_ssa_noalloc(spec, 53, x0, T, 21, out, precision=precision)
        assert ev == ev_ref, call
        assert np.array_equal(out.cpu().numpy(), ref), call
    # a host output buffer works too
    host = np.zeros(ref.size)
    assert parrep_ssa_noalloc(spec, 53, x0, T, 21, host, precision=precision) == ev_ref
    assert np.array_equal(host, ref)


def _code(fn):
    with pytest.raises(ParRepError) as e:
        fn()
    return e.value.code


def test_noalloc_rejects_sizes_beyond_its_scratch():
    spec = dict(K.toggle(hist_max=(300, 300)))  # 90601 bins > 65536
    assert _code(lambda: parrep_ssa_noalloc(spec, 4, [10, 10], 1.0, 0, np.zeros(301 * 301))) == L.PARREP_EINVAL
    # 4097 states of one species: fewer bins than the limit, more states than the tables hold
    sch = dict(K.schlogl_classic(), hist_max=4096)
    assert _code(lambda: parrep_ssa_noalloc(sch, 4, [85], 1.0, 0, np.zeros(4097))) == L.PARREP_EINVAL


def test_noalloc_rejects_what_the_allocating_entry_point_rejects():
    bad_hill = dict(K.toggle(alpha=20, n=2.5, hist_max=(63, 63)))
    bad_hill["c"] = list(bad_hill["c"])
    bad_hill["c"][1] = float("nan")
    neg_rate = dict(K.schlogl_classic())
    neg_rate["c"] = list(neg_rate["c"])
    neg_rate["c"][3] = -3.5
    for spec, x0 in [(bad_hill, [15, 2]), (neg_rate, [85])]:
        nb = int(np.prod(np.atleast_1d(spec["hist_max"]) + 1))
        assert _code(lambda: parrep_ssa(spec, 4, x0, 1.0, 0)) == L.PARREP_EINVAL
        assert _code(lambda: parrep_ssa_noalloc(spec, 4, x0, 1.0, 0, np.zeros(nb))) == L.PARREP_EINVAL


def test_noalloc_range_error_does_not_leak_into_the_next_call():
    # 64 Schloegl chains confined to [0, 100] and started at its edge leave it
    # within a few jumps: ERANGE; the next, valid call must be clean
    small = dict(K.schlogl_classic(), hist_max=100)
    assert _code(lambda: parrep_ssa_noalloc(small, 64, [100], 50.0, 3, np.zeros(101))) == L.PARREP_ERANGE
    spec = K.schlogl_classic()
    ref, ev_ref, _ = parrep_ssa(spec, 53, [85], 2.0, 9)
    host = np.zeros(ref.size)
    assert parrep_ssa_noalloc(spec, 53, [85], 2.0, 9, host) == ev_ref
    assert np.array_equal(host, ref)
