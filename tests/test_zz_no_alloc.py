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

from paper_1705_06807_gb300 import configs as K
from paper_1705_06807_gb300.api import ParRepError, parrep_ssa, parrep_ssa_noalloc

pytestmark = pytest.mark.gpu

# the tolerance of the GPU SSA parity tests: fixed-point sums of the same kernel
RTOL = 1e-12


def _atol(events, T):
    return 4e-12 * max(events, 1) + 1e-12 * T


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("spec,x0,T", [(K.schlogl_classic(), [85], 3.0),
                                        (K.toggle(alpha=20, n=2.5, hist_max=(63, 63)), [15, 2], 40.0)])
def test_noalloc_matches_allocating_entry_point_twice(spec, x0, T, precision):
    import torch

    ref, ev_ref, _ = parrep_ssa(spec, 53, x0, T, 21, precision=precision)
    for call in range(2):
        out = torch.full((ref.size,), -1.0, dtype=torch.float64, device="cuda")
        ev = parrep_ssa_noalloc(spec, 53, x0, T, 21, out, precision=precision)
        got = out.cpu().numpy()
        assert ev == ev_ref, call
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=_atol(ev_ref, 53 * T))
    # a host output buffer works too
    host = np.zeros(ref.size)
    assert parrep_ssa_noalloc(spec, 53, x0, T, 21, host, precision=precision) == ev_ref
    np.testing.assert_allclose(host, ref, rtol=RTOL, atol=_atol(ev_ref, 53 * T))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    spec = dict(K.toggle(hist_max=(300, 300)))  # 90601 bins > 65536
    with pytest.raises(ParRepError):
        parrep_ssa_noalloc(spec, 4, [10, 10], 1.0, 0, np.zeros(301 * 301))
