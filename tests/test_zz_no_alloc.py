"""The allocation-free field sum (lbm_field_sum_noalloc) against the context's own FP64 mass.

Callers that cannot allocate device memory use lbm_field_sum_noalloc, whose working memory is a
file-scope device array of the library.  This file is collected last so that a run stopping at
the first failure has already run every other test; it also passes when run on its own.
"""
import numpy as np
import pytest

import workloads as W
from tests._parity import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_sum_matches_context_mass_twice_in_a_row():
    import torch
    from paper_2201_06039_gb300 import lbm
    case = W.pool_boiling(40, 36, 48, height=16.0, hot_sigma=4.0)
    rho, T, u = inputs(case)
    lat = lbm.Lattice(lbm.params_from_setup(case["setup"]))
    lat.init(rho, T)
    lat.step(7)
    mass, _, _ = lat.totals()                       # existing entry point (context scratch)
    d_rho = torch.empty(case["setup"].shape, dtype=torch.float32, device="cuda")
    lbm.lbm_get_moments(lat.ctx, d_rho, None, None, None, None)
    n = d_rho.numel()
    for _ in range(2):                              # two calls in a row share the scratch
        s = lbm.lbm_field_sum_noalloc(d_rho, n)
        assert abs(s / mass - 1.0) < 1e-12, (s, mass)
    # an exactly representable case: every partial sum is exact in FP64
    ones = torch.ones(1234567, dtype=torch.float32, device="cuda")
    assert lbm.lbm_field_sum_noalloc(ones, ones.numel()) == 1234567.0
    assert lbm.lbm_field_sum_noalloc(ones, 0) == 0.0
    lat.close()


def test_noalloc_sum_rejects_sizes_beyond_the_maximum():
    import torch
    from paper_2201_06039_gb300 import lbm
    x = torch.ones(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:               # raw pointer: the library's own check
        lbm.lbm_field_sum_noalloc(x.data_ptr(), lbm.LBM_NOALLOC_MAX_ELEMENTS + 1)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "exceeds the maximum" in str(ei.value)


def test_noalloc_sum_rejects_host_memory_and_ranges_past_the_buffer():
    """Bad inputs are refused on the host before any launch: a host pointer, a tensor count above
    the tensor's size (wrapper) and a raw-pointer range that runs past the allocation (library)."""
    import torch
    from paper_2201_06039_gb300 import lbm
    host = np.ones(64, dtype=np.float32)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_field_sum_noalloc(host.ctypes.data, 64)
    assert ei.value.status == lbm.LBM_EINVAL and "host memory" in str(ei.value)
    x = torch.ones(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        lbm.lbm_field_sum_noalloc(x, 1001)
    with pytest.raises(ValueError):
        lbm.lbm_field_sum_noalloc(x.cpu(), 10)
    # a raw pointer with a count far past its (caching-allocator) block is refused by the library
    y = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_field_sum_noalloc(y.data_ptr(), (1 << 31) - 1)
    assert ei.value.status == lbm.LBM_EINVAL and "past the end" in str(ei.value)
    # the context stays usable: a valid call right after the refusals
    assert lbm.lbm_field_sum_noalloc(x, 1000) == 1000.0
