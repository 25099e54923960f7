"""The allocation-free Barnes-Hut entry point (mm_repulsion_noalloc).

It exists for callers that cannot allocate device memory on their path
(custom or pool allocators that forbid outside allocations, real-time loops
that cannot take cudaFree's synchronisation): its tree workspace is a fixed
static device array inside the library.  It must give the same forces as the
allocating entry point mm_repulsion on the same input, call after call, since
every call reuses (and finds the previous contents in) the same array.

This file is collected last on purpose so a failure here never hides another
test's result.
"""
import numpy as np
import pytest
import torch

from paper_1506_04383_gb300 import graphs

pytestmark = pytest.mark.gpu


def _inv_dist_sum(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(len(x))
    for i in range(0, len(x), 512):
        d = np.sqrt(((x[i:i + 512, None, :] - x[None, :, :]) ** 2).sum(-1))
        with np.errstate(divide="ignore"):
            out[i:i + 512] = np.where(d > 0, 1.0 / d, 0.0).sum(1)
    return out


def test_noalloc_matches_allocating_entry_point_twice(mm):
    # two calls in a row with different sizes and inputs: the second call
    # finds the first call's tree in the shared scratch
    for n, seed, theta in ((20000, 11, 0.5), (7001, 12, 0.7)):
        x = graphs.uniform_positions(n, seed, 0.0, 100.0).astype(np.float32)
        rp, col = graphs.path(n)
        p = mm.default_params(k=1, coarsest_n=n)
        h = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p)
        xd = torch.from_numpy(x).cuda()
        ref = mm.repulsion(h, 0, xd, theta).cpu().numpy()
        got = mm.repulsion_noalloc(xd, theta).cpu().numpy()
        tol = 2e-4 * _inv_dist_sum(x)[:, None]
        assert np.all(np.abs(got - ref) <= tol)


def test_noalloc_rejects_sizes_beyond_its_limit(mm):
    x = torch.zeros((32769, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.repulsion_noalloc(x, 0.5)
    assert e.value.status == 1
    assert "32768" in str(e.value)
