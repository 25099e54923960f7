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
import math

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


def test_noalloc_at_its_size_limit_then_smaller_then_at_the_limit_again(mm):
    # n = 32768 is the largest size the fixed array holds (its worst-case
    # carve); a smaller call in between leaves stale tree records beyond its
    # own 2n - 1 nodes, which the next full-size call must overwrite
    for n, seed in ((32768, 21), (5000, 22), (32768, 23)):
        x = graphs.uniform_positions(n, seed, 0.0, 50.0).astype(np.float32)
        rp, col = graphs.path(n)
        p = mm.default_params(k=1, coarsest_n=n)
        h = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p)
        xd = torch.from_numpy(x).cuda()
        ref = mm.repulsion(h, 0, xd, 0.5).cpu().numpy()
        got = mm.repulsion_noalloc(xd, 0.5).cpu().numpy()
        tol = 2e-4 * _inv_dist_sum(x)[:, None]
        assert np.all(np.abs(got - ref) <= tol), n


def test_noalloc_within_the_barnes_hut_bounds_of_the_oracle(mm):
    # against the FP64 oracle: per vertex within the multipole remainder
    # bound 2 theta^2 sum_v 1/|x_u - x_v| of the exact sum, and in RMS within
    # 5 % of the oracle's own Barnes-Hut error at the same theta
    import oracle
    n, theta = 6000, 0.5
    x = graphs.uniform_positions(n, 31, 0.0, 80.0).astype(np.float32)
    got = mm.repulsion_noalloc(torch.from_numpy(x).cuda(), theta).cpu().numpy()
    x64 = x.astype(np.float64)
    exact = oracle.repulsion_exact(x64)
    bh = oracle.repulsion_bh(x64, theta)
    inv = _inv_dist_sum(x)
    err = np.sqrt(((got - exact) ** 2).sum(1))
    assert np.all(err <= 2 * theta ** 2 * inv + 2e-4 * inv)
    rms_gpu = math.sqrt((err ** 2).mean())
    rms_orc = math.sqrt((((bh - exact) ** 2).sum(1)).mean())
    assert rms_gpu <= 1.05 * rms_orc, (rms_gpu, rms_orc)
    # theta = 0 is the exact sum
    got0 = mm.repulsion_noalloc(torch.from_numpy(x).cuda(), 0.0).cpu().numpy()
    assert np.all(np.abs(got0 - exact) <= 2e-4 * inv[:, None])


def test_noalloc_rejects_malformed_buffers(mm):
    x = torch.rand((1000, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        mm.repulsion_noalloc(x.reshape(-1), 0.5)           # flat [2n]
    with pytest.raises(ValueError):
        mm.repulsion_noalloc(x, 0.5, F_out=torch.empty((999, 2), device="cuda"))
    with pytest.raises(TypeError):
        mm.repulsion_noalloc(x, 0.5, F_out=torch.empty((1000, 2), dtype=torch.float64,
                                                       device="cuda"))
    with pytest.raises(TypeError):
        mm.repulsion_noalloc(x, 0.5, F_out=torch.empty((1000, 2)))   # host tensor
    # the C entry point itself refuses host memory for x or F_out
    import ctypes
    host = np.zeros((1000, 2), dtype=np.float32)
    lib = mm.load()
    F = torch.empty_like(x)
    st = lib.mm_repulsion_noalloc(1000, ctypes.c_void_p(host.ctypes.data), ctypes.c_float(0.5),
                                  ctypes.c_void_p(F.data_ptr()), None)
    assert st == 1
    st = lib.mm_repulsion_noalloc(1000, ctypes.c_void_p(x.data_ptr()), ctypes.c_float(0.5),
                                  ctypes.c_void_p(host.ctypes.data), None)
    assert st == 1
    # and a valid call still works after the refusals
    ok = mm.repulsion_noalloc(x, 0.5)
    assert torch.isfinite(ok).all()
