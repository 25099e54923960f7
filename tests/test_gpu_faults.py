"""Failure paths of the C-ABI, driven from the host without faulting the GPU.

* Non-finite coordinates: a caller's start layout holding NaN or Inf goes
  through the whole sweep (bounding square, Morton keys, sort, tree, walk,
  update: every index there comes from integer keys, which clamp NaN and Inf
  to a valid cell) and the update's reduction flags the non-finite result;
  mm_sweep and mm_layout return MM_ERR_NONFINITE.
* A bounded device wait that gives up: mm_selftest_wait_timeout launches the
  sort's look-back pass so that its wait can never be satisfied (the tile it
  waits for never runs); the wait stops after its poll limit and the call
  returns MM_ERR_TIMEOUT.
After each failure the same hierarchy and context must still lay out a
finite start correctly, so the tests also check that the context stays
usable.
"""
import math

import numpy as np
import pytest
import torch

from paper_1506_04383_gb300 import graphs

pytestmark = pytest.mark.gpu

MM_ERR_NONFINITE = 5
MM_ERR_TIMEOUT = 6


def _grid_hierarchy(mm, fused):
    rp, col = graphs.grid(12, 12)
    n = len(rp) - 1
    p = mm.default_params(k=2, theta=0.5, coarsest_n=n, fused_max_n=fused)
    h = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p)
    x = graphs.uniform_positions(n, 1506).astype(np.float32)
    return h, p, x


@pytest.mark.parametrize("fused", [0, -1], ids=["fused-level-kernel", "multi-kernel-sweep"])
@pytest.mark.parametrize("bad", [math.nan, math.inf, -math.inf], ids=["nan", "inf", "-inf"])
def test_sweep_of_nonfinite_start_returns_nonfinite(mm, fused, bad):
    h, p, x = _grid_hierarchy(mm, fused)
    good, _ = mm.sweep(h, 0, 0.3, torch.from_numpy(x).cuda())
    xb = x.copy()
    xb[7, 0] = bad
    with pytest.raises(mm.MMError) as e:
        mm.sweep(h, 0, 0.3, torch.from_numpy(xb).cuda())
    assert e.value.status == MM_ERR_NONFINITE
    # the hierarchy and the context stay usable: the finite start gives the
    # same sweep as before
    again, _ = mm.sweep(h, 0, 0.3, torch.from_numpy(x).cuda())
    assert torch.allclose(good, again, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("fused", [0, -1], ids=["fused-level-kernel", "multi-kernel-sweep"])
def test_layout_from_nonfinite_start_returns_nonfinite(mm, fused):
    h, p, x = _grid_hierarchy(mm, fused)
    p.max_iters_at_min = 10
    xb = x.copy()
    xb[3, 1] = math.nan
    with pytest.raises(mm.MMError) as e:
        mm.layout(h, p, x_init=torch.from_numpy(xb).cuda())
    assert e.value.status == MM_ERR_NONFINITE
    xo, st = mm.layout(h, p, x_init=torch.from_numpy(x).cuda())
    assert torch.isfinite(xo).all() and st["total_sweeps"] > 0


@pytest.mark.parametrize("limit", [1, 64, 4096])
def test_bounded_wait_gives_up_and_returns_timeout(mm, limit):
    assert mm.selftest_wait_timeout(limit) == MM_ERR_TIMEOUT
    # the context is still usable: a Barnes-Hut sweep through the
    # multi-kernel path (whose sort passes use the same look-back) succeeds
    h, p, x = _grid_hierarchy(mm, -1)
    xo, st = mm.sweep(h, 0, 0.3, torch.from_numpy(x).cuda())
    assert torch.isfinite(xo).all()


def test_wait_timeout_selftest_rejects_bad_limits(mm):
    from paper_1506_04383_gb300.mm import MM_OK
    assert mm.selftest_wait_timeout(0) == 1       # MM_ERR_INVALID_ARG
    assert mm.selftest_wait_timeout(1 << 23) == 1
    assert MM_OK == 0
