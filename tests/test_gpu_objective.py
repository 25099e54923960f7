"""Oracle-matched maxent-stress at the benchmark's scale.

The final objective M (Eq. 1 at alpha = 0.008, Sec. 4) of the GPU's
multilevel layout on the oracle's own hierarchy (the oracle's coarsening fed
to the device, same seed, so the prolongation draws and the schedule are
the same) must be within 1 % of the FP64 oracle's layout on that hierarchy:

* the 100k random geometric graph (k = 2, theta = 0.5): both layouts are
  computed here and M is evaluated exactly over all pairs by the oracle;
* the Delaunay triangulation of 2^20 points (k = 1, theta = 0.6): the
  oracle's layout takes minutes of CPU time, so its M is read from
  tests/golden/oracle_layouts.json (written by make_oracle_layouts.py, which
  calls only the oracle); both sides use the oracle's estimator (exact stress
  over S, the ln-sum outside S from the same 2e7 random pairs).

At 2^20 vertices the GPU's exact O(n^2) objective (mm_objective) is also
checked against the oracle's sampled estimate of the same layout: within 5
standard errors.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1506_04383_gb300 import graphs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_layouts.json")


def _to_device(levels):
    out = []
    for L in levels:
        d = dict(row_ptr=torch.from_numpy(L["rp"]).cuda(), col=torch.from_numpy(L["col"]).cuda(),
                 omega=torch.from_numpy(L["ew"].astype(np.float32)).cuda(),
                 c=torch.from_numpy(L["c"].astype(np.float32)).cuda())
        if L["map"] is not None:
            d["map"] = torch.from_numpy(L["map"]).cuda()
        out.append(d)
    return out


def test_rgg100k_same_hierarchy_objective_within_1pct_of_oracle(mm):
    rp, col, _, _ = graphs.rgg(100000, 8.0, 1506)
    kw = dict(k=2, theta=0.5, coarsest_n=100)
    po = oracle.params(**kw)
    levels = oracle.build_hierarchy(rp, col, po)
    xo, info = oracle.layout(rp, col, po, levels=levels)
    h = mm.build_hierarchy_levels(_to_device(levels), mm.default_params(**kw))
    x, st = mm.layout(h)
    xs = x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(xs))
    S = levels[0]["S"]
    sg, lg, Mg = oracle.objective(xs, S, 0.008)
    so, lo, Mo = oracle.objective(xo, S, 0.008)
    assert abs(Mg - Mo) <= 0.01 * abs(Mo), (Mg, Mo)
    # the entropy term dominates M; the stress term is held to 5 %
    assert abs(sg - so) <= 0.05 * so, (sg, so)
    # the device's own exact objective of its layout agrees with the oracle's
    _, _, Mgpu = mm.objective(h, 0, x, 0.008)
    assert Mgpu == pytest.approx(Mg, rel=1e-5)


def test_del20_same_hierarchy_objective_within_1pct_of_stored_oracle_layout(mm):
    with open(GOLDEN) as fh:
        g = json.load(fh)["del20"]
    rp, col, _ = graphs.delaunay(1 << 20, 1506)
    assert len(rp) - 1 == g["n"] and len(col) // 2 == g["m"]
    po = oracle.params(**g["params"])
    levels = oracle.build_hierarchy(rp, col, po)
    assert [int(L["n"]) for L in levels] == g["level_n"]
    h = mm.build_hierarchy_levels(_to_device(levels), mm.default_params(**g["params"]))
    x, st = mm.layout(h)
    xs = x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(xs))
    S = levels[0]["S"]
    est = oracle.objective_sampled(xs, S, 0.008, samples=g["samples"], seed=g["sample_seed"])
    assert abs(est["M"] - g["M"]) <= 0.01 * abs(g["M"]), (est["M"], g["M"])
    # exact M over all 5.5e11 pairs on the device vs the sampled estimate
    _, _, Mgpu = mm.objective(h, 0, x, 0.008)
    assert abs(Mgpu - est["M"]) <= 5 * est["se_M"], (Mgpu, est["M"], est["se_M"])


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.7])
def test_barnes_hut_objective_against_the_oracle(mm, theta):
    # mm_objective_bh: log potentials from the quadtree walk (accepted cells
    # count x ln of the centroid distance) instead of the O(n^2) pass.  theta = 0
    # opens every cell: the exact sum, to FP32 rounding (relative 1e-5 of M).
    # theta > 0: about its centroid a cell's first-order term vanishes, and the
    # second-order remainder of ln|1 - z| is at most |z|^2 / (2 (1 - |z|)) per
    # point, |z| = (distance of a point from the centroid) / (distance of the
    # centroid) <= sqrt(2) w / D < sqrt(2) theta for an accepted cell of side
    # w (point and centroid both in the cell); so, for sqrt(2) theta < 1,
    # |lnsum_bh - lnsum| <= pairs x that bound.
    rp, col, _, _ = graphs.rgg(5000, 8.0, 44)
    n = len(rp) - 1
    h = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(),
                           mm.default_params(k=2, coarsest_n=100))
    x, _ = mm.layout(h)
    xs = x.cpu().numpy().astype(np.float64)
    S = oracle.build_S(rp, col, 2)
    so, lo, Mo = oracle.objective(xs, S, 0.008)
    sb, lb, Mb = mm.objective_bh(h, 0, x, 0.008, theta)
    assert sb == pytest.approx(so, rel=1e-6)
    if theta == 0.0:
        assert Mb == pytest.approx(Mo, rel=1e-5)
        assert lb == pytest.approx(lo, rel=1e-5)
    else:
        z = theta * np.sqrt(2.0)
        if z < 1.0:
            bound = n * (n - 1) / 2 * z * z / (2 * (1 - z))
            assert abs(lb - lo) <= bound
        # in practice far inside that bound: a few parts in 10^4 of the sum
        assert abs(lb - lo) <= 1e-3 * abs(lo), (lb, lo)
