"""Batched layout: many graphs of uneven sizes laid out together.

Every graph of a batch must get exactly the layout the single-graph path
gives it with the same seed (graph i of the batch uses seed + i): the batch
runs the same kernels on the same per-graph hierarchies, only grouped into
shared launches (a CTA per small graph-level, a WHILE loop per larger level
in parallel graph branches).
"""
import numpy as np
import pytest
import torch

from paper_1506_04383_gb300 import graphs

pytestmark = pytest.mark.gpu


def _batch(sizes, base_seed):
    gs = [graphs.batch_graph(i, s, base_seed) for i, s in enumerate(sizes)]
    return gs, graphs.concat_graphs(gs)


def test_batch_equals_single_graph_layouts(mm):
    sizes = [300, 2500, 700, 5000, 200, 1200, 2048, 2049, 900]
    gs, (rp, col, gp) = _batch(sizes, 77)
    kw = dict(k=2, theta=0.5, coarsest_n=2, seed=1506)
    p = mm.default_params(**kw)
    hb = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p,
                            graph_ptr=gp)
    xb, st = mm.layout(hb, p)
    xb = xb.cpu().numpy()
    assert np.all(np.isfinite(xb))
    vu = 0
    for i, (grp, gcol) in enumerate(gs):
        pi = mm.default_params(**dict(kw, seed=1506 + i))
        h = mm.build_hierarchy(torch.from_numpy(grp).cuda(), torch.from_numpy(gcol).cuda(), pi)
        x, sti = mm.layout(h, pi)
        vu += sti["vertex_updates"]
        np.testing.assert_array_equal(xb[gp[i]:gp[i + 1]], x.cpu().numpy())
    assert st["vertex_updates"] == vu


def test_batch_reports_bad_graph_ptr(mm):
    rp, col = graphs.grid(4, 4)
    p = mm.default_params()
    with pytest.raises(mm.MMError):
        mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p,
                           graph_ptr=np.array([0, 10, 8, 16], dtype=np.int32))
    # an edge crossing two graphs of the batch
    with pytest.raises(mm.MMError):
        mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p,
                           graph_ptr=np.array([0, 6, 16], dtype=np.int32))


def test_autotune_keeps_objective(mm):
    rp, col, _, _ = graphs.rgg(20000, 8.0, 5)
    p = mm.default_params(k=2, theta=0.5, coarsest_n=100)
    h = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p)
    r = mm.autotune(h, thetas=[0.5, 0.6, 0.7], max_rel_drift=0.01)
    assert r["theta"] in (0.5, np.float32(0.6), np.float32(0.7))
    assert abs(r["objective"] - r["objective_ref"]) <= 0.01 * abs(r["objective_ref"]) + 1e-9
    for lanes, warps in zip(r["gather_lanes"], r["traverse_warps"]):
        # the tuner times 1, 2, 4, 8 and 16 warps per walk task
        assert lanes in (0, 1, 2, 4, 8, 16, 32) and warps in (0, 1, 2, 4, 8, 16)
    x, st = mm.layout(h)
    assert np.all(np.isfinite(x.cpu().numpy()))


def _oracle_levels_from_device(mm, h, k):
    """The device hierarchy's levels (exported) in the oracle's format: the
    oracle then lays out the graph on exactly these levels."""
    import oracle
    levels = []
    for l in range(h.levels()):
        e = mm.level_export(h, l)
        n = e["c"].numel()
        L = dict(n=n, rp=e["row_ptr"].cpu().numpy().astype(np.int64),
                 col=e["col"].cpu().numpy().astype(np.int32),
                 ew=e["omega"].cpu().numpy().astype(np.float64),
                 c=e["c"].cpu().numpy().astype(np.float64), elen=None, coarse=l > 0,
                 map=e["map"].cpu().numpy().astype(np.int32) if l < h.levels() - 1 else None)
        L["S"] = oracle.build_S(L["rp"], L["col"], k, c=L["c"], coarse=L["coarse"])
        levels.append(L)
    return levels


def test_batched_layouts_match_oracle_on_the_same_hierarchies(mm):
    # a few graphs of one batch: each graph's part of the batched layout
    # against the FP64 oracle's layout of that graph on the same levels (the
    # device's per-graph hierarchy, exported; graph i uses seed + i); final
    # objective (Eq. 1 at alpha = 0.008) within 1 %
    import oracle
    sizes = [1500, 400, 3000, 800]
    gs, (rp, col, gp) = _batch(sizes, 91)
    kw = dict(k=2, theta=0.5, coarsest_n=2, seed=1506)
    p = mm.default_params(**kw)
    hb = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p,
                            graph_ptr=gp)
    xb, st = mm.layout(hb, p)
    xb = xb.cpu().numpy().astype(np.float64)
    for i, (grp, gcol) in enumerate(gs):
        pi = mm.default_params(**dict(kw, seed=1506 + i))
        h = mm.build_hierarchy(torch.from_numpy(grp).cuda(), torch.from_numpy(gcol).cuda(), pi)
        levels = _oracle_levels_from_device(mm, h, kw["k"])
        po = oracle.params(**dict(kw, seed=1506 + i))
        xo, _ = oracle.layout(grp, gcol, po, levels=levels)
        S = levels[0]["S"]
        Mb = oracle.objective(xb[gp[i]:gp[i + 1]], S, 0.008)[2]
        Mo = oracle.objective(xo, S, 0.008)[2]
        assert abs(Mb - Mo) <= 0.01 * abs(Mo), (i, Mb, Mo)
