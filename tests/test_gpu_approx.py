"""Parity of the hierarchy approximation of Eq. 3 (MulMent_h, Sec. 3.2)
between the CUDA library (through its C-ABI) and the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1506_04383_gb300 import graphs

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def inv_dist_sum(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(len(x))
    for i in range(0, len(x), 512):
        d = np.sqrt(((x[i:i + 512, None, :] - x[None, :, :]) ** 2).sum(-1))
        with np.errstate(divide="ignore"):
            out[i:i + 512] = np.where(d > 0, 1.0 / d, 0.0).sum(1)
    return out


def composed_map(mm, h, level, hh):
    """The map of `level` to min(level + hh, coarsest), from the exported
    per-level maps."""
    top = h.levels() - 1
    t = min(level + hh, top)
    m = np.arange(h.level_info(level)[0])
    for j in range(level, t):
        m = mm.level_export(h, j)["map"].cpu().numpy()[m]
    return m.astype(np.int32)


@pytest.mark.parametrize("hh", [1, 2, 4])
def test_repulsion_h_matches_oracle(mm, hh):
    rp, col, pts, _ = graphs.rgg(3000, 8.0, 61)
    p = mm.default_params(k=2, coarsest_n=100, approx_levels=hh)
    h = mm.build_hierarchy(cu(rp), cu(col), p)
    L = h.levels()
    assert L >= 4
    for level in (0, 1, L - 2, L - 1):
        n = h.level_info(level)[0]
        x = f32(graphs.uniform_positions(n, 70 + level, 0.0, math.sqrt(n)))
        F = mm.repulsion_h(h, level, cu(x)).cpu().numpy().astype(np.float64)
        cmap = composed_map(mm, h, level, hh)
        if level == L - 1:
            assert np.array_equal(cmap, np.arange(n))
        Fo = oracle.repulsion_h(x.astype(np.float64), cmap)
        tol = 2e-4 * inv_dist_sum(x)[:, None]
        assert np.all(np.abs(F - Fo) <= tol), (level, np.abs(F - Fo).max())


def test_repulsion_h_needs_an_approximating_hierarchy(mm):
    rp, col, _, _ = graphs.rgg(500, 8.0, 62)
    h = mm.build_hierarchy(cu(rp), cu(col), mm.default_params(k=1, coarsest_n=50))
    x = cu(f32(graphs.uniform_positions(h.level_info(0)[0], 1, 0.0, 20.0)))
    with pytest.raises(mm.MMError):
        mm.repulsion_h(h, 0, x)


def test_sweep_h_matches_oracle(mm):
    rp, col, pts, _ = graphs.rgg(3000, 8.0, 63)
    n = len(rp) - 1
    p = mm.default_params(k=2, coarsest_n=100, approx_levels=3)
    h = mm.build_hierarchy(cu(rp), cu(col), p)
    x = f32(pts * math.sqrt(n))
    xg, st = mm.sweep(h, 0, 0.3, cu(x))
    S = oracle.build_S(rp, col, 2)
    cmap = composed_map(mm, h, 0, 3)
    xo, sto = oracle.sweep(x.astype(np.float64), S, 0.3, 2, cmap=cmap)
    diam = float(np.ptp(xo, axis=0).max())
    assert np.abs(xg.cpu().numpy() - xo).max() <= 1e-4 * diam
    np.testing.assert_allclose(st, sto, rtol=1e-4)


def oracle_levels_to_device(levels):
    out = []
    for L in levels:
        d = dict(row_ptr=cu(L["rp"]), col=cu(L["col"]), omega=cu(f32(L["ew"])),
                 c=cu(f32(L["c"])))
        if L["map"] is not None:
            d["map"] = cu(L["map"])
        out.append(d)
    return out


@pytest.mark.parametrize("hh", [1, 3])
def test_layout_h_same_hierarchy_matches_oracle_objective(mm, hh):
    # the oracle's coarsening fed to the GPU (same levels, seed and maps):
    # MulMent_h layouts of both must end within 1% of each other's
    # objective (Eq. 1 at alpha = 0.008)
    rp, col, _, _ = graphs.rgg(3000, 8.0, 36)
    kw = dict(k=2, coarsest_n=100, approx_levels=hh)
    po = oracle.params(**kw)
    levels = oracle.build_hierarchy(rp, col, po)
    xo, info = oracle.layout(rp, col, po, levels=levels)
    h = mm.build_hierarchy_levels(oracle_levels_to_device(levels), mm.default_params(**kw))
    x, st = mm.layout(h)
    xs = x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(xs))
    S = levels[0]["S"]
    Mg = oracle.objective(xs, S, 0.008)[2]
    Mo = oracle.objective(xo, S, 0.008)[2]
    assert abs(Mg - Mo) <= 0.01 * abs(Mo), (Mg, Mo)


def test_layout_h_and_barnes_hut_reach_comparable_objectives(mm):
    # Sec. 4: MulMent_h trades quality for time; on a 3000-vertex RGG the
    # h = 1 layout's objective stays within 5% of the Barnes-Hut layout's
    rp, col, _, _ = graphs.rgg(3000, 8.0, 64)
    out = {}
    for hh in (0, 1):
        p = mm.default_params(k=2, coarsest_n=100, approx_levels=hh)
        h = mm.build_hierarchy(cu(rp), cu(col), p)
        x, st = mm.layout(h, p)
        out[hh] = mm.objective(h, 0, x, 0.008)[2]
    assert abs(out[1] - out[0]) <= 0.05 * abs(out[0]), out


@pytest.mark.parametrize("hh", [0, 3])
def test_dynamic_update_matches_oracle(mm, hh):
    # Sec. 4.3, update algorithm: the perturbed graph Q is laid out from a
    # layout of the original G, starting at alpha = 0.008 on the finest level
    # of Q's hierarchy cut after h levels (h = 0: the exact sum).  Same
    # hierarchy and start on both sides; objectives within 1%.
    rp, col, _, _ = graphs.rgg(2000, 8.0, 65)
    xG, _ = oracle.layout(rp, col, oracle.params(k=1, coarsest_n=20))
    qrp, qcol = graphs.perturb_edges(rp, col, 5.0, 16, 4)
    ku = dict(k=1, coarsest_n=2, alpha0=0.008, max_levels=hh + 1, approx_levels=hh,
              exact_repulsion=1 if hh == 0 else 0)
    po = oracle.params(**ku)
    levels = oracle.build_hierarchy(qrp, qcol, po)
    assert len(levels) == hh + 1
    xo, _ = oracle.layout(qrp, qcol, po, x_init=xG, levels=levels)
    p = mm.default_params(**ku)
    h = mm.build_hierarchy_levels(oracle_levels_to_device(levels), p)
    x, st = mm.layout(h, p, x_init=cu(f32(xG)))
    assert st["num_levels"] == hh + 1
    xs = x.cpu().numpy().astype(np.float64)
    S = levels[0]["S"]
    Mg = oracle.objective(xs, S, 0.008)[2]
    Mo = oracle.objective(xo, S, 0.008)[2]
    assert abs(Mg - Mo) <= 0.01 * abs(Mo), (Mg, Mo)
    # the update starts from a good layout: far better than a random start
    M0 = oracle.objective(graphs.uniform_positions(len(xs), 2, 0, 40), S, 0.008)[2]
    assert Mg < M0


# ------------------------------------------------ full stress (Sec. 4) ---
@pytest.mark.parametrize("case", ["rgg", "grid", "path"])
def test_full_stress_matches_oracle(mm, case):
    # all-pairs hop distances by 64-source breadth-first searches on the
    # device against the oracle's one-source-at-a-time searches; sizes span
    # several 64-source batches and a ragged last batch
    if case == "rgg":
        rp, col, pts, _ = graphs.rgg(2500, 8.0, 66)
        n = len(rp) - 1
        x = pts * math.sqrt(n)
    elif case == "grid":
        rp, col = graphs.grid(37, 29)
        n = len(rp) - 1
        x = graphs.uniform_positions(n, 3, 0.0, 30.0)
    else:
        rp, col = graphs.path(130)
        n = 130
        x = np.stack([np.arange(130.0), np.zeros(130)], 1)
    h = mm.build_hierarchy(cu(rp), cu(col), mm.default_params(k=1, coarsest_n=n))
    xf = f32(x)
    F, s, Fs, pairs = mm.full_stress(h, cu(xf))
    Fo, so, Fso, po = oracle.full_stress(rp, col, xf.astype(np.float64))
    assert pairs == po == n * (n - 1) // 2
    assert F == pytest.approx(Fo, rel=1e-4, abs=1e-3)
    assert s == pytest.approx(so, rel=1e-4)
    assert Fs == pytest.approx(Fso, rel=1e-4, abs=1e-3)


def test_full_stress_refuses_weighted_and_large_graphs(mm):
    rp, col = graphs.path(10)
    el = np.full(len(col), 2.0, dtype=np.float32)
    h = mm.build_hierarchy(cu(rp), cu(col), mm.default_params(k=1, coarsest_n=10), edge_len=cu(el))
    with pytest.raises(mm.MMError):
        mm.full_stress(h, cu(f32(np.zeros((10, 2)))))


def test_approx_levels_refused_for_batches(mm):
    gs = [graphs.grid(10, 10), graphs.grid(8, 12)]
    rp, col, gp = graphs.concat_graphs(gs)
    p = mm.default_params(k=2, coarsest_n=2, approx_levels=2)
    with pytest.raises(mm.MMError):
        mm.build_hierarchy(cu(rp), cu(col), p, graph_ptr=gp)
