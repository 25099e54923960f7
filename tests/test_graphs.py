"""The seeded synthetic inputs match the recipes the workloads state (host
only): valid symmetric CSR, connectivity, sizes and degrees."""
import numpy as np
import pytest

from paper_1506_04383_gb300 import graphs

csg = pytest.importorskip("scipy.sparse.csgraph")
sps = pytest.importorskip("scipy.sparse")


def _valid(rp, col):
    n = len(rp) - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(col)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(src != col)                         # no self-loops
    for u in range(0, n, max(1, n // 97)):
        assert np.all(np.diff(col[rp[u]:rp[u + 1]]) > 0)   # sorted, no duplicates
    A = sps.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    assert (A != A.T).nnz == 0                         # symmetric
    return A


def test_rgg_mean_degree_and_connectivity():
    rp, col, pts, r = graphs.rgg(20000, 8.0, 1506)
    A = _valid(rp, col)
    n = len(rp) - 1
    assert csg.connected_components(A, directed=False)[0] == 1
    assert 0.95 * 20000 < n <= 20000                   # largest component
    # the radius is tuned so that the whole point set has mean degree 8 +- 0.05
    full_rp, full_col, _, _ = graphs.rgg(20000, 8.0, 1506, lcc=False)
    assert abs(len(full_col) / 20000 - 8.0) <= 0.05
    # every edge joins points closer than r
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(np.sqrt(((pts[src] - pts[col]) ** 2).sum(1)) < r)


def test_delaunay_is_a_planar_triangulation():
    rp, col, pts = graphs.delaunay(4096, 7)
    A = _valid(rp, col)
    n, m = 4096, len(col) // 2
    assert csg.connected_components(A, directed=False)[0] == 1
    # a triangulation of n points with h on the hull has 3n - 3 - h edges
    from scipy.spatial import ConvexHull
    h = len(ConvexHull(pts).vertices)
    assert m == 3 * n - 3 - h


def test_rmat_scale_and_skew():
    rp, col = graphs.rmat(14, 8, 3)
    A = _valid(rp, col)
    n = len(rp) - 1
    assert csg.connected_components(A, directed=False)[0] == 1
    assert n <= 1 << 14
    deg = np.diff(rp)
    # power-law skew: the largest degree is far above the mean
    assert deg.max() > 20 * deg.mean()


def test_grid_cycle_path_tree_shapes():
    rp, col = graphs.grid(32, 32)
    _valid(rp, col)
    assert len(col) // 2 == 1984 and len(rp) - 1 == 1024
    rp, col = graphs.cycle(10)
    assert np.all(np.diff(rp) == 2)
    rp, col = graphs.path(10)
    assert len(col) // 2 == 9
    rp, col = graphs.binary_tree(1023)
    _valid(rp, col)
    assert len(col) // 2 == 1022
    rp, col = graphs.random_tree(500, 4)
    A = _valid(rp, col)
    assert len(col) // 2 == 499 and csg.connected_components(A, directed=False)[0] == 1


def test_batch_sizes_and_graphs():
    sizes = graphs.batch_sizes(512, 1506)
    assert len(sizes) == 512 and min(sizes) >= 200 and max(sizes) <= 50000
    assert 2000 < np.median(sizes) < 4500            # lognormal, median 3000
    gs = [graphs.batch_graph(i, s, 1506) for i, s in enumerate(sizes[:6])]
    rp, col, gp = graphs.concat_graphs(gs)
    _valid(rp, col)
    assert gp[0] == 0 and gp[-1] == len(rp) - 1 and len(gp) == 7
    # block diagonal: no edge leaves its graph
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    gid = np.searchsorted(gp, np.arange(len(rp) - 1), side="right") - 1
    assert np.all(gid[src] == gid[col])


def test_generators_are_seeded():
    a = graphs.rgg(3000, 8.0, 5)
    b = graphs.rgg(3000, 8.0, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(graphs.uniform_positions(10, 3), graphs.uniform_positions(10, 3))
