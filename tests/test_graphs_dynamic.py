"""The dynamic-graph model of the paper's update experiments (Sec. 4.3):
checks of the seeded edge-perturbation generator (host only)."""
import numpy as np
import pytest

from paper_1506_04383_gb300 import graphs

sps = pytest.importorskip("scipy.sparse")
csg = pytest.importorskip("scipy.sparse.csgraph")


def _edges(rp, col):
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    m = src < col
    return set(zip(src[m].tolist(), col[m].tolist()))


@pytest.mark.parametrize("pct,D", [(1.0, 2), (5.0, 16)])
def test_perturb_edges_model(pct, D):
    rp, col, _, _ = graphs.rgg(2000, 8.0, 11)
    n = len(rp) - 1
    qrp, qcol = graphs.perturb_edges(rp, col, pct, D, 3)
    # a valid symmetric CSR with sorted rows, no loops, same vertex count
    assert len(qrp) == n + 1 and np.all(np.diff(qrp) >= 0)
    src = np.repeat(np.arange(n), np.diff(qrp))
    assert np.all(src != qcol)
    for u in range(0, n, 97):
        row = qcol[qrp[u]:qrp[u + 1]]
        assert np.all(np.diff(row) > 0)
    A = sps.csr_matrix((np.ones(len(qcol)), qcol, qrp), shape=(n, n))
    assert (A != A.T).nnz == 0
    # connected (a spanning tree of the original graph is kept)
    assert csg.connected_components(A, directed=False)[0] == 1
    G, Q = _edges(rp, col), _edges(qrp, qcol)
    removed, inserted = G - Q, Q - G
    k = int(round(pct / 100.0 * len(G)))
    assert len(removed) == k and len(inserted) == k and len(Q) == len(G)
    # inserted edges join vertices at distance 1 < d <= D in the original
    AG = sps.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    ins = np.array(sorted(inserted))
    d = csg.shortest_path(AG, unweighted=True, indices=ins[:, 0])
    dd = d[np.arange(len(ins)), ins[:, 1]]
    assert np.all((dd > 1) & (dd <= D))


def test_perturb_edges_is_seeded():
    rp, col = graphs.grid(20, 20)
    a = graphs.perturb_edges(rp, col, 5.0, 4, 9)
    b = graphs.perturb_edges(rp, col, 5.0, 4, 9)
    c = graphs.perturb_edges(rp, col, 5.0, 4, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))
