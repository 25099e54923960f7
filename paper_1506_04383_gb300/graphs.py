"""Seeded synthetic graph and position generators.

This module serves both the CUDA path and the FP64 oracle, so it holds none
of the layout method's arithmetic: it only builds graphs (symmetric CSR with
sorted rows, no self-loops, no duplicates) and seeded initial coordinates.

The generators stand in for the paper's instance families (Table of basic
properties, appendix): meshes and Delaunay triangulations of random points
(del16/del20), road-like sparse graphs (random geometric graphs), power-law
graphs (R-MAT), trees (btree) and grids.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def csr_from_edges(n: int, u, v):
    """Undirected edge list -> symmetric CSR (int64 row_ptr, int32 col).

    Drops self-loops and duplicates; rows are sorted ascending."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = np.unique(a * n + b)
    a = key // n
    b = key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, a + 1, 1)
    rp = np.cumsum(rp)
    return rp, b.astype(np.int32)


def components(rp, col):
    """Connected component label per vertex (iterative BFS, host side)."""
    n = len(rp) - 1
    comp = -np.ones(n, dtype=np.int64)
    c = 0
    for s in range(n):
        if comp[s] >= 0:
            continue
        comp[s] = c
        frontier = np.array([s])
        while len(frontier):
            nb = np.concatenate([col[rp[i]:rp[i + 1]] for i in frontier]) if len(frontier) < 64 \
                else col[np.concatenate([np.arange(rp[i], rp[i + 1]) for i in frontier])]
            nb = np.unique(nb)
            nb = nb[comp[nb] < 0]
            comp[nb] = c
            frontier = nb
        c += 1
    return comp


def largest_component(rp, col):
    """Restrict a CSR graph to its largest connected component (the paper
    draws the largest component of every instance, Sec. 4)."""
    try:
        import scipy.sparse as sps
        import scipy.sparse.csgraph as csg
        n = len(rp) - 1
        A = sps.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
        _, comp = csg.connected_components(A, directed=False)
    except Exception:  # pragma: no cover - scipy missing
        comp = components(rp, col)
    counts = np.bincount(comp)
    big = int(np.argmax(counts))
    keep = np.nonzero(comp == big)[0]
    if len(keep) == len(rp) - 1:
        return rp, col, keep
    newid = -np.ones(len(rp) - 1, dtype=np.int64)
    newid[keep] = np.arange(len(keep))
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    m = (newid[src] >= 0) & (newid[col] >= 0)
    rp2, col2 = csr_from_edges(len(keep), newid[src[m]], newid[col[m]])
    return rp2, col2, keep


def grid(nx: int, ny: int):
    """nx x ny grid graph with unit edges."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return csr_from_edges(nx * ny, u, v)


def cycle(n: int):
    i = np.arange(n)
    return csr_from_edges(n, i, (i + 1) % n)


def path(n: int):
    i = np.arange(n - 1)
    return csr_from_edges(n, i, i + 1)


def complete(n: int):
    u, v = np.triu_indices(n, 1)
    return csr_from_edges(n, u, v)


def binary_tree(n: int):
    """Complete binary tree on n vertices (btree of the instance table)."""
    v = np.arange(1, n)
    return csr_from_edges(n, (v - 1) // 2, v)


def random_tree(n: int, seed: int):
    """Uniform random labelled tree from a random Pruefer sequence."""
    rng = _rng(seed)
    if n <= 1:
        return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    if n == 2:
        return csr_from_edges(2, [0], [1])
    seq = rng.integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    np.add.at(degree, seq, 1)
    import heapq
    leaves = [i for i in range(n) if degree[i] == 1]
    heapq.heapify(leaves)
    us, vs = [], []
    for s in seq:
        leaf = heapq.heappop(leaves)
        us.append(leaf)
        vs.append(int(s))
        degree[s] -= 1
        if degree[s] == 1:
            heapq.heappush(leaves, int(s))
    a = heapq.heappop(leaves)
    b = heapq.heappop(leaves)
    us.append(a)
    vs.append(b)
    return csr_from_edges(n, us, vs)


def _pairs_within(pts, r):
    from scipy.spatial import cKDTree
    tree = cKDTree(pts)
    pairs = tree.query_pairs(r, output_type="ndarray")
    return pairs[:, 0], pairs[:, 1]


def rgg(n: int, mean_degree: float, seed: int, tune: bool = True, lcc: bool = True):
    """Random geometric graph: n points uniform in the unit square, edges
    between points closer than r.  r starts at sqrt(deg / (pi n)) and is
    bisected until the realised mean degree is within 0.05 of the target
    (boundary effects lower it).  Returns (rp, col, points, r)."""
    rng = _rng(seed)
    pts = rng.random((n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    u, v = _pairs_within(pts, r)
    if tune:
        lo, hi = r, r * 1.2
        for _ in range(40):
            deg = 2.0 * len(u) / n
            if abs(deg - mean_degree) <= 0.05:
                break
            if deg < mean_degree:
                lo = r
            else:
                hi = r
            r = 0.5 * (lo + hi) if deg > mean_degree or hi > lo * 1.0001 else r * 1.01
            u, v = _pairs_within(pts, r)
    rp, col = csr_from_edges(n, u, v)
    if lcc:
        rp, col, keep = largest_component(rp, col)
        pts = pts[keep]
    return rp, col, pts, r


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19):
    """R-MAT generator (recursive quadrant choice per edge sample, no noise).
    Self-loops and duplicates dropped, symmetrised, vertex ids randomly
    permuted, largest component kept."""
    rng = _rng(seed)
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale):
        r = rng.random(m)
        ubit = (r >= ab).astype(np.int64)
        vbit = (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64)
        u |= ubit << bit
        v |= vbit << bit
    perm = rng.permutation(n)
    rp, col = csr_from_edges(n, perm[u], perm[v])
    rp, col, _ = largest_component(rp, col)
    return rp, col


def delaunay(n: int, seed: int):
    """Delaunay triangulation of n uniform random points in the unit square
    (the del-X family of the instance table).  Returns (rp, col, points)."""
    from scipy.spatial import Delaunay
    rng = _rng(seed)
    pts = rng.random((n, 2))
    tri = Delaunay(pts)
    s = tri.simplices
    u = np.concatenate([s[:, 0], s[:, 1], s[:, 2]])
    v = np.concatenate([s[:, 1], s[:, 2], s[:, 0]])
    rp, col = csr_from_edges(n, u, v)
    return rp, col, pts


def uniform_positions(n: int, seed: int, lo: float = 0.0, hi: float = 1.0):
    """n points uniform in [lo, hi]^2 (float64), seeded."""
    return lo + (hi - lo) * _rng(seed).random((n, 2))


def batch_sizes(count: int, seed: int, median: float = 3000.0, sigma: float = 1.0,
                lo: int = 200, hi: int = 50000):
    """Lognormal graph sizes (median, sigma), resampled into [lo, hi]."""
    rng = _rng(seed)
    out = []
    while len(out) < count:
        s = int(round(math.exp(math.log(median) + sigma * rng.standard_normal())))
        if lo <= s <= hi:
            out.append(s)
    return out


def batch_graph(i: int, size: int, base_seed: int):
    """Graph i of the mixed batch: thirds of near-square grids, RGGs with
    mean degree 6..12, and uniform random trees."""
    seed = base_seed + i
    kind = i % 3
    if kind == 0:
        nx = max(2, int(round(math.sqrt(size))))
        ny = max(2, int(round(size / nx)))
        rp, col = grid(nx, ny)
    elif kind == 1:
        deg = 6 + (seed % 7)
        rp, col, _, _ = rgg(size, float(deg), seed, tune=False)
    else:
        rp, col = random_tree(size, seed)
    return rp, col


def concat_graphs(graphs):
    """Block-diagonal union of CSR graphs; returns (rp, col, graph_ptr)."""
    rps, cols, gp = [], [], [0]
    off_v, off_e = 0, 0
    for rp, col in graphs:
        n = len(rp) - 1
        rps.append(rp[:-1] + off_e)
        cols.append(col.astype(np.int64) + off_v)
        off_v += n
        off_e += int(rp[-1])
        gp.append(off_v)
    rps.append(np.array([off_e]))
    return (np.concatenate(rps).astype(np.int64), np.concatenate(cols).astype(np.int32),
            np.array(gp, dtype=np.int32))


def _within(rp, col, a: int, D: int, seen):
    """Vertices at hop distance 2..D from a (level-synchronous BFS; `seen`
    is a boolean scratch array of n entries, left all False)."""
    frontier = np.array([a], dtype=np.int64)
    seen[a] = True
    touched = [frontier]
    out = []
    for d in range(1, D + 1):
        if len(frontier) == 0:
            break
        deg = rp[frontier + 1] - rp[frontier]
        tot = int(deg.sum())
        if tot == 0:
            break
        starts = np.repeat(rp[frontier] - np.concatenate([[0], np.cumsum(deg)[:-1]]), deg)
        nb = np.unique(col[starts + np.arange(tot)].astype(np.int64))
        nb = nb[~seen[nb]]
        seen[nb] = True
        touched.append(nb)
        if d >= 2:
            out.append(nb)
        frontier = nb
    for t in touched:
        seen[t] = False
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def perturb_edges(rp, col, pct: float, D: int, seed: int):
    """The dynamic-graph model of the paper's experiments (Sec. 4.3): a BFS
    spanning tree from a random vertex is kept, pct % of the undirected edges
    that are not in it are removed at random (the graph stays connected), and
    as many new edges are inserted, each between a random vertex and a random
    vertex at distance 1 < d <= D in the original graph.  Returns the
    perturbed CSR (same vertex ids)."""
    import scipy.sparse as sps
    import scipy.sparse.csgraph as csg
    rng = _rng(seed)
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    und = src < col
    eu, ev = src[und].astype(np.int64), col[und].astype(np.int64)
    m = len(eu)
    A = sps.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    start = int(rng.integers(n))
    T = csg.breadth_first_tree(A, start, directed=False).tocoo()
    tree = set(zip(np.minimum(T.row, T.col).tolist(), np.maximum(T.row, T.col).tolist()))
    tkey = np.array(sorted(a * n + b for a, b in tree), dtype=np.int64)
    non_tree = np.nonzero(~np.isin(eu * n + ev, tkey))[0]
    k = int(round(pct / 100.0 * m))
    k = min(k, len(non_tree))
    drop = rng.choice(non_tree, size=k, replace=False) if k else np.zeros(0, dtype=np.int64)
    keep = np.ones(m, dtype=bool)
    keep[drop] = False
    edges = set(zip(eu[keep].tolist(), ev[keep].tolist()))
    added = 0
    seen = np.zeros(n, dtype=bool)
    while added < k:
        a = int(rng.integers(n))
        cand = _within(rp, col, a, D, seen)
        if len(cand) == 0:
            continue
        b = int(cand[int(rng.integers(len(cand)))])
        e = (min(a, b), max(a, b))
        if e in edges:
            continue
        edges.add(e)
        added += 1
    u = np.array([e[0] for e in edges], dtype=np.int64)
    v = np.array([e[1] for e in edges], dtype=np.int64)
    return csr_from_edges(n, u, v)
