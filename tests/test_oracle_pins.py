"""Pins of the FP64 oracle against values the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a
published known-answer vector, a closed form derived from Eq. 1 / Eq. 2 on a
symmetric configuration, an exact invariant, or a hand-worked example.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1506_04383_gb300 import graphs
from golden_io import contract_example, philox_kat


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# --------------------------------------------------------------------------
def test_philox_known_answers():
    for ctr, key, expect in philox_kat():
        assert oracle.philox4x32_10(ctr, key).tolist() == expect


# --------------------------------------------------------------------------
# k-hop S (Sec. 2.3 footnote): hand-counted neighbourhoods
# --------------------------------------------------------------------------
def test_S_grid_32x32_counts():
    rp, col = graphs.grid(32, 32)
    assert int(rp[-1]) == 2 * 1984
    sp, scol, sd, rho = oracle.build_S(rp, col, 2)
    # 1984 edges + 1920 straight distance-2 pairs + 1922 diagonal pairs,
    # each stored in both directions
    assert len(scol) == 2 * (1984 + 1920 + 1922) == 11652
    assert np.all(sd[sd > 1] == 2.0)
    assert np.count_nonzero(sd == 2.0) == 2 * (1920 + 1922)
    # interior vertex: 4 neighbours (w=1) and 8 at distance 2 (w=1/4)
    u = 5 * 32 + 5
    assert sp[u + 1] - sp[u] == 12
    assert rho[u] == pytest.approx(4 + 8 / 4.0)


def test_S_path_and_coarse_lengths():
    rp, col = graphs.path(5)
    sp, scol, sd, rho = oracle.build_S(rp, col, 3)
    assert scol[sp[0]:sp[1]].tolist() == [1, 2, 3]
    assert sd[sp[0]:sp[1]].tolist() == [1.0, 2.0, 3.0]
    # coarse level: edge length sqrt(c_u) + sqrt(c_v) (Sec. 3.2)
    c = np.array([1.0, 4.0, 9.0, 16.0, 25.0])
    sp, scol, sd, rho = oracle.build_S(rp, col, 2, c=c, coarse=True)
    row0 = dict(zip(scol[sp[0]:sp[1]].tolist(), sd[sp[0]:sp[1]].tolist()))
    assert row0 == {1: 1 + 2, 2: (1 + 2) + (2 + 3)}
    row2 = dict(zip(scol[sp[2]:sp[3]].tolist(), sd[sp[2]:sp[3]].tolist()))
    assert row2 == {0: 8.0, 1: 5.0, 3: 7.0, 4: 7.0 + 9.0}


def test_S_shortest_path_prefers_cheaper_route():
    # square 0-1-2-3-0 plus chord 0-2; with k=2 the pair (1,3) is reached via
    # 0 or 2; the coarse lengths make one route cheaper
    rp, col = graphs.csr_from_edges(4, [0, 1, 2, 3, 0], [1, 2, 3, 0, 2])
    c = np.array([1.0, 1.0, 100.0, 1.0])
    sp, scol, sd, _ = oracle.build_S(rp, col, 2, c=c, coarse=True)
    row1 = dict(zip(scol[sp[1]:sp[2]].tolist(), sd[sp[1]:sp[2]].tolist()))
    assert row1[3] == pytest.approx(2.0 + 2.0)  # via vertex 0 (sqrt c = 1)
    assert row1[2] == pytest.approx(1.0 + 10.0)  # direct edge


# --------------------------------------------------------------------------
# Eq. 2 sweep: regular polygon closed form
#   one exact sweep maps a regular n-gon of radius R to a regular n-gon at the
#   same angles with radius
#   R' = [sum_{v in S} w_v (R cos phi_v + d_v |sin(phi_v/2)|)
#         + alpha (n - 1 - |S_u|) / (2R)] / rho
# --------------------------------------------------------------------------
def polygon(n, R, center=(0.0, 0.0)):
    ang = 2 * np.pi * np.arange(n) / n
    return np.stack([center[0] + R * np.cos(ang), center[1] + R * np.sin(ang)], 1)


def polygon_radius_after_sweep(n, k, R, alpha):
    num = rho = 0.0
    cnt = 0
    for m in range(1, k + 1):
        phi = 2 * math.pi * m / n
        w = 1.0 / m ** 2
        num += 2 * w * (R * math.cos(phi) + m * abs(math.sin(phi / 2)))
        rho += 2 * w
        cnt += 2
    return (num + alpha * (n - 1 - cnt) / (2 * R)) / rho


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("n", [7, 16, 51])
@pytest.mark.parametrize("alpha", [1.0, 0.027, 0.008])
def test_sweep_regular_polygon(k, n, alpha):
    rp, col = graphs.cycle(n)
    S = oracle.build_S(rp, col, k)
    R = 1.3
    x = polygon(n, R, center=(0.25, -0.5))
    xn, st = oracle.sweep(x, S, alpha, rep_mode=0)
    expect = polygon(n, polygon_radius_after_sweep(n, k, R, alpha), center=(0.25, -0.5))
    np.testing.assert_allclose(xn, expect, rtol=0, atol=1e-12)
    # stress of the input over S: n pairs at distance 1 (+ n at distance 2)
    stress = n * (2 * R * math.sin(math.pi / n) - 1) ** 2
    if k == 2:
        stress += n * 0.25 * (2 * R * math.sin(2 * math.pi / n) - 2) ** 2
    assert st[2] == pytest.approx(stress, rel=1e-12)


def test_sweep_polygon_fixed_point_k1():
    # R* = (1 + sqrt(1 + 2 alpha (n-3))) / (4 sin(pi/n)) is a fixed point
    n, alpha = 24, 0.3
    Rs = (1 + math.sqrt(1 + 2 * alpha * (n - 3))) / (4 * math.sin(math.pi / n))
    rp, col = graphs.cycle(n)
    S = oracle.build_S(rp, col, 1)
    x = polygon(n, Rs)
    xn, st = oracle.sweep(x, S, alpha, 0)
    np.testing.assert_allclose(xn, x, atol=1e-12)
    assert st[0] < 1e-20


def test_sweep_two_vertices_map():
    # K2 at distance D with target d: the vertices swap to distance |2d - D|
    rp, col = graphs.path(2)
    for D, d in [(0.5, 1.0), (3.0, 1.0), (1.7, 2.5)]:
        S = oracle.build_S(rp, col, 1, elen=np.array([d, d]))
        x = np.array([[0.0, 0.0], [D, 0.0]])
        xn, _ = oracle.sweep(x, S, 0.7, 0)
        np.testing.assert_allclose(xn, [[D - d, 0.0], [d, 0.0]], atol=1e-14)
    # the two-vertex initial layout (distance d) is a fixed point
    S = oracle.build_S(rp, col, 1, c=np.array([3.0, 5.0]), coarse=True)
    D = math.sqrt(3) + math.sqrt(5)
    x = np.array([[-D / 2, 0.0], [D / 2, 0.0]])
    xn, st = oracle.sweep(x, S, 1.0, 0)
    np.testing.assert_allclose(xn, x, atol=1e-14)


def _random_graph(n, seed):
    rp, col, pts, _ = graphs.rgg(n, 6.0, seed, tune=False)
    return rp, col, pts


@pytest.mark.parametrize("rep_mode", [0, 1])
def test_sweep_translation_rotation_equivariance(rep_mode):
    rp, col, pts = _random_graph(300, 3)
    S = oracle.build_S(rp, col, 2)
    x = graphs.uniform_positions(len(rp) - 1, 11, 0.0, 10.0)
    theta = 0.0  # BH with theta = 0 must match the exact sweep
    y, _ = oracle.sweep(x, S, 0.09, rep_mode, theta)
    t = np.array([3.5, -7.25])
    yt, _ = oracle.sweep(x + t, S, 0.09, rep_mode, theta)
    np.testing.assert_allclose(yt, y + t, atol=1e-9)
    a = 0.7
    Rm = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    yr, _ = oracle.sweep(x @ Rm.T, S, 0.09, rep_mode, theta)
    np.testing.assert_allclose(yr, y @ Rm.T, atol=1e-9)


def test_sweep_bh_theta0_equals_exact():
    rp, col, pts = _random_graph(400, 5)
    S = oracle.build_S(rp, col, 2)
    x = graphs.uniform_positions(len(rp) - 1, 2, 0.0, 20.0)
    a, _ = oracle.sweep(x, S, 0.3, 0)
    b, _ = oracle.sweep(x, S, 0.3, 1, 0.0)
    np.testing.assert_allclose(a, b, atol=1e-11)


# --------------------------------------------------------------------------
# Barnes-Hut (Sec. 2.2)
# --------------------------------------------------------------------------
def test_bh_far_cluster_closed_form():
    # u alone in its quadrant, a cluster B of N points with an off-centre
    # centroid in the opposite quadrant: B is accepted as one cell and
    # F(u) = N r(u, centroid(B)) exactly.
    B = np.array([[10.0 + 0.001 * i, 10.0 + 0.0007 * i] for i in range(9)] + [[10.1, 10.1]])
    x = np.vstack([[0.0, 0.0], B])
    c = B.mean(axis=0)
    expect = len(B) * (x[0] - c) / np.sum((x[0] - c) ** 2)
    for theta in (0.05, 0.3, 0.4):
        F = oracle.repulsion_bh(x, theta)
        np.testing.assert_allclose(F[0], expect, rtol=1e-13)
    # opened all the way (theta = 0): the exact sum, which differs
    F0 = oracle.repulsion_bh(x, 0.0)
    ex = oracle.repulsion_exact(x)
    np.testing.assert_allclose(F0, ex, rtol=1e-13)
    assert np.abs(F0[0] - expect).max() > 1e-9


@pytest.mark.parametrize("theta", [0.2, 0.5, 0.7])
def test_bh_multipole_remainder_bound(theta):
    # For an accepted cell of side w at centroid distance D > w / theta the
    # first-order term vanishes and the remainder of each member v is
    # |delta_v|^2 / (D^2 |x_u - x_v|) <= 2 theta^2 / |x_u - x_v|, so
    # |F_BH(u) - F(u)| <= 2 theta^2 sum_{v != u} 1 / |x_u - x_v|.
    rng = np.random.default_rng(7)
    x = np.vstack([rng.random((700, 2)) * 5.0, rng.normal(8.0, 0.3, (300, 2))])
    F = oracle.repulsion_bh(x, theta)
    ex = oracle.repulsion_exact(x)
    diff = x[:, None, :] - x[None, :, :]
    dist = np.sqrt((diff ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    bound = 2 * theta ** 2 * (1.0 / dist).sum(1)
    err = np.sqrt(((F - ex) ** 2).sum(1))
    assert np.all(err <= bound * (1 + 1e-9))
    assert err.max() > 0  # cells really were accepted


def test_bh_coincident_points():
    x = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0], [1.0, 0.0], [0.5, 2.0]])
    F = oracle.repulsion_bh(x, 0.5)
    ex = oracle.repulsion_exact(x)
    np.testing.assert_allclose(F, ex, atol=1e-12)
    # coincident partner contributes nothing
    np.testing.assert_allclose(ex[0], [-2.0 / 1.0 * 1 + -0.5 / 4.25, -2.0 / 4.25], atol=1e-12)


# --------------------------------------------------------------------------
# Objective, Eq. 1
# --------------------------------------------------------------------------
def test_objective_two_vertices():
    rp, col = graphs.path(2)
    S = oracle.build_S(rp, col, 1)
    for D in (0.3, 1.0, 2.5):
        x = np.array([[0.0, 0.0], [D, 0.0]])
        stress, lns, M = oracle.objective(x, S, 0.008)
        assert stress == pytest.approx((D - 1.0) ** 2)
        assert lns == 0.0 and M == pytest.approx((D - 1.0) ** 2)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("n", [9, 40])
def test_objective_regular_polygon(k, n):
    # sum over all unordered pairs of ln|x_i - x_j| on a regular n-gon:
    # prod_{j=1}^{n-1} 2 sin(pi j / n) = n gives (n/2) ((n-1) ln R + ln n).
    R, alpha = 2.2, 0.008
    rp, col = graphs.cycle(n)
    S = oracle.build_S(rp, col, k)
    x = polygon(n, R)
    stress, lns, M = oracle.objective(x, S, alpha)
    total = 0.5 * n * ((n - 1) * math.log(R) + math.log(n))
    exp_stress = 0.0
    for m in range(1, k + 1):
        dist = 2 * R * math.sin(math.pi * m / n)
        total -= n * math.log(dist)
        exp_stress += n * (dist - m) ** 2 / m ** 2
    assert lns == pytest.approx(total, rel=1e-12)
    assert stress == pytest.approx(exp_stress, rel=1e-12)
    assert M == pytest.approx(exp_stress - alpha * total, rel=1e-12)


def test_objective_sampled_regular_polygon_closed_form():
    # the estimator of the ln-sum (pairs outside S drawn at random) against
    # the same closed form: within 5 standard errors; the stress over S is
    # summed exactly
    n, R, alpha, k = 400, 7.0, 0.008, 2
    rp, col = graphs.cycle(n)
    S = oracle.build_S(rp, col, k)
    x = polygon(n, R)
    total = 0.5 * n * ((n - 1) * math.log(R) + math.log(n))
    exp_stress = 0.0
    for m in range(1, k + 1):
        dist = 2 * R * math.sin(math.pi * m / n)
        total -= n * math.log(dist)
        exp_stress += n * (dist - m) ** 2 / m ** 2
    est = oracle.objective_sampled(x, S, alpha, samples=400000, seed=3)
    assert est["stress"] == pytest.approx(exp_stress, rel=1e-12)
    assert 0 < est["se_lnsum"] < 2e-3 * abs(total)
    assert abs(est["lnsum"] - total) <= 5 * est["se_lnsum"]
    assert est["M"] == pytest.approx(est["stress"] - alpha * est["lnsum"], rel=1e-12)
    assert est["se_M"] == pytest.approx(alpha * est["se_lnsum"], rel=1e-12)
    # rejected draws: u == v (1/n of them) and pairs in S (2k/n of them)
    assert abs(est["kept"] / 400000 - (1 - (2 * k + 1) / n)) < 0.005


def test_objective_sampled_against_the_exact_sum_and_its_error_bars():
    rp, col = graphs.grid(25, 20)
    n = len(rp) - 1
    S = oracle.build_S(rp, col, 2)
    x = graphs.uniform_positions(n, 17, 0.0, 30.0)
    stress, lns, M = oracle.objective(x, S, 0.008)
    z = []
    for seed in range(8):
        est = oracle.objective_sampled(x, S, 0.008, samples=200000, seed=seed)
        assert est["stress"] == pytest.approx(stress, rel=1e-12)
        z.append((est["lnsum"] - lns) / est["se_lnsum"])
    # unbiased with the stated error: z-scores of 8 independent estimates
    assert max(abs(v) for v in z) < 4.5
    assert abs(np.mean(z)) < 4.5 / math.sqrt(8)
    # the same seed draws the same pairs
    a = oracle.objective_sampled(x, S, 0.008, samples=50000, seed=4)
    b = oracle.objective_sampled(x, S, 0.008, samples=50000, seed=4)
    assert a == b


def test_objective_sampled_coincident_points_give_zero():
    rp, col = graphs.path(50)
    S = oracle.build_S(rp, col, 1)
    est = oracle.objective_sampled(np.ones((50, 2)), S, 0.008, samples=10000, seed=1)
    assert est["lnsum"] == 0.0 and est["se_lnsum"] == 0.0
    assert est["stress"] == pytest.approx(49.0)  # 49 edges at distance 0, d = 1


# --------------------------------------------------------------------------
# SCLaP (Sec. 3.1): invariants and order-free cases
# --------------------------------------------------------------------------
def _cluster_weights(labels, c):
    w = {}
    for v, L in enumerate(labels):
        w[L] = w.get(L, 0.0) + c[v]
    return w


def test_sclap_matching_pairs():
    n = 40
    rp, col = graphs.csr_from_edges(n, np.arange(0, n, 2), np.arange(1, n, 2))
    lab = oracle.sclap(rp, col, np.ones(n), U=2.0, rounds=10, seed=1, level=0)
    for v in range(0, n, 2):
        assert lab[v] == lab[v + 1]
    assert len(set(lab.tolist())) == n // 2


def test_sclap_star_one_cluster():
    n = 30
    rp, col = graphs.csr_from_edges(n, np.zeros(n - 1, dtype=int), np.arange(1, n))
    for seed in range(5):
        lab = oracle.sclap(rp, col, np.ones(n), U=float(n), rounds=10, seed=seed, level=0)
        assert len(set(lab.tolist())) == 1


@pytest.mark.parametrize("U", [2.0, 3.0, 7.5])
def test_sclap_size_bound_and_partition(U):
    rp, col, _, _ = graphs.rgg(2000, 8.0, 9, tune=False)
    n = len(rp) - 1
    c = np.ones(n)
    lab = oracle.sclap(rp, col, c, U=U, rounds=10, seed=3, level=0)
    assert lab.shape == (n,) and lab.min() >= 0 and lab.max() < n
    w = _cluster_weights(lab, c)
    assert max(w.values()) <= U
    assert len(w) < n  # something merged


# Hand-worked rounds with the visiting order fixed (the order is the random
# draw of Sec. 3.1; passing it in makes the outcome checkable by hand).
def _wgraph(n, edges):
    """Symmetric CSR with per-entry weights omega from (u, v, w) triples."""
    adj = [[] for _ in range(n)]
    for u, v, w in edges:
        adj[u].append((v, w))
        adj[v].append((u, w))
    rp = np.zeros(n + 1, dtype=np.int64)
    col, ew = [], []
    for u in range(n):
        for v, w in sorted(adj[u]):
            col.append(v)
            ew.append(w)
        rp[u + 1] = len(col)
    return rp, np.array(col, dtype=np.int32), np.array(ew, dtype=np.float64)


def test_sclap_strongest_connection_not_most_neighbours_nor_first():
    # p = 5 sees three clusters: {0} by one edge of omega 0.5 (its first
    # neighbour in row order), {1, 2} by two edges of omega 1 (the most
    # neighbours, after 1 joined 2 over their omega-10 edge) and {3} by one
    # edge of omega 3: the strongest connection, sum 3 > 2 > 0.5, wins.
    rp, col, ew = _wgraph(6, [(1, 2, 10.0), (1, 5, 1.0), (2, 5, 1.0), (3, 5, 3.0),
                              (0, 5, 0.5), (4, 3, 0.25)])
    order = [[1, 2, 5, 3, 0, 4]]
    lab = oracle.sclap(rp, col, np.ones(6), U=10.0, rounds=1, seed=0, level=0, ew=ew,
                       order=order)
    # 1 -> {2}; 2 stays; 5 -> {3}; 3 stays (its cluster holds 5, omega 3);
    # 0 -> {3, 5} (its only neighbour); 4 -> {3, 5, 0} (its only neighbour)
    assert lab.tolist() == [3, 2, 2, 3, 3, 3]


def test_sclap_tie_keeps_own_cluster():
    # 2 joins 3 first (its only neighbour); then 3's own cluster {2, 3} has
    # connection 2 and the cluster {0, 1} (formed over omega 10) also 2:
    # a tie with the own cluster among the best keeps it, although label 1
    # is smaller.
    rp, col, ew = _wgraph(4, [(0, 1, 10.0), (0, 3, 1.0), (1, 3, 1.0), (2, 3, 2.0)])
    lab = oracle.sclap(rp, col, np.ones(4), U=10.0, rounds=1, seed=0, level=0, ew=ew,
                       order=[[0, 2, 3, 1]])
    assert lab.tolist() == [1, 1, 3, 3]


def test_sclap_tie_elsewhere_takes_smallest_label():
    # 4's two neighbouring clusters {0, 3} (label 3, reached through vertex 0,
    # the first entry of 4's row) and {2, 1} (label 1) both connect with 1;
    # its own singleton connects with 0: the smallest label, 1, wins.
    rp, col, ew = _wgraph(5, [(0, 3, 10.0), (2, 1, 10.0), (0, 4, 1.0), (2, 4, 1.0)])
    lab = oracle.sclap(rp, col, np.ones(5), U=10.0, rounds=1, seed=0, level=0, ew=ew,
                       order=[[0, 2, 4, 3, 1]])
    assert lab.tolist() == [3, 1, 1, 3, 1]


def test_sclap_overload_forces_second_best_and_bound_is_inclusive():
    # U = 3: vertex 0 weighs 3, so 3 cannot join it (3 + 1 > U) and takes
    # its second-strongest cluster {1}; 2 then joins {1, 3} reaching exactly
    # U (weight + c(v) <= U is allowed); 0 can join nothing.
    rp, col, ew = _wgraph(4, [(0, 3, 3.0), (1, 3, 2.0), (2, 3, 1.0)])
    c = np.array([3.0, 1.0, 1.0, 1.0])
    lab = oracle.sclap(rp, col, c, U=3.0, rounds=1, seed=0, level=0, ew=ew,
                       order=[[3, 1, 2, 0]])
    assert lab.tolist() == [0, 1, 1, 1]
    # with room for it, the strongest cluster {0} is taken
    lab = oracle.sclap(rp, col, c, U=4.0, rounds=1, seed=0, level=0, ew=ew,
                       order=[[3, 1, 2, 0]])
    assert lab[3] == 0


def test_sclap_converged_labels_are_locally_optimal():
    # After label propagation has converged (a round moved nothing), no
    # vertex has a neighbouring cluster that would fit it (weight + c(v) <=
    # U) and connects more strongly than its own cluster (Sec. 3.1: a vertex
    # moves to the strongest connection).  Random omega makes this differ
    # from counting neighbours.
    rp, col, _, _ = graphs.rgg(1500, 7.0, 31, tune=False)
    n = len(rp) - 1
    rng = np.random.default_rng(5)
    src = np.repeat(np.arange(n), np.diff(rp))
    key = np.minimum(src, col).astype(np.int64) * n + np.maximum(src, col)
    _, inv = np.unique(key, return_inverse=True)
    ew = rng.uniform(0.1, 5.0, inv.max() + 1)[inv]   # symmetric omega
    c = rng.integers(1, 4, n).astype(np.float64)
    U = 9.0
    lab = oracle.sclap(rp, col, c, U=U, rounds=400, seed=8, level=2, ew=ew)
    wt = np.zeros(n)
    np.add.at(wt, lab, c)
    assert wt.max() <= U
    checked = 0
    for v in range(n):
        conn = {}
        for e in range(rp[v], rp[v + 1]):
            L = int(lab[col[e]])
            conn[L] = conn.get(L, 0.0) + ew[e]
        own = conn.get(int(lab[v]), 0.0)
        for L, s in conn.items():
            if L != lab[v] and wt[L] + c[v] <= U:
                assert s <= own + 1e-12, (v, L, s, own)
                checked += 1
    assert checked > n // 2  # the condition was tested on many candidate moves


# --------------------------------------------------------------------------
# Coarsening schedule (Sec. 3.1): W = min(b^(h+1), |V|/f), U = max(max c, W),
# f := 0.7 f after a contraction that shrinks by at most 10 %, a contraction
# that merges nothing discarded (f := 0.7 f, retried)
# --------------------------------------------------------------------------
def test_coarsening_schedule_hand_worked_on_a_star():
    # A star with centre 0 and 199 leaves (|V| = 200).  Leaves touch only the
    # centre, so on every level the centre's cluster grows to floor(U)
    # (integral weights) whatever the visiting order, nothing else merges,
    # and each level is again a star.  Worked by hand, attempt by attempt
    # (f_j = 20 * 0.7^j):
    #   h  f    W = min(2^(h+1), 200/f)   U = max(max c, W)  n -> n'
    #   0  f0   min(2, 10)      = 2        2                 200 -> 199  1 %: f := 0.7 f
    #   1  f1   min(4, 14.29)   = 4        4                 199 -> 197  f := 0.7 f
    #   2  f2   min(8, 20.41)   = 8        8                 197 -> 193  f := 0.7 f
    #   3  f3   min(16, 29.15)  = 16       16                193 -> 185  f := 0.7 f
    #   4  f4   min(32, 41.65)  = 32       32                185 -> 169  8.6 %: f := 0.7 f
    #   5  f5   min(64, 59.50)  = 59.50    59.50             169 -> 142  16 %: f kept
    #   6  f5   59.50                      59.50 (centre 59) nothing merges: discarded, f := 0.7 f
    #   6  f6   min(128, 85.00) = 85.00    85.00             142 -> 117  f kept
    #   7  f6   85.00                      85.00 (centre 84) discarded, f := 0.7 f
    #   7  f7   min(256, 121.43)           121.43            117 -> 80
    #   8  f7   121.43                     (centre 121)      discarded, f := 0.7 f
    #   8  f8   min(512, 173.47)           173.47             80 -> 28
    #   9  f8   173.47                     (centre 173)      discarded, f := 0.7 f
    #   9  f9.. 247.81, ...: the whole star merges into one vertex (n' < 2):
    #      discarded, f := 0.7 f, until max_stalls = 10 ends the coarsening
    n = 200
    rp, col = graphs.csr_from_edges(n, np.zeros(n - 1, dtype=int), np.arange(1, n))
    log = []
    p = oracle.params(k=1, coarsest_n=2, seed=11)
    levels = oracle.build_hierarchy(rp, col, p, log=log)
    assert [L["n"] for L in levels] == [200, 199, 197, 193, 185, 169, 142, 117, 80, 28]
    assert [float(L["c"].max()) for L in levels] == [1, 2, 4, 8, 16, 32, 59, 84, 121, 173]
    T, F = True, False
    rows = [  # (h, f, W, U, n, n', kept)
        (0, 20.0, 2.0, 2.0, 200, 199, T),
        (1, 14.0, 4.0, 4.0, 199, 197, T),
        (2, 9.8, 8.0, 8.0, 197, 193, T),
        (3, 6.86, 16.0, 16.0, 193, 185, T),
        (4, 4.802, 32.0, 32.0, 185, 169, T),
        (5, 3.3614, 59.499018266, 59.499018266, 169, 142, T),
        (6, 3.3614, 59.499018266, 59.499018266, 142, 142, F),
        (6, 2.35298, 84.998597523, 84.998597523, 142, 117, T),
        (7, 2.35298, 84.998597523, 84.998597523, 117, 117, F),
        (7, 1.647086, 121.426567890, 121.426567890, 117, 80, T),
        (8, 1.647086, 121.426567890, 121.426567890, 80, 80, F),
        (8, 1.1529602, 173.466525557, 173.466525557, 80, 28, T),
        (9, 1.1529602, 173.466525557, 173.466525557, 28, 28, F),
    ]
    assert len(log) == len(rows) + 9
    for got, want in zip(log, rows):
        assert got[0] == want[0] and got[4:] == want[4:], (got, want)
        assert got[1:4] == pytest.approx((want[2], want[3], want[1]), rel=1e-9), (got, want)
    f = 1.1529602
    for got in log[len(rows):]:
        f *= 0.7
        assert got[0] == 9 and got[3] == pytest.approx(f, rel=1e-9)
        assert got[5] == 1 and not got[6]


# --------------------------------------------------------------------------
# Initial layout of the coarsest level (Sec. 3.1 'Initial Layout')
# --------------------------------------------------------------------------
def test_place_coarsest_radius_and_moments():
    # more than two coarsest vertices: polar placement around the origin,
    # angle uniform in [0, 2 pi), radius uniform in [0, sqrt(sum c))
    n = 200000
    c = np.tile([1.0, 2.0, 5.0], n // 3 + 1)[:n]
    x = oracle.place_coarsest(c, seed=5, level=7)
    R = math.sqrt(c.sum())
    r = np.sqrt((x ** 2).sum(1))
    assert np.all(r < R)
    t = r / R
    assert abs(t.mean() - 0.5) < 0.005 and abs(t.var() - 1 / 12) < 0.002
    ang = np.arctan2(x[:, 1], x[:, 0])
    assert abs(np.cos(ang).mean()) < 0.01 and abs(np.sin(ang).mean()) < 0.01
    assert abs((np.cos(ang) ** 2).mean() - 0.5) < 0.01
    # the angle histogram is flat (8 sectors, 5 sigma)
    hist = np.histogram(ang, bins=8, range=(-math.pi, math.pi))[0]
    assert np.all(np.abs(hist - n / 8) < 5 * math.sqrt(n / 8))
    # reproducible; another seed or level draws other numbers; and not the
    # prolongation's draws (another Philox counter)
    assert np.array_equal(x, oracle.place_coarsest(c, seed=5, level=7))
    assert not np.array_equal(x, oracle.place_coarsest(c, seed=6, level=7))
    assert not np.array_equal(x, oracle.place_coarsest(c, seed=5, level=8))
    xp = oracle.prolong(np.zeros(n, dtype=np.int32), np.zeros((1, 2)), np.array([c.sum()]),
                        seed=5, level=7)
    assert not np.allclose(x, xp)


def test_initial_layout_two_vertices_at_target_distance():
    # two coarsest vertices are placed at their target distance, which on a
    # coarse level is sqrt(c_u) + sqrt(c_v) (Sec. 3.2); that is a fixed
    # point of Eq. 2 with S = E (one sweep leaves it in place)
    rp, col = graphs.path(2)
    c = np.array([4.0, 9.0])
    S = oracle.build_S(rp, col, 1, c=c, coarse=True)
    L = dict(n=2, S=S, c=c)
    x = oracle.initial_layout(L, oracle.params(), 3)
    assert np.linalg.norm(x[0] - x[1]) == pytest.approx(5.0, rel=1e-15)
    x1, st = oracle.sweep(x, S, 1.0, 0)
    assert np.allclose(x1, x, atol=1e-12)


# --------------------------------------------------------------------------
# Contraction (Sec. 3.1): hand-worked example and invariants
# --------------------------------------------------------------------------
def test_contract_hand_example():
    g = contract_example()
    mp, cc, crp, ccol, cew = oracle.contract(g["rp"], g["col"], np.ones(g["n"]), g["labels"],
                                             ew=g["ew"])
    assert mp.tolist() == g["map"].tolist()
    assert cc.tolist() == g["c"].tolist()
    assert crp.tolist() == g["crp"].tolist()
    assert ccol.tolist() == g["ccol"].tolist()
    assert cew.tolist() == g["cew"].tolist()


def test_contract_invariants():
    rp, col, _, _ = graphs.rgg(3000, 8.0, 21, tune=False)
    n = len(rp) - 1
    c = np.ones(n)
    lab = oracle.sclap(rp, col, c, U=4.0, rounds=10, seed=5, level=1)
    mp, cc, crp, ccol, cew = oracle.contract(rp, col, c, lab)
    nc = len(cc)
    assert cc.sum() == n
    src = np.repeat(np.arange(n), np.diff(rp))
    cut = mp[src] != mp[col]
    assert cew.sum() == cut.sum()  # sum of omega over cut entries is preserved
    csrc = np.repeat(np.arange(nc), np.diff(crp))
    assert np.all(csrc != ccol)  # no self-loops
    pairs = set(zip(csrc.tolist(), ccol.tolist()))
    assert all((b, a) in pairs for a, b in pairs)  # symmetric
    assert len(graphs.largest_component(crp, ccol)[2]) == nc  # connected


# --------------------------------------------------------------------------
# Prolongation (Sec. 3.2)
# --------------------------------------------------------------------------
def test_prolong_radius_and_moments():
    nf, nc = 200000, 3
    mp = np.arange(nf) % nc
    xc = np.array([[0.0, 0.0], [10.0, 5.0], [-4.0, 2.0]])
    cc = np.array([1.0, 4.0, 9.0])
    xf = oracle.prolong(mp, xc, cc, seed=77, level=2)
    off = xf - xc[mp]
    r = np.sqrt((off ** 2).sum(1))
    R = np.sqrt(cc)[mp]
    assert np.all(r <= R)
    # radius uniform in [0, R): mean R/2, var R^2/12; angle uniform
    t = r / R
    assert abs(t.mean() - 0.5) < 0.005 and abs(t.var() - 1 / 12) < 0.002
    ang = np.arctan2(off[:, 1], off[:, 0])
    assert abs(np.cos(ang).mean()) < 0.01 and abs(np.sin(ang).mean()) < 0.01
    # reproducible, and different levels draw different numbers
    assert np.array_equal(xf, oracle.prolong(mp, xc, cc, seed=77, level=2))
    assert not np.array_equal(xf, oracle.prolong(mp, xc, cc, seed=77, level=3))


# --------------------------------------------------------------------------
# alpha schedule (Sec. 3.2, Sec. 4 'Algorithm Configuration')
# --------------------------------------------------------------------------
def test_alpha_rounds_values():
    p = oracle.params()
    assert oracle.alpha_rounds(p) == pytest.approx([1.0, 0.3, 0.09, 0.027, 0.0081, 0.008])


def test_schedule_counts():
    rp, col = graphs.path(2)
    S = oracle.build_S(rp, col, 1)
    x = np.array([[-0.5, 0.0], [0.5, 0.0]])   # fixed point: every round exits after 1
    p = oracle.params()
    _, sweeps = oracle.schedule(S, x, p, 0)
    assert sweeps == 6
    p = oracle.params(early_exit=0, max_iters_at_min=90)
    _, sweeps = oracle.schedule(S, x, p, 0)
    assert sweeps == 100


def test_layout_small_multilevel_runs():
    rp, col = graphs.grid(12, 12)
    p = oracle.params(k=2, theta=0.5, coarsest_n=2, seed=4)
    x, info = oracle.layout(rp, col, p)
    assert x.shape == (144, 2) and np.all(np.isfinite(x))
    levels = info["levels"]
    assert levels[-1]["n"] <= 2
    for a, b in zip(levels[:-1], levels[1:]):
        assert b["n"] < a["n"]
        assert b["c"].sum() == 144
    # the layout is far better than the random start in Eq. 1
    S = levels[0]["S"]
    M_lay = oracle.objective(x, S, 0.008)[2]
    M_rand = oracle.objective(graphs.uniform_positions(144, 1, 0, 12), S, 0.008)[2]
    assert M_lay < M_rand


# ------------------------------------------------- Eq. 3 (MulMent_h) ---
def test_repulsion_h_identity_and_single_cluster_are_exact():
    # Sec. 3.2: with M the identity Eq. 3 is the exact sum of Eq. 2; with one
    # cluster holding every vertex its first sum is the exact sum and the
    # second is empty
    x = graphs.uniform_positions(60, 4, 0.0, 10.0)
    F = oracle.repulsion_exact(x)
    scale = np.abs(F).max()
    assert np.abs(oracle.repulsion_h(x, np.arange(60)) - F).max() <= 1e-12 * scale
    assert np.abs(oracle.repulsion_h(x, np.zeros(60, dtype=np.int32)) - F).max() <= 1e-12 * scale


def _two_clusters(D, rng_seed=3):
    rng = np.random.default_rng(rng_seed)
    a = rng.uniform(-1, 1, (5, 2))
    b = rng.uniform(-1, 1, (7, 2)) + np.array([D, 0.0])
    x = np.vstack([a, b])
    cmap = np.array([0] * 5 + [1] * 7, dtype=np.int32)
    return x, cmap


def test_repulsion_h_far_field_error_is_third_order():
    # the far cluster is replaced by nu = 7 copies of its midpoint: with the
    # plain midpoint the first-order (dipole) term of the expansion vanishes,
    # so the error at the near cluster falls as 1/D^3 (a weighted midpoint
    # or a wrong nu would leave a 1/D^2 or 1/D error); exact within a cluster
    errs = []
    for D in (20.0, 40.0, 80.0):
        x, cmap = _two_clusters(D)
        Fh = oracle.repulsion_h(x, cmap)
        Fe = oracle.repulsion_exact(x)
        errs.append(np.abs(Fh[:5] - Fe[:5]).max())
        # the near part is exact: removing the far cluster's exact and
        # approximated contributions leaves the same numbers
        far_exact = np.zeros((5, 2))
        for i in range(5):
            d = x[i] - x[5:]
            far_exact[i] = (d / (d ** 2).sum(1, keepdims=True)).sum(0)
        mid = x[5:].mean(0)
        d = x[:5] - mid
        far_h = 7 * d / (d ** 2).sum(1, keepdims=True)
        assert np.allclose(Fh[:5] - far_h, Fe[:5] - far_exact, rtol=0, atol=1e-12)
    assert 6.5 <= errs[0] / errs[1] <= 9.5, errs
    assert 6.5 <= errs[1] / errs[2] <= 9.5, errs


def test_repulsion_h_equivariance_and_scaling():
    x = graphs.uniform_positions(40, 9, 0.0, 8.0)
    cmap = np.random.default_rng(2).integers(0, 6, 40).astype(np.int32)
    F = oracle.repulsion_h(x, cmap)
    c, s = math.cos(0.7), math.sin(0.7)
    R = np.array([[c, -s], [s, c]])
    assert np.allclose(oracle.repulsion_h(x + np.array([3.0, -5.0]), cmap), F, atol=1e-10)
    assert np.allclose(oracle.repulsion_h(x @ R.T, cmap), F @ R.T, atol=1e-10)
    assert np.allclose(oracle.repulsion_h(2.5 * x, cmap), F / 2.5, atol=1e-10)


def test_sweep_h_with_identity_map_is_the_exact_sweep():
    rp, col = graphs.grid(6, 7)
    n = len(rp) - 1
    S = oracle.build_S(rp, col, 2)
    x = graphs.uniform_positions(n, 5, 0.0, 6.0)
    xe, ste = oracle.sweep(x, S, 0.3, 0)
    xh, sth = oracle.sweep(x, S, 0.3, 2, cmap=np.arange(n))
    assert np.abs(xh - xe).max() <= 1e-10 * np.abs(xe).max()
    assert np.allclose(sth, ste, rtol=1e-12)


def test_exact_max_n_selects_the_exact_sum_by_level_size():
    # levels of at most exact_max_n vertices take the exact entropy sum: with
    # the threshold above every level the layout is the exact_repulsion = 1
    # layout bit for bit; with threshold 0 only the coarsest level is exact
    # and the Barnes-Hut levels give a different layout; a threshold between
    # two level sizes makes exactly the levels below it exact
    rp, col = graphs.grid(12, 12)
    base = dict(k=2, theta=0.5, coarsest_n=2, seed=4)
    levels = oracle.build_hierarchy(rp, col, oracle.params(**base))
    x_all, _ = oracle.layout(rp, col, oracle.params(**base, exact_max_n=144), levels=levels)
    x_ex, _ = oracle.layout(rp, col, oracle.params(**base, exact_repulsion=1), levels=levels)
    x_bh, _ = oracle.layout(rp, col, oracle.params(**base, exact_max_n=0), levels=levels)
    assert np.array_equal(x_all, x_ex)
    assert not np.array_equal(x_all, x_bh)
    # threshold = the size of level 1: the coarse levels are exact (the same
    # sweeps as the all-exact run, step for step), level 0 is Barnes-Hut
    n1 = int(levels[1]["n"])
    tr_mid, tr_ex = [], []
    _, info_mid = oracle.layout(rp, col, oracle.params(**base, exact_max_n=n1), levels=levels,
                                trace=tr_mid)
    _, info_ex = oracle.layout(rp, col, oracle.params(**base, exact_repulsion=1), levels=levels,
                               trace=tr_ex)
    assert info_mid["sweeps"][1:] == info_ex["sweeps"][1:]
    coarse = sum(info_ex["sweeps"][1:])
    assert tr_mid[:coarse] == tr_ex[:coarse]
    assert tr_mid[coarse:] != tr_ex[coarse:]


def test_layout_h_runs_and_maps_compose():
    rp, col = graphs.grid(12, 12)
    p = oracle.params(k=2, coarsest_n=2, seed=4, approx_levels=2)
    levels = oracle.build_hierarchy(rp, col, p)
    # the composed map of level 0 is the two maps applied in turn
    m = oracle.approx_map(levels, 0, 2)
    assert np.array_equal(m, levels[1]["map"][levels[0]["map"]])
    assert m.max() + 1 == levels[2]["n"]
    top = len(levels) - 1
    assert np.array_equal(oracle.approx_map(levels, top - 1, 5),
                          levels[top - 1]["map"])
    x, info = oracle.layout(rp, col, p, levels=levels)
    assert np.all(np.isfinite(x))
    S = levels[0]["S"]
    M_lay = oracle.objective(x, S, 0.008)[2]
    M_rand = oracle.objective(graphs.uniform_positions(144, 1, 0, 12), S, 0.008)[2]
    assert M_lay < M_rand


# --------------------------------------------- full stress and scale s ---
def test_full_stress_path_on_a_line():
    # a path drawn on a line with unit spacing realises every distance:
    # F = 0 and s = 1; drawn at spacing 2, F = one per pair and s = 1/2
    rp, col = graphs.path(12)
    x = np.stack([np.arange(12.0), np.zeros(12)], 1)
    F, s, Fs, pairs = oracle.full_stress(rp, col, x)
    assert pairs == 66 and F == pytest.approx(0.0, abs=1e-12) and s == pytest.approx(1.0)
    F, s, Fs, pairs = oracle.full_stress(rp, col, 2.0 * x)
    assert F == pytest.approx(66.0) and s == pytest.approx(0.5) and Fs == pytest.approx(0.0, abs=1e-9)


def test_full_stress_two_vertices():
    rp, col = graphs.path(2)
    x = np.array([[0.0, 0.0], [3.0, 4.0]])   # |dx| = 5, d = 1
    F, s, Fs, pairs = oracle.full_stress(rp, col, x)
    assert F == pytest.approx(16.0) and s == pytest.approx(0.2) and Fs == pytest.approx(0.0, abs=1e-12)


def test_full_stress_matches_library_shortest_paths():
    csg = pytest.importorskip("scipy.sparse.csgraph")
    sps = pytest.importorskip("scipy.sparse")
    rp, col, _, _ = graphs.rgg(300, 6.0, 12)
    n = len(rp) - 1
    x = graphs.uniform_positions(n, 3, 0.0, 10.0)
    D = csg.shortest_path(sps.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n)),
                          unweighted=True)
    iu = np.triu_indices(n, 1)
    d = D[iu]
    L = np.sqrt(((x[iu[0]] - x[iu[1]]) ** 2).sum(1))
    w = 1.0 / d ** 2
    F_ref = (w * (L - d) ** 2).sum()
    s_ref = (w * d * L).sum() / (w * L * L).sum()
    F, s, Fs, pairs = oracle.full_stress(rp, col, x)
    assert pairs == len(d)
    assert F == pytest.approx(F_ref, rel=1e-12) and s == pytest.approx(s_ref, rel=1e-12)
    assert Fs == pytest.approx((w * (s_ref * L - d) ** 2).sum(), rel=1e-9)


# --------------------------------------- whole multilevel layout, closed form ---
@pytest.mark.parametrize("n", [3, 4, 5])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_layout_complete_graph_ends_as_stress_optimal_polygon(n, seed):
    # K_n with k = 1: S holds every pair, so Eq. 2 has no entropy term and the
    # whole multilevel run (coarsening, coarsest placement, prolongation,
    # schedule) must end at a stress minimum; for n = 3, 4, 5 that is the
    # regular n-gon whose circumradius R minimises sum (chord - 1)^2 over all
    # pairs: R = sum m_j L_j / sum m_j L_j^2 with L_j = 2 sin(pi j / n) and m_j
    # chords of each length
    rp, col = graphs.complete(n)
    x, info = oracle.layout(rp, col, oracle.params(k=1, coarsest_n=2, seed=seed))
    js = np.arange(1, n // 2 + 1)
    m = np.where(2 * js == n, n / 2, n)
    L = 2 * np.sin(np.pi * js / n)
    R = (m * L).sum() / (m * L * L).sum()
    r = np.sqrt(((x - x.mean(0)) ** 2).sum(1))
    assert np.allclose(r, R, rtol=2e-3), (r, R)
    D = np.sort(np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1))[np.triu_indices(n, 1)])
    chords = np.sort(np.concatenate([np.full(int(mj), R * Lj) for mj, Lj in zip(m, L)]))
    assert np.allclose(D, chords, rtol=3e-3), (D, chords)
    assert len(info["levels"]) >= 2


def test_layout_path3_with_k2_ends_collinear_at_unit_spacing():
    # P3 with k = 2: S holds every pair (distances 1, 1, 2), no entropy term;
    # the stress-free layout is the path on a line at unit spacing
    rp, col = graphs.path(3)
    x, _ = oracle.layout(rp, col, oracle.params(k=2, coarsest_n=2, seed=1,
                                                 max_iters_at_min=2000, eps_final=1e-9))
    d = [np.linalg.norm(x[0] - x[1]), np.linalg.norm(x[1] - x[2]), np.linalg.norm(x[0] - x[2])]
    assert np.allclose(d, [1.0, 1.0, 2.0], rtol=1e-3), d


@pytest.mark.parametrize("n,seed", [(12, 1), (12, 2), (24, 1), (24, 2)])
def test_layout_cycle_ends_as_the_fixed_point_polygon(n, seed):
    # C_n with k = 1 and the exact entropy sum: run to convergence, the whole
    # multilevel layout ends at the regular n-gon of radius
    # R* = (1 + sqrt(1 + 2 alpha (n - 3))) / (4 sin(pi / n)) at alpha_min, the
    # fixed point of Eq. 2 on a regular polygon (see the sweep pins above)
    rp, col = graphs.cycle(n)
    x, _ = oracle.layout(rp, col, oracle.params(k=1, coarsest_n=2, seed=seed,
                                                 exact_repulsion=1, max_iters_at_min=3000,
                                                 eps_final=1e-10))
    alpha = 0.008
    Rs = (1 + math.sqrt(1 + 2 * alpha * (n - 3))) / (4 * math.sin(math.pi / n))
    c = x.mean(0)
    r = np.sqrt(((x - c) ** 2).sum(1))
    assert np.allclose(r, Rs, rtol=1e-4), (r.min(), r.max(), Rs)
    # neighbours along the cycle are adjacent corners of the polygon
    d = np.sqrt(((x - np.roll(x, 1, axis=0)) ** 2).sum(1))
    assert np.allclose(d, 2 * Rs * math.sin(math.pi / n), rtol=1e-4)
