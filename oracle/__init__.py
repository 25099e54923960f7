"""FP64 CPU oracle for the MulMent hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it; the only shared module is the seeded input generator
(``paper_1506_04383_gb300.graphs``), which contains none of the method's
arithmetic.

Arithmetic lives in ``mm_oracle.c`` (plain C99, double precision); this module
wraps it with numpy arrays and runs the multilevel orchestration of Sec. 3 of
the paper (coarsening, initial layout, prolongation, alpha schedule) step by
step in the order the paper gives them.

Pins (tests under ``tests/test_oracle_*.py``, all CPU):
  * Philox4x32-10 against published known-answer vectors.
  * ``build_S`` on cycles/paths/grids against hand-counted neighbourhoods.
  * ``sweep`` (exact) against the regular-polygon closed form for cycles
    (one sweep maps a regular n-gon to a regular n-gon with a radius given by
    a formula derived from Eq. 2), the two-vertex map |2d - D|, translation
    and rotation equivariance.
  * ``repulsion_bh`` equals the exact sum at theta = 0 and stays within the
    2-D multipole remainder bound for far clusters.
  * ``objective`` against closed forms for K2 and for a regular polygon (the
    product identity prod_j 2 sin(pi j / n) = n).
  * ``sclap`` by invariants (partition, size bound U), order-free cases
    (perfect matching, star), hand-worked rounds with the visiting order
    passed in (strongest connection rather than most neighbours or first
    neighbour, both tie rules, the inclusive overload bound that forces the
    second-best cluster) and local optimality of converged labels on a
    weighted random graph.
  * ``build_hierarchy``'s schedule (W = min(b^(h+1), |V|/f), U, f := 0.7 f
    after a shrink of at most 10 %, discarded empty contractions) level by
    level against a hand-worked star.
  * ``contract`` against a hand-worked example and invariants.
  * ``prolong`` and ``place_coarsest`` by their radius bounds and
    distribution moments; two coarsest vertices at their target distance.
  * ``objective_sampled`` (the ln-sum outside S from random pairs) against
    the polygon closed form and the exact sum, within its standard error.
Multilevel ``layout`` composes pinned steps; beyond that its end-to-end
result is pinned by closed-form final layouts of small graphs (complete
graphs, cycles, a path).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_DEPTH = 16  # quadtree depth limit (buckets below it)


def build(force: bool = False) -> str:
    """Compile mm_oracle.c into liboracle.so (gcc, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_build_S.argtypes = [i32, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.orc_build_S.restype = i64
        lib.orc_repulsion_exact.argtypes = [i32, P, P]
        lib.orc_repulsion_bh.argtypes = [i32, P, f64, ctypes.c_int, P, P]
        lib.orc_sweep.argtypes = [i32, P, P, P, P, P, f64, ctypes.c_int, f64, ctypes.c_int, P,
                                  i32, P, P]
        lib.orc_repulsion_h.argtypes = [i32, P, P, i32, P]
        lib.orc_full_stress.argtypes = [i32, P, P, P, P]
        lib.orc_objective.argtypes = [i32, P, P, P, P, f64, P]
        lib.orc_objective_sampled.argtypes = [i32, P, P, P, P, f64, i64, u64, P]
        lib.orc_sclap.argtypes = [i32, P, P, P, P, f64, ctypes.c_int, u64, i32, P, P]
        lib.orc_contract.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_contract.restype = i32
        lib.orc_prolong.argtypes = [i32, P, P, P, u64, i32, P]
        lib.orc_place_coarsest.argtypes = [i32, P, u64, i32, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: four 32-bit counter words, two key words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def build_S(rp, col, k: int, elen=None, c=None, coarse: bool = False):
    """k-hop pair set S with distances d and rho (Sec. 2.3 footnote, Eq. 2).

    Returns (sp, scol, sd, rho); rows ascending in vertex id."""
    lib = _load()
    rp, col = _i64(rp), _i32(col)
    n = len(rp) - 1
    elen, c = _f64(elen), _f64(c)
    sp = np.zeros(n + 1, dtype=np.int64)
    nnz = lib.orc_build_S(n, _p(rp), _p(col), _p(elen), _p(c), int(coarse), int(k),
                          _p(sp), None, None, None)
    if nnz < 0:
        raise ValueError("orc_build_S failed")
    scol = np.zeros(max(nnz, 1), dtype=np.int32)
    sd = np.zeros(max(nnz, 1), dtype=np.float64)
    rho = np.zeros(max(n, 1), dtype=np.float64)
    lib.orc_build_S(n, _p(rp), _p(col), _p(elen), _p(c), int(coarse), int(k),
                    _p(sp), _p(scol), _p(sd), _p(rho))
    return sp, scol[:nnz], sd[:nnz], rho[:n]


def repulsion_exact(x) -> np.ndarray:
    """F_u = sum_{v != u} r(u, v) (Sec. 2.3 r-values), exact."""
    lib = _load()
    x = _f64(x).reshape(-1, 2)
    F = np.zeros_like(x)
    lib.orc_repulsion_exact(len(x), _p(x), _p(F))
    return F


def repulsion_bh(x, theta: float, max_depth: int = MAX_DEPTH, counts: bool = False):
    """Barnes-Hut estimate of F_u with a pointer quadtree (Sec. 2.2)."""
    lib = _load()
    x = _f64(x).reshape(-1, 2)
    F = np.zeros_like(x)
    nacc = np.zeros(len(x), dtype=np.int64) if counts else None
    lib.orc_repulsion_bh(len(x), _p(x), float(theta), int(max_depth), _p(F), _p(nacc))
    return (F, nacc) if counts else F


def repulsion_h(x, cmap) -> np.ndarray:
    """The first two sums of Eq. 3 (Sec. 3.2, "Faster Local Improvement"):
    exact r-values within u's coarse representative, one nu-scaled r-value
    towards the midpoint of every other one.  cmap maps the current level's
    vertices to the vertices of the approximating level."""
    lib = _load()
    x = _f64(x).reshape(-1, 2)
    cmap = _i32(cmap)
    nc = int(cmap.max()) + 1 if len(cmap) else 0
    F = np.zeros_like(x)
    lib.orc_repulsion_h(len(x), _p(x), _p(cmap), nc, _p(F))
    return F


def sweep(x, S, alpha: float, rep_mode: int = 0, theta: float = 0.5,
          max_depth: int = MAX_DEPTH, cmap=None):
    """One Jacobi iteration of Eq. 2.  rep_mode 0 = exact, 1 = Barnes-Hut,
    2 = the hierarchy approximation of Eq. 3 with the map cmap.

    Returns (x_new, stats) with stats = [sum|dx|^2, sum|x|^2, stress(x)]."""
    lib = _load()
    sp, scol, sd, rho = S
    x = _f64(x).reshape(-1, 2)
    out = np.zeros_like(x)
    st = np.zeros(3, dtype=np.float64)
    cm = _i32(cmap) if cmap is not None else None
    nc = int(cm.max()) + 1 if cm is not None and len(cm) else 0
    lib.orc_sweep(len(x), _p(x), _p(_i64(sp)), _p(_i32(scol)), _p(_f64(sd)),
                  _p(_f64(rho)), float(alpha), int(rep_mode), float(theta),
                  int(max_depth), _p(cm), nc, _p(out), _p(st))
    return out, st


def objective(x, S, alpha: float):
    """Eq. 1 over S: returns (stress, ln-sum over pairs not in S, M)."""
    lib = _load()
    sp, scol, sd, _ = S
    x = _f64(x).reshape(-1, 2)
    out = np.zeros(3, dtype=np.float64)
    lib.orc_objective(len(x), _p(x), _p(_i64(sp)), _p(_i32(scol)), _p(_f64(sd)),
                      float(alpha), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def objective_sampled(x, S, alpha: float, samples: int = 10_000_000, seed: int = 1506):
    """Eq. 1 with the stress over S exact and the ln-sum over pairs outside
    S estimated from `samples` random pairs (for graphs whose O(n^2) sum is
    out of reach; Sec. 4 calls the exact measures infeasible for large
    graphs).  Returns dict(stress, lnsum, M, se_lnsum, se_M, kept); the
    standard errors are those of the sample mean.  The same seed draws the
    same pairs, so two layouts of one graph are compared on common pairs."""
    lib = _load()
    sp, scol, sd, _ = S
    x = _f64(x).reshape(-1, 2)
    out = np.zeros(5, dtype=np.float64)
    lib.orc_objective_sampled(len(x), _p(x), _p(_i64(sp)), _p(_i32(scol)), _p(_f64(sd)),
                              float(alpha), int(samples), int(seed) & 0xFFFFFFFFFFFFFFFF,
                              _p(out))
    return dict(stress=float(out[0]), lnsum=float(out[1]), M=float(out[2]),
                se_lnsum=float(out[3]), se_M=float(alpha * out[3]), kept=int(out[4]))


def full_stress(rp, col, x):
    """Full stress over all connected unordered pairs with hop distances and
    w = d^-2, the stress-minimising scale s and the stress at s x (Sec. 4,
    methodology).  Returns (F(x), s, F(s x), pairs)."""
    lib = _load()
    x = _f64(x).reshape(-1, 2)
    out = np.zeros(4, dtype=np.float64)
    lib.orc_full_stress(len(x), _p(_i64(rp)), _p(_i32(col)), _p(x), _p(out))
    return float(out[0]), float(out[1]), float(out[2]), int(out[3])


def sclap(rp, col, c, U: float, rounds: int, seed: int, level: int, ew=None, order=None):
    """Size-constrained label propagation (Sec. 3.1); returns labels.

    order: optional [rounds, n] visiting orders, one permutation per round,
    in place of the seeded random order (tests fix the random draws this
    way)."""
    lib = _load()
    rp, col = _i64(rp), _i32(col)
    n = len(rp) - 1
    labels = np.zeros(max(n, 1), dtype=np.int32)
    od = None
    if order is not None:
        od = _i32(order).reshape(-1, n)
        if od.shape[0] < rounds or any(sorted(r.tolist()) != list(range(n)) for r in od):
            raise ValueError("order must hold one permutation of the vertices per round")
    lib.orc_sclap(n, _p(rp), _p(col), _p(_f64(ew)), _p(_f64(c)), float(U), int(rounds),
                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(level), _p(od), _p(labels))
    return labels[:n]


def contract(rp, col, c, labels, ew=None):
    """Cluster contraction (Sec. 3.1).  Returns (map, c', rp', col', ew')."""
    lib = _load()
    rp, col = _i64(rp), _i32(col)
    n = len(rp) - 1
    nnz = int(rp[-1])
    labels = _i32(labels)
    mp = np.zeros(max(n, 1), dtype=np.int32)
    cc = np.zeros(max(n, 1), dtype=np.float64)
    crp = np.zeros(n + 1, dtype=np.int64)
    ccol = np.zeros(max(nnz, 1), dtype=np.int32)
    cew = np.zeros(max(nnz, 1), dtype=np.float64)
    cnnz = np.zeros(1, dtype=np.int64)
    nc = lib.orc_contract(n, _p(rp), _p(col), _p(_f64(ew)), _p(_f64(c)), _p(labels),
                          _p(mp), _p(cc), _p(crp), _p(ccol), _p(cew), _p(cnnz))
    m = int(cnnz[0])
    return mp[:n], cc[:nc], crp[:nc + 1].copy(), ccol[:m], cew[:m]


def prolong(mp, xc, cc, seed: int, level: int):
    """Random polar prolongation around the coarse representative (Sec. 3.2)."""
    lib = _load()
    mp = _i32(mp)
    xc = _f64(xc).reshape(-1, 2)
    xf = np.zeros((len(mp), 2), dtype=np.float64)
    lib.orc_prolong(len(mp), _p(mp), _p(xc), _p(_f64(cc)),
                    int(seed) & 0xFFFFFFFFFFFFFFFF, int(level), _p(xf))
    return xf


def place_coarsest(c, seed: int, level: int):
    lib = _load()
    c = _f64(c)
    x = np.zeros((len(c), 2), dtype=np.float64)
    lib.orc_place_coarsest(len(c), _p(c), int(seed) & 0xFFFFFFFFFFFFFFFF, int(level), _p(x))
    return x


# --------------------------------------------------------------------------
# orchestration (Sec. 3): hierarchy, initial layout, alpha schedule, layout
# --------------------------------------------------------------------------
DEFAULTS = dict(
    k=2, theta=0.5, exact_repulsion=0, coarsest_n=2, f=20.0, b=2.0, lp_rounds=10,
    iters_per_alpha=2, alpha0=1.0, alpha_factor=0.3, alpha_min=0.008, eps=1e-4,
    eps_final=1e-4, max_iters_at_min=100, early_exit=1, seed=1506, max_levels=64,
    max_stalls=10, approx_levels=0, exact_max_n=16384,
)


def params(**kw):
    p = dict(DEFAULTS)
    for key, v in kw.items():
        if key not in p:
            raise KeyError(key)
        p[key] = v
    return p


def build_hierarchy(rp, col, p, elen=None, log=None):
    """Coarsening (Sec. 3.1).  Level h is clustered by SCLaP with
    U = max(max c, W), W = min(b^(h+1), |V|/f) with |V| the input graph's
    vertex count (the unit of the node weights c, and their sum on every
    level); the contraction becomes level h+1.  A contraction that shrinks the graph by at most 10 percent sets
    f := 0.7 f.  One that merges nothing is discarded (f := 0.7 f, retried up
    to max_stalls times).  Coarsening stops at n <= coarsest_n.

    log: optional list; every clustering attempt appends
    (h, W, U, f, n, n_coarse, kept) with the values it used."""
    rp, col = _i64(rp), _i32(col)
    n = len(rp) - 1
    lv = dict(n=n, rp=rp, col=col, ew=np.ones(len(col)), c=np.ones(n),
              elen=None if elen is None else _f64(elen), coarse=False, map=None)
    levels = [lv]
    f = float(p["f"])
    stalls = 0
    while (levels[-1]["n"] > p["coarsest_n"] and len(levels) < p["max_levels"]
           and stalls < p["max_stalls"]):
        cur = levels[-1]
        h = len(levels) - 1
        W = min(p["b"] ** (h + 1), n / f)
        U = max(float(np.max(cur["c"])), W)
        labels = sclap(cur["rp"], cur["col"], cur["c"], U, p["lp_rounds"], p["seed"], h,
                       ew=cur["ew"])
        mp, cc, crp, ccol, cew = contract(cur["rp"], cur["col"], cur["c"], labels, ew=cur["ew"])
        nc = len(cc)
        kept = not (nc >= cur["n"] or nc < 2)
        if log is not None:
            log.append((h, W, U, f, cur["n"], nc, kept))
        if not kept:
            f *= 0.7
            stalls += 1
            continue
        stalls = 0
        if nc > 0.9 * cur["n"]:
            f *= 0.7
        cur["map"] = mp
        levels.append(dict(n=nc, rp=crp, col=ccol, ew=cew, c=cc, elen=None, coarse=True,
                           map=None))
    for L in levels:
        L["S"] = build_S(L["rp"], L["col"], p["k"], elen=L["elen"], c=L["c"],
                         coarse=L["coarse"])
    return levels


def relative_change(st):
    """|x^{l+1} - x^l| / |x^l| (Sec. 3.2), Euclidean over all coordinates."""
    if st[1] > 0:
        return math.sqrt(st[0]) / math.sqrt(st[1])
    return 0.0 if st[0] == 0 else math.inf


def alpha_rounds(p):
    """The alpha values of the schedule (Sec. 3.2 and Sec. 4 configuration):
    alpha0, then alpha := max(alpha_factor * alpha, alpha_min)."""
    a = float(p["alpha0"])
    out = [a]
    while a > p["alpha_min"]:
        a = max(a * p["alpha_factor"], p["alpha_min"])
        out.append(a)
    return out


def schedule(S, x, p, rep_mode: int, trace=None, start_at_min: bool = False, cmap=None):
    """Rounds of Jacobi iterations (Sec. 3.2): at most iters_per_alpha
    iterations per alpha, fewer if the relative change drops below eps; at
    alpha_min iterate until the relative change is below eps_final (capped at
    max_iters_at_min).  early_exit = 0 runs the caps exactly.  One schedule
    spans the whole multilevel run: it starts at alpha0 on the coarsest level,
    which ends only once alpha_min is reached and converged, so every finer
    level runs at alpha_min (start_at_min)."""
    x = _f64(x).reshape(-1, 2)
    sweeps = 0
    rounds = alpha_rounds(p)
    if start_at_min:
        rounds = rounds[-1:]
    for alpha in rounds:
        at_min = alpha <= p["alpha_min"]
        cap = p["max_iters_at_min"] if at_min else p["iters_per_alpha"]
        tol = p["eps_final"] if at_min else p["eps"]
        it = 0
        while True:
            x, st = sweep(x, S, alpha, rep_mode, p["theta"], cmap=cmap)
            rel = relative_change(st)
            it += 1
            sweeps += 1
            if trace is not None:
                trace.append((alpha, rel, st[2]))
            if (p["early_exit"] and rel < tol) or it >= cap:
                break
    return x, sweeps


def initial_layout(L, p, level_index):
    """Coarsest level (Sec. 3.1 'Initial Layout'): two vertices at their
    target distance; more than two are placed around the origin."""
    n = L["n"]
    if n == 1:
        return np.zeros((1, 2))
    if n == 2:
        sp, scol, sd, _ = L["S"]
        D = float(sd[0])
        return np.array([[-0.5 * D, 0.0], [0.5 * D, 0.0]])
    return place_coarsest(L["c"], p["seed"], level_index)


def approx_map(levels, level: int, h: int):
    """Map of level `level`'s vertices to the level used by Eq. 3: h levels
    down, or the coarsest level if there are fewer (Sec. 3.2)."""
    top = len(levels) - 1
    t = min(level + h, top)
    m = np.arange(levels[level]["n"], dtype=np.int64)
    for j in range(level, t):
        m = levels[j]["map"][m]
    return m.astype(np.int32)


def layout(rp, col, p, elen=None, x_init=None, levels=None, trace=None):
    """Multilevel maxent-stress layout (Sec. 3).  alpha is set to alpha0
    once, at the start (coarsest level), and reduced by rounds down to
    alpha_min; the finer levels refine at alpha_min.  With x_init the whole
    schedule runs on the finest level only, from x_init.  approx_levels = h
    > 0 takes the entropy sum of every level but the coarsest from Eq. 3
    (MulMent_h); the coarsest level always uses the exact sum.  Returns
    (x, info)."""
    if levels is None:
        levels = build_hierarchy(rp, col, p, elen=elen)
    top = len(levels) - 1
    happ = int(p["approx_levels"])

    def mode(level):
        if p["exact_repulsion"]:
            return 0, None
        if happ > 0 and level < top:
            return 2, approx_map(levels, level, happ)
        # levels of at most exact_max_n vertices take the exact sum
        if levels[level]["n"] <= p["exact_max_n"]:
            return 0, None
        return 1, None

    sweeps = []
    if x_init is not None:
        rm, cm = mode(0)
        x, s = schedule(levels[0]["S"], x_init, p, rm, trace, cmap=cm)
        return x, dict(levels=levels, sweeps=[s])
    x = initial_layout(levels[top], p, top)
    x, s = schedule(levels[top]["S"], x, p, 0, trace)
    sweeps.append(s)
    for h in range(top - 1, -1, -1):
        x = prolong(levels[h]["map"], x, levels[h + 1]["c"], p["seed"], h)
        rm, cm = mode(h)
        x, s = schedule(levels[h]["S"], x, p, rm, trace, start_at_min=True, cmap=cm)
        sweeps.append(s)
    return x, dict(levels=levels, sweeps=sweeps[::-1])
