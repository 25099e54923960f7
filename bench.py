#!/usr/bin/env python3
"""Benchmark of the GB300 MulMent layout (multilevel maxent-stress, Sec. 3).

One step = one full multilevel layout of the workload graph through
mm_layout (every level: prolongation + the alpha schedule of Eq. 2 sweeps,
each sweep = Barnes-Hut tree rebuild + walk + fused gather/update +
controller), with the hierarchy already built and resident in HBM.

  value  = vertex updates (sum over sweeps of the level size) per second
  e2e    = the same metric through the one-call host API mm_layout_host
           (host CSR in, host layout out: H2D copy, hierarchy build, layout,
           D2H copy all inside the timed region)

Default workload: Delaunay triangulation of 2^20 uniform points in the unit
square (the paper's del20 family; n = 1,048,576, m = 3,145,684), k = 1,
Barnes-Hut theta = 0.6, coarsening to <= 100 vertices; R-MAT scale 20 is
timed the same way as a second table (second_workloads).  L2 (129 MB) is
flushed by a 256 MB write before every timed step.

Beside the timed number, outside the timed region: the final objective
against the FP64 oracle's layout of the same graph (objective_vs_oracle: on
the oracle's own hierarchy and on the GPU's; M estimated the same way for
both), the exact O(n^2) objective against the oracle's sampled estimate, a
level-by-level breakdown of the layout time with time-weighted rooflines,
and the measured FP32 FMA peak used as the ALU roofline's denominator.

Multi-GPU (torchrun, N > 1): replicas only -- every rank lays out its own
copy; value = all ranks' vertex updates / max rank time.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (Barnes-Hut sweeps of the finest level).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "vertex-updates/s per sweep; time-to-layout at oracle-matched maxent-stress"
UNIT = "vertex-updates/s"

WORKLOADS = {
    "rgg100k": dict(kind="rgg", n=100000, deg=8.0, seed=1506, k=2, theta=0.5, coarsest_n=100,
                    desc="random geometric graph, 100k points in the unit square, mean degree 8, "
                         "largest component, k=2, Barnes-Hut theta=0.5, coarsen to <=100"),
    "grid32": dict(kind="grid", nx=32, ny=32, k=2, exact=1, single=100,
                   desc="32x32 grid, k=2, exact O(n^2) repulsion, uniform [0,1]^2 start, "
                        "100 Jacobi sweeps (single level)"),
    "rmat20": dict(kind="rmat", scale=20, ef=8, seed=1506, k=1, theta=0.6, coarsest_n=100,
                   desc="R-MAT scale 20 (a=0.57 b=c=0.19), 8 edge samples per vertex, largest "
                        "component, k=1, theta=0.6"),
    "del20": dict(kind="delaunay", n=1 << 20, seed=1506, k=1, theta=0.6, coarsest_n=100,
                  also=("rmat20",),
                  desc="Delaunay triangulation of 2^20 uniform points (the paper's del20 "
                       "family), k=1, Barnes-Hut theta=0.6, coarsen to <=100"),
    "learned2m": dict(kind="rgg", n=2000000, deg=8.0, seed=2027, k=2, theta=0.5, coarsest_n=100,
                      learned=True,
                      desc="learned prolongation: network trained on coarse-to-converged pairs of "
                           "random geometric graphs of 10k-200k vertices, evaluated on an unseen "
                           "2M-vertex random geometric graph (mean degree 8), k=2, theta=0.5; "
                           "timed at the smallest per-level sweep cap whose objective matches "
                           "the plain layout's"),
    "del16h": dict(kind="delaunay", n=1 << 16, seed=1506, k=1, theta=0.5, coarsest_n=2,
                   approx=10, hsweep=(0, 1, 2, 3, 5, 7, 10), nolearn=True,
                   desc="MulMent_h (Eq. 3): Delaunay triangulation of 2^16 uniform points, k=1, "
                        "coarsen to 2, entropy sum from the level h=10 below; table over "
                        "h = 0 (exact), 1, 2, 3, 5, 7, 10 as in the paper's del16 h table"),
    "dyn16": dict(kind="delaunay", n=1 << 16, seed=1506, k=1, theta=0.5, coarsest_n=2,
                  approx=7, dynamic=(5.0, 16), nolearn=True,
                  dyn_table=((1.0, 2), (1.0, 16), (5.0, 2), (5.0, 16)), dyn_h=(0, 7),
                  desc="dynamic update (Sec. 4.3): Delaunay 2^16, k=1; G laid out from scratch "
                       "(MulMent_7), 5% of its non-tree edges replaced by edges to vertices at "
                       "distance <= 16; the timed step lays out the perturbed graph from G's "
                       "layout at alpha = 0.008 on the finest level of a hierarchy cut after "
                       "h = 7 levels (MulMent_7); table over x in {1, 5}%, D in {2, 16}, "
                       "h in {0, 7} against the scratch layout"),
    "batch512": dict(kind="batch", count=512, seed=1506, k=2, theta=0.5, coarsest_n=2,
                     desc="512 graphs, lognormal sizes (median 3000, sigma 1) in [200, 50000], "
                          "thirds grids / random geometric (mean degree 6-12) / random trees, "
                          "k=2, theta=0.5, one batched layout"),
}


def make_graph(w):
    from paper_1506_04383_gb300 import graphs
    if w["kind"] == "rgg":
        rp, col, _, _ = graphs.rgg(w["n"], w["deg"], w["seed"])
    elif w["kind"] == "grid":
        rp, col = graphs.grid(w["nx"], w["ny"])
    elif w["kind"] == "rmat":
        rp, col = graphs.rmat(w["scale"], w["ef"], w["seed"])
    elif w["kind"] == "batch":
        sizes = graphs.batch_sizes(w["count"], w["seed"])
        gs = [graphs.batch_graph(i, sz, w["seed"]) for i, sz in enumerate(sizes)]
        rp, col, gp = graphs.concat_graphs(gs)
        return rp, col, gp, gs
    else:
        rp, col, _ = graphs.delaunay(w["n"], w["seed"])
    return rp, col


# training set of the learned prolongation: random geometric graphs (mean
# degree 8) of these sizes and seeds, none of them a bench workload
TRAIN_RGG = [(10000, 9001), (20000, 9002), (50000, 9003), (100000, 9004), (200000, 9005)]
CAPS = [5, 10, 20, 30, 50, 100]


def train_prolongation(mm, p, steps=2000, lr=3e-3):
    """Trains the learned prolongation on the method's own pairs; returns
    (net, summary)."""
    import numpy as np
    import torch
    from paper_1506_04383_gb300 import graphs, learned
    t0 = time.perf_counter()
    pairs = []
    for n_, sd in TRAIN_RGG:
        rp, col, _, _ = graphs.rgg(n_, 8.0, sd)
        hh = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p)
        pairs += learned.level_pairs(hh, p)
    t1 = time.perf_counter()
    net = mm.Net(learned.init_params(1))
    losses = learned.train(net, pairs, steps, lr=lr, seed=0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"train_graphs": [n_ for n_, _ in TRAIN_RGG], "pairs": len(pairs),
                 "steps": steps, "pairs_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2),
                 "loss_first100": float(np.mean(losses[:100])),
                 "loss_last100": float(np.mean(losses[-100:]))}


def timed_layout(mm, h, p, reps=2):
    """Median device time (ms) of mm_layout after one warm-up, L2 flushed."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    x, st = mm.layout(h, p)
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        x, st = mm.layout(h, p)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts), st, x


def learned_vs_plain(mm, h, p, net, tol=0.01):
    """Time to an equal objective: the plain layout at the default per-level
    sweep cap sets the reference objective M_ref (Eq. 1 at alpha_min); both
    the plain and the learned prolongation then take the smallest cap in
    CAPS whose objective is within tol of M_ref (or better; the tolerance the
    oracle parity of layouts uses).  Returns (summary, params of the
    matching learned run)."""
    ms_ref, st_ref, x = timed_layout(mm, h, p)
    M_ref = mm.objective(h, 0, x, p.alpha_min)[2]
    bound = M_ref + tol * abs(M_ref)
    out = {"reference": {"cap": p.max_iters_at_min, "ms": round(ms_ref, 2),
                         "sweeps": st_ref["total_sweeps"], "M": M_ref},
           "tolerance": tol}
    best = {}
    for name in ("plain", "learned"):
        rows = []
        for cap in CAPS:
            q = mm.default_params()
            ctypes_copy(q, p)
            q.max_iters_at_min = cap
            if name == "learned":
                q.learned_prolong = 1
                mm.set_net(h, net)
            ms, st, x = timed_layout(mm, h, q)
            M = mm.objective(h, 0, x, q.alpha_min)[2]
            mm.set_net(h, None)
            rows.append({"cap": cap, "ms": round(ms, 2), "sweeps": st["total_sweeps"], "M": M})
            if M <= bound:
                best[name] = (q, rows[-1])
                break
        out[name] = rows
    if len(best) == 2:
        out["speedup_at_equal_objective"] = best["plain"][1]["ms"] / best["learned"][1]["ms"]
        out["sweep_ratio_at_equal_objective"] = (best["plain"][1]["sweeps"] /
                                                 best["learned"][1]["sweeps"])
    return out, best.get("learned", (None,))[0]


def params_of(mm, w):
    kw = dict(k=w["k"])
    if w.get("single"):
        kw.update(exact_repulsion=w.get("exact", 0), early_exit=0,
                  max_iters_at_min=w["single"] - 10)
    else:
        kw.update(theta=w["theta"], coarsest_n=w["coarsest_n"])
    if w.get("approx"):
        kw.update(approx_levels=w["approx"])
    return kw


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [t.strip() for t in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class OracleSweeps:
    """The FP64 oracle as it stands, prepared once for the finest level of a
    workload: Barnes-Hut, exact or Eq. 3 sweeps of Eq. 2 on the host cores."""

    def __init__(self, w, rp, col):
        import oracle
        from paper_1506_04383_gb300 import graphs
        self.oracle = oracle
        self.n = len(rp) - 1
        self.S = oracle.build_S(rp, col, w["k"])
        self.x = graphs.uniform_positions(self.n, 1506, 0.0, math.sqrt(self.n))
        exact = bool(w.get("exact"))
        self.theta = w.get("theta", 0.5)
        self.mode, self.cmap = (0 if exact else 1), None
        self.what = "exact" if exact else "Barnes-Hut theta=%g" % self.theta
        if w.get("approx"):
            # the oracle's own coarsening supplies the map to the level h below
            po = oracle.params(k=w["k"], coarsest_n=w["coarsest_n"],
                               approx_levels=w["approx"])
            levels = oracle.build_hierarchy(rp, col, po)
            self.mode, self.cmap = 2, oracle.approx_map(levels, 0, w["approx"])
            self.what = f"Eq. 3 (h={w['approx']}, {int(self.cmap.max()) + 1} representatives)"

    def run(self, sweeps=None, budget_s=None):
        """Runs `sweeps` sweeps (or until budget_s elapsed); returns
        (sweeps, seconds)."""
        done, t0 = 0, time.perf_counter()
        while True:
            self.x, _ = self.oracle.sweep(self.x, self.S, 0.3, self.mode, self.theta,
                                          cmap=self.cmap)
            done += 1
            el = time.perf_counter() - t0
            if (sweeps and done >= sweeps) or (budget_s and el >= budget_s):
                return done, el

    def sample(self, sweeps):
        return (f"{sweeps} {self.what} Eq. 2 sweeps of the finest level (n={self.n}, "
                f"|S|={len(self.S[1])}), FP64 oracle, OpenMP")


def cpu_baseline(w, rp, col, budget_s=15.0):
    """The oracle's throughput on the host cores over a bounded sample (after
    a short warm-up).  Returns (vertex-updates/s, cores, sample, seconds)."""
    o = OracleSweeps(w, rp, col)
    o.run(budget_s=min(1.0, budget_s / 10))
    sweeps, el = o.run(budget_s=budget_s)
    return o.n * sweeps / el, o.oracle.num_threads(), o.sample(sweeps), el


def run_reference(args, w, rank, world):
    """The reference arm: the oracle, prepared once; every step is the same
    number of sweeps (calibrated in the warm-up to about 0.5 s of work)."""
    if rank != 0:
        return 0
    rp, col = make_graph(w)
    o = OracleSweeps(w, rp, col)
    done, el = o.run(budget_s=0.5)
    per_step = max(1, int(done * 0.5 / max(el, 1e-9)))
    for _ in range(args.warmup):
        o.run(sweeps=per_step)
    times = [o.run(sweeps=per_step)[1] for _ in range(args.steps)]
    value = o.n * per_step * args.steps / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": w["desc"], "n": o.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.oracle.num_threads(),
                             "kind": "oracle", "sample": "per step: " + o.sample(per_step)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def job_time_and_value(local_ms, vu_per_step, steps, world, device):
    """Replicas: the job's time is the slowest rank's timed region (max over
    ranks), and its value is every rank's vertex updates over that time."""
    total = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total, world * vu_per_step * steps / (total / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="del20", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--learned", type=int, default=1,
                    help="also train the learned prolongation and compare it with the plain "
                         "layout at equal objective (single-graph multilevel workloads)")
    ap.add_argument("--batch-compare", type=int, default=64,
                    help="graphs of the batch also laid out one by one for comparison")
    ap.add_argument("--extras", type=int, default=1,
                    help="0: skip the oracle comparison, the second workloads and the "
                         "level-by-level breakdown (a shorter run, e.g. for a launch list)")
    ap.add_argument("--profile-level", type=int, default=-1,
                    help="profiling aid (e.g. under ncu): build the workload's hierarchy, run "
                         "one profiled sweep (mm_sweep_profile, 2 repetitions) of this level "
                         "from uniform positions of the layout's scale, print its stage times "
                         "and exit")
    ap.add_argument("--profile-gemm", type=int, default=0,
                    help="profiling aid: one launch each of the learned prolongation's two "
                         "tensor-core kernels on this many vertices (after a warm-up), then exit")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, w, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1506_04383_gb300 import build as _build, mm
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    mm.load()

    def barrier():
        if world > 1:
            dist.barrier()

    if args.profile_gemm > 0:
        f_ms, b_ms = mm.net_gemm_profile(args.profile_gemm, reps=1)
        print(json.dumps({"profile_gemm": args.profile_gemm, "layer_product_ms": f_ms,
                          "weight_gradient_ms": b_ms}), flush=True)
        return 0
    made = make_graph(w)
    rp, col = made[0], made[1]
    if args.profile_level >= 0:
        from paper_1506_04383_gb300 import graphs
        hp = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(),
                                mm.default_params(**params_of(mm, w)))
        lv = min(args.profile_level, hp.levels() - 1)
        nl = hp.level_info(lv)[0]
        xl = torch.from_numpy(graphs.uniform_positions(nl, 7, 0.0, math.sqrt(nl))
                              .astype(np.float32)).cuda()
        pr = mm.sweep_profile(hp, lv, xl, reps=2)
        print(json.dumps({"profile_level": lv, "n": nl, "stage_ms": dict(zip(
            pr["stage_names"], pr["stage_ms"])), "visits": pr["visits"],
            "interactions": pr["interactions"], "nnz_S": pr["nnz_S"]}), flush=True)
        return 0
    gp = made[2] if len(made) > 2 else None
    n = len(rp) - 1
    kw = params_of(mm, w)
    p = mm.default_params(**kw)
    x_init = None
    dyn = None
    if w.get("dynamic"):
        # the update algorithm: G laid out from scratch, then the perturbed
        # graph from G's layout on a hierarchy cut after h levels
        rpG, colG = rp, col
        hG = mm.build_hierarchy(torch.from_numpy(rpG).cuda(), torch.from_numpy(colG).cuda(), p)
        xG, _ = mm.layout(hG, p)
        del hG
        pct, D = w["dynamic"]
        rp, col = perturbed(rpG, colG, pct, D, w["seed"])
        kw = dict(kw, max_levels=w["approx"] + 1, alpha0=0.008)
        p = mm.default_params(**kw)
        x_init = xG
        args.e2e_steps = 0  # the host API lays out from scratch, not from a layout
        dyn = dyn_table(mm, rpG, colG, w)
    drp = torch.from_numpy(rp).cuda()
    dcol = torch.from_numpy(col).cuda()
    if w.get("single"):
        from paper_1506_04383_gb300 import graphs
        x_init = torch.from_numpy(graphs.uniform_positions(n, 1506).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h = mm.build_hierarchy(drp, dcol, p, graph_ptr=gp)
    e1.record()
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    tune = None
    if args.autotune:
        tune = mm.autotune(h, max_rel_drift=0.01)
    learned_cmp = None
    if w.get("learned") or (args.learned and gp is None and not w.get("single")
                            and not w.get("nolearn")):
        net, tr = train_prolongation(mm, p)
        cmp_, best = learned_vs_plain(mm, h, p, net)
        learned_cmp = {"training": tr, **cmp_,
                       "tensor_core_rooflines": mpnn_roofline(mm, n, measured_peaks()[0])}
        if w.get("learned"):
            if best is None:
                best = mm.default_params()
                ctypes_copy(best, p)
                best.learned_prolong = 1
            mm.set_net(h, net)
            p = best
        else:
            mm.set_net(h, None)
    xbuf = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 0)):
        _, st = mm.layout(h, p, x_init=x_init, x_out=xbuf)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stats = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        for a, b in evs:
            flush.fill_(1)
            a.record()
            _, st = mm.layout(h, p, x_init=x_init, x_out=xbuf)
            b.record()
            stats.append(st)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    vu = stats[-1]["vertex_updates"]
    total_ms, value = job_time_and_value(sum(step_ms), vu, args.steps, world, "cuda")
    launches = sum(s["kernel_launches"] for s in stats)

    # quality: objective of the final layout (Eq. 1 at alpha = 0.008)
    M = None if gp is not None else mm.objective(h, 0, xbuf, 0.008)[2]
    batch_cmp = None
    if gp is not None:
        batch_cmp = compare_batch(mm, made[3], p, args.batch_compare)

    # warm hierarchy builds (the first build above also pays for the
    # stream-ordered pool's growth and first-touch costs)
    builds = []
    for _ in range(3 if gp is None else 1):
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        hw = mm.build_hierarchy(drp, dcol, p, graph_ptr=gp)
        b1.record()
        torch.cuda.synchronize()
        builds.append(b0.elapsed_time(b1))
        del hw
    build_warm_ms = statistics.median(builds)

    # roofline of the dominant kernel on the finest level, live with events;
    # the ALU peak is this device's measured FP32 FMA rate
    peaks, src = measured_peaks()
    clk_sum = clk.summary()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_tf, fp32_ms = mm.measure_fp32_peak(20)
    fp32 = (fp32_tf, f"measured FP32 FMA peak of this device ({sms} SMs): {fp32_tf:.2f} TFLOP/s "
                     f"(mm_measure_fp32_peak, {fp32_ms:.2f} ms per launch)")
    breakdown = None
    if w.get("approx"):
        roof = roofline_h(mm, h, xbuf, int(w["approx"]), peaks, src, clk_sum, fp32=fp32)
    elif gp is None:
        prof = mm.sweep_profile(h, 0, xbuf, reps=10)
        roof = roofline(prof, peaks, src, clk_sum, n, exact=bool(w.get("exact")),
                        workload=args.workload, fp32=fp32)
        if not w.get("single") and args.extras:
            breakdown = layout_breakdown(mm, h, p, stats[-1], peaks, src, fp32_tf)
    else:
        big = int(np.argmax(np.diff(gp)))
        grp, gcol = made[3][big]
        hb = mm.build_hierarchy(torch.from_numpy(grp).cuda(), torch.from_numpy(gcol).cuda(),
                                mm.default_params(**dict(kw, seed=int(kw.get("seed", 1506)))))
        xb, _ = mm.layout(hb)
        prof = mm.sweep_profile(hb, 0, xb, reps=10)
        roof = roofline(prof, peaks, src, clk_sum, len(grp) - 1, fp32=fp32)
        roof["graph"] = f"largest graph of the batch (n={len(grp) - 1})"
    roof["sms"] = sms

    # end to end through the host API (pinned host buffers)
    e2e = None
    if args.e2e_steps > 0:
        prp = torch.from_numpy(rp).pin_memory().numpy()
        pcol = torch.from_numpy(col).pin_memory().numpy()
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if w.get("learned"):
                xh, sth = layout_host_learned(mm, prp, pcol, p, h._net)
            elif gp is None:
                xh, sth = mm.layout_host(prp, pcol, p)
            else:
                xh, sth = layout_host_batch(mm, prp, pcol, gp, p)
            t1 = time.perf_counter()
            if i > 0:
                times.append(t1 - t0)
        e2e = {"value": sth["vertex_updates"] / statistics.mean(times), "unit": UNIT,
               "h2d_bytes_per_step": int(prp.nbytes + pcol.nbytes),
               "d2h_bytes_per_step": int(xh.nbytes),
               "time_to_layout_s": statistics.mean(times)}

    htab = h_table(mm, drp, dcol, w, kw) if w.get("hsweep") else None

    # the final objective against the oracle's layout of the same graph
    ovo = None
    if (args.extras and rank == 0 and gp is None and not w.get("dynamic")
            and not w.get("learned")):
        t0 = time.perf_counter()
        Mb = mm.objective_bh(h, 0, xbuf, 0.008, float(kw.get("theta", 0.5)))[2]
        mbh = (Mb, (time.perf_counter() - t0) * 1e3)
        ovo = objective_vs_oracle(mm, args.workload, rp, col, kw, xbuf, M, mbh)
    # the other workloads of the same configuration family
    sides = ([side_table(mm, o) for o in w.get("also", ())]
             if rank == 0 and args.extras else [])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample, el = cpu_baseline(w, rp, col, budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": round(el, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "n": n,
                       "m": int(len(col) // 2), "levels": stats[-1]["num_levels"],
                       "level_n": stats[-1]["level_n"],
                       "sweeps": stats[-1]["total_sweeps"],
                       "level_sweeps": stats[-1]["level_sweeps"],
                       "level_rel_change": [round(v, 6) for v in stats[-1]["level_rel_change"]],
                       "max_iters_at_min": int(p.max_iters_at_min), "eps_final": p.eps_final,
                       "vertex_updates_per_step": vu, "l2": "flushed (256 MB write) before "
                       "every timed step", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "time_to_layout_s": (build_warm_ms + statistics.mean(step_ms)) / 1e3,
            "hierarchy_build_ms": build_warm_ms,
            "hierarchy_build_cold_ms": build_ms,
            "objective_M": M,
            "objective_vs_oracle": ovo,
            "second_workloads": sides or None,
            "layout_breakdown": breakdown,
            "batch_vs_plain": batch_cmp,
            "learned_vs_plain": learned_cmp,
            "h_table": htab,
            "dynamic_table": dyn,
            "autotune": tune,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk_sum,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def layout_host_batch(mm, rp, col, gp, p):
    """End to end for a batch: host CSR in, hierarchy build, batched layout,
    host layout out (the batch needs graph_ptr, which the one-call host API
    does not take)."""
    import numpy as np
    import torch
    drp = torch.from_numpy(rp).cuda(non_blocking=True)
    dcol = torch.from_numpy(col).cuda(non_blocking=True)
    h = mm.build_hierarchy(drp, dcol, p, graph_ptr=gp)
    x, st = mm.layout(h, p)
    return x.cpu().numpy(), st


def layout_host_learned(mm, rp, col, p, net):
    """End to end with the learned prolongation: host CSR in, hierarchy
    build, network attached, layout, host layout out."""
    import torch
    drp = torch.from_numpy(rp).cuda(non_blocking=True)
    dcol = torch.from_numpy(col).cuda(non_blocking=True)
    h = mm.build_hierarchy(drp, dcol, p)
    mm.set_net(h, net)
    x, st = mm.layout(h, p)
    return x.cpu().numpy(), st


def compare_batch(mm, gs, p, count):
    """The first `count` graphs laid out one by one (plain per-graph
    mm_layout, hierarchy prebuilt) against the same graphs as one batch."""
    import numpy as np
    import torch
    from paper_1506_04383_gb300 import graphs
    count = min(count, len(gs))
    sub = gs[:count]
    hs = []
    for i, (rp, col) in enumerate(sub):
        pi = mm.default_params()
        ctypes_copy(pi, p)
        pi.seed = p.seed + i
        hs.append((mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(),
                                      pi), pi))
    rp, col, gp = graphs.concat_graphs(sub)
    hb = mm.build_hierarchy(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), p,
                            graph_ptr=gp)
    for h, pi in hs:
        mm.layout(h, pi)
    xb, _ = mm.layout(hb, p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, pi in hs:
        mm.layout(h, pi)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    xb, _ = mm.layout(hb, p)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    return {"graphs": count, "plain_sequential_ms": t_plain * 1e3,
            "batched_ms": t_batch * 1e3, "speedup": t_plain / t_batch}


def ctypes_copy(dst, src):
    import ctypes
    ctypes.memmove(ctypes.addressof(dst), ctypes.addressof(src), ctypes.sizeof(src))


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one
# ncu capture of the kernel on level 0 of the workload, with the source file
# of the kernel and its SHA-256 prefix at capture time: reported only while
# that source is unchanged (null otherwise).
NCU_TRAFFIC = {
    # profiles/gather_light_del20.md (the walk's capture in
    # profiles/traverse_dyn_kernel_del20.md predates its current records)
    ("del20", "gather"): (77.58e6, "paper_1506_04383_gb300/csrc/k_sweep.cu", "195d1391b37d2281"),
}


def ncu_traffic(workload, kernel):
    e = NCU_TRAFFIC.get((workload, kernel))
    if not e:
        return None
    nbytes, rel, sha = e
    return nbytes if _src_sha(rel) == sha else None


def h_table(mm, drp, dcol, w, kw, reps=2):
    """Layouts with the entropy sum of Eq. 3 from h levels below (h = 0: the
    exact sum on every level), the shape of the paper's h table on del16:
    time per layout (CUDA events, L2 flushed), sweeps and M (Eq. 1 at
    alpha = 0.008, exact), F (full stress over all pairs, hop distances) and
    the stress-minimising scale s with F(s x) (Sec. 4, methodology)."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for hh in w["hsweep"]:
        kh = dict(kw, approx_levels=hh)
        if hh == 0:
            kh.update(exact_repulsion=1)
        p = mm.default_params(**kh)
        h = mm.build_hierarchy(drp, dcol, p)
        x, st = mm.layout(h, p)
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            x, st = mm.layout(h, p)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        F, s, Fs, _ = mm.full_stress(h, x)
        rows.append({"h": hh, "ms": round(min(ts), 3), "sweeps": st["total_sweeps"],
                     "levels": st["num_levels"], "M": mm.objective(h, 0, x, 0.008)[2],
                     "F": F, "s": s, "F_scaled": Fs})
        del h
    return rows


_PERTURBED = {}


def perturbed(rp, col, pct, D, seed):
    """graphs.perturb_edges, computed once per (x, D, seed) in a run."""
    from paper_1506_04383_gb300 import graphs
    key = (len(rp), pct, D, seed)
    if key not in _PERTURBED:
        _PERTURBED[key] = graphs.perturb_edges(rp, col, pct, D, seed)
    return _PERTURBED[key]


def dyn_table(mm, rpG, colG, w, reps=2):
    """Update vs scratch layouts of perturbed graphs (Sec. 4.3): for every
    (x %, D) the perturbed graph Q is laid out from scratch with MulMent_h and
    updated from the scratch layout of G (alpha = 0.008, finest level of a
    hierarchy cut after h levels; h = 0: one level, exact sum).  Times are
    CUDA events with L2 flushed (min of reps), M is Eq. 1 at alpha = 0.008, F
    the full stress over all pairs at the stress-minimising scale (Sec. 4)."""
    import torch
    from paper_1506_04383_gb300 import graphs
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(h, p, x0=None):
        x, st = mm.layout(h, p, x_init=x0)
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            x, st = mm.layout(h, p, x_init=x0)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts), st, x

    base = dict(k=w["k"], coarsest_n=w["coarsest_n"])
    pert = {(pct, D): perturbed(rpG, colG, pct, D, w["seed"]) for pct, D in w["dyn_table"]}
    rows = []
    for hh in w["dyn_h"]:
        ks = dict(base, approx_levels=hh, exact_repulsion=1 if hh == 0 else 0)
        ps = mm.default_params(**ks)
        hG = mm.build_hierarchy(torch.from_numpy(rpG).cuda(), torch.from_numpy(colG).cuda(), ps)
        xG, _ = mm.layout(hG, ps)
        del hG
        for pct, D in w["dyn_table"]:
            rq, cq = pert[(pct, D)]
            drq, dcq = torch.from_numpy(rq).cuda(), torch.from_numpy(cq).cuda()
            hs = mm.build_hierarchy(drq, dcq, ps)
            t_s, st_s, x_s = timed(hs, ps)
            M_s = mm.objective(hs, 0, x_s, 0.008)[2]
            pu = mm.default_params(**dict(ks, max_levels=hh + 1, alpha0=0.008))
            hu = mm.build_hierarchy(drq, dcq, pu)
            t_u, st_u, x_u = timed(hu, pu, xG)
            M_u = mm.objective(hs, 0, x_u, 0.008)[2]
            F_s = mm.full_stress(hs, x_s)[2]   # at the stress-minimising scale
            F_u = mm.full_stress(hs, x_u)[2]
            rows.append({"x_pct": pct, "D": D, "h": hh, "scratch_ms": round(t_s, 3),
                         "update_ms": round(t_u, 3), "speedup": round(t_s / t_u, 2),
                         "scratch_sweeps": st_s["total_sweeps"],
                         "update_sweeps": st_u["total_sweeps"], "M_scratch": M_s,
                         "M_update": M_u, "F_scratch": F_s, "F_update": F_u})
            del hs, hu
    return rows


def roofline_h(mm, h, x, hh, peaks, src, clk, reps=10, fp32=None):
    """The Eq. 3 sums on the finest level (mm_repulsion_h: midpoints, then one
    thread per vertex over all other representatives and its own group):
    FP32-ALU bound, 10 FP32 ops per pair term, n (n' - 1) far terms plus
    sum_c m_c (m_c - 1) near terms for groups of sizes m_c."""
    import numpy as np
    import torch
    n = h.level_info(0)[0]
    top = h.levels() - 1
    # composed map of level 0 (sizes of the groups)
    m = np.arange(n)
    for j in range(0, min(hh, top)):
        m = mm.level_export(h, j)["map"].cpu().numpy()[m]
    sizes = np.bincount(m)
    nt = len(sizes)
    terms = n * (nt - 1) + float((sizes * (sizes - 1)).sum())
    mm.repulsion_h(h, 0, x)
    evs = []
    for _ in range(reps):
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        mm.repulsion_h(h, 0, x)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / reps
    peak, note = fp32
    ach = 10.0 * terms / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "peak_source": "measured", "kernel": "approx_force",
            "note": f"{note}; {nt} representatives, "
                    f"{terms:.4g} pair terms per call, {ms * 1e3:.1f} us per call"}


def roofline(prof, peaks, src, clk, n, exact=False, workload=None, fp32=None):
    """Dominant kernel of a finest-level sweep against its roofline.

    traverse (Barnes-Hut walk): ALU bound; algorithmic work = 10 FP32 ops per
    lane interaction (accepted cell or leaf point), peak = 152 SMs x 128 FP32
    lanes x 2 (FMA) x SM clock.  With exact repulsion the same stage is the
    all-pairs sum: n (n - 1) interactions of 10 FP32 ops.  gather: HBM bound; algorithmic bytes per
    vertex = 4 (row_ptr) + 8 (x_u) + 8 (x'_u) + 8 (F_u) + 4 (rho_u) + 8 per S
    entry (col, d); neighbour positions are L2 hits and not counted.
    sort: HBM bound; 4 look-back passes x (8 B read + 8 B write) per element.
    """
    st = prof["stage_ms"]
    names = prof["stage_names"]
    dom = max(range(len(st)), key=lambda i: st[i])
    alu_peak, alu_note = fp32
    hbm = peaks.get("hbm_gbs", 6800.0)
    nnzS = prof["nnz_S"]
    kern = {}
    t_trav = max(st[names.index("traverse")], 1e-9) / 1e3
    flops = 10.0 * (n * (n - 1) if exact else prof["interactions"])
    kern["traverse"] = {"bound": "alu", "achieved": flops / t_trav / 1e12, "peak": alu_peak,
                        "unit": "TFLOP/s", "traffic": None, "note": alu_note}
    t_g = st[names.index("gather")] / 1e3
    gbytes = n * 32.0 + nnzS * 8.0
    kern["gather"] = {"bound": "hbm", "achieved": gbytes / t_g / 1e9, "peak": hbm, "unit": "GB/s",
                      "traffic": None}
    t_s = st[names.index("sort")] / 1e3
    sbytes = 3 * 16.0 * n  # three 8-bit passes over 24-bit keys (group walk)
    kern["sort"] = {"bound": "hbm", "achieved": sbytes / t_s / 1e9, "peak": hbm, "unit": "GB/s",
                    "traffic": None}
    for name_, v in kern.items():
        v["frac"] = v["achieved"] / v["peak"]
        v["peak_source"] = "measured" if v["bound"] == "alu" else src
        v["traffic"] = ncu_traffic(workload, name_)
    name = names[dom]
    out = dict(kern.get(name, kern["traverse"]))
    out["kernel"] = name if name in kern else "traverse"
    out["stage_ms"] = dict(zip(names, st))
    out["others"] = {k: {kk: vv for kk, vv in v.items() if kk in ("achieved", "peak", "unit",
                                                                   "frac", "bound", "traffic")}
                     for k, v in kern.items() if k != out["kernel"]}
    return out


def oracle_golden():
    path = os.path.join(ROOT, "tests", "golden", "oracle_layouts.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def objective_vs_oracle(mm, wname, rp, col, kw, x_own, M_exact, M_bh=None):
    """Final maxent-stress (Eq. 1 at alpha = 0.008) of the GPU's layouts
    against the FP64 oracle's layout of the same graph (Sec. 3 algorithm on
    the oracle's own hierarchy, stored by tests/golden/make_oracle_layouts.py).
    Every M here is the oracle's estimator: exact stress over S, ln-sum over
    the pairs outside S from the same 2e7 random pairs (common pairs, so the
    gaps carry far less noise than either standard error).
      same_hierarchy: the oracle's coarsening fed to the GPU, GPU layout;
      own_hierarchy: the GPU's own coarsening (the timed layout);
      exact_vs_sampled: the GPU's exact O(n^2) M of the timed layout against
        the sampled estimate of the same layout, in standard errors."""
    import numpy as np
    import torch

    import oracle
    g = oracle_golden().get(wname)
    if g is None:
        return None
    t0 = time.perf_counter()
    po = oracle.params(**g["params"])
    levels = oracle.build_hierarchy(rp, col, po)
    if [int(L["n"]) for L in levels] != g["level_n"]:
        return {"error": "the oracle's hierarchy differs from the stored one",
                "level_n": [int(L["n"]) for L in levels], "stored_level_n": g["level_n"]}
    dev = []
    for L in levels:
        d = dict(row_ptr=torch.from_numpy(L["rp"]).cuda(), col=torch.from_numpy(L["col"]).cuda(),
                 omega=torch.from_numpy(L["ew"].astype(np.float32)).cuda(),
                 c=torch.from_numpy(L["c"].astype(np.float32)).cuda())
        if L["map"] is not None:
            d["map"] = torch.from_numpy(L["map"]).cuda()
        dev.append(d)
    hs = mm.build_hierarchy_levels(dev, mm.default_params(**kw))
    xs, sts = mm.layout(hs)
    S = levels[0]["S"]

    def est(x):
        return oracle.objective_sampled(x.cpu().numpy().astype(np.float64), S, 0.008,
                                        samples=g["samples"], seed=g["sample_seed"])
    e_same, e_own = est(xs), est(x_own)
    Mo = g["M"]
    out = {
        "estimator": f"exact stress over S + ln-sum over {g['samples']:.0e} random pairs "
                     f"(seed {g['sample_seed']}), alpha = 0.008",
        "oracle_M": Mo, "oracle_se_M": g["se_M"], "oracle_level_sweeps": g["level_sweeps"],
        "same_hierarchy": {"M": e_same["M"], "rel_gap": (e_same["M"] - Mo) / abs(Mo),
                           "level_sweeps": sts["level_sweeps"],
                           "within_1pct": abs(e_same["M"] - Mo) <= 0.01 * abs(Mo)},
        "own_hierarchy": {"M": e_own["M"], "rel_gap": (e_own["M"] - Mo) / abs(Mo),
                          "within_1pct": abs(e_own["M"] - Mo) <= 0.01 * abs(Mo)},
        "seconds": None,
    }
    if M_exact is not None:
        out["exact_vs_sampled"] = {"M_exact_gpu": M_exact, "M_sampled": e_own["M"],
                                   "se_M": e_own["se_M"],
                                   "z": (M_exact - e_own["M"]) / max(e_own["se_M"], 1e-300)}
    if M_bh is not None:
        out["barnes_hut_estimate"] = {"theta": kw.get("theta", 0.5), "M_bh_gpu": M_bh[0],
                                      "rel_to_exact": (M_bh[0] - M_exact) / abs(M_exact)
                                      if M_exact else None, "ms": M_bh[1]}
    out["seconds"] = round(time.perf_counter() - t0, 2)
    return out


def layout_breakdown(mm, h, p, stats, peaks, src, fp32_peak, reps=5):
    """Where a layout's time goes, level by level: mm_sweep_profile stage
    times of every multi-kernel level (from that level's own final layout)
    times its sweep count; fused levels (one launch each) are the remainder
    of the measured layout time.  Per kernel class the time-weighted share
    and, for the walk, the gather and the sort, their achieved rate summed
    over all levels against the roofline (same algorithmic work per unit as
    the finest-level roofline)."""
    xs = mm.layout_levels(h, p)
    hbm = peaks.get("hbm_gbs", 6800.0)
    cls = {"walk": 0.0, "sort+keys": 0.0, "tree": 0.0, "gather": 0.0, "other": 0.0}
    work = {"walk_flops": 0.0, "gather_bytes": 0.0, "sort_bytes": 0.0}
    rows = []
    for l in range(stats["num_levels"]):
        n, sw = stats["level_n"][l], stats["level_sweeps"][l]
        if n <= 2048 or sw == 0:
            rows.append({"level": l, "n": n, "sweeps": sw, "fused": True})
            continue
        pr = mm.sweep_profile(h, l, xs[l], reps=reps)
        st = dict(zip(pr["stage_names"], pr["stage_ms"]))
        cls["walk"] += sw * st["traverse"]
        cls["sort+keys"] += sw * (st["morton_hist"] + st["sort"])
        cls["tree"] += sw * (st["radix_tree_scan"] + st["records"])
        cls["gather"] += sw * st["gather"]
        cls["other"] += sw * (st["bbox"] + st["controller"])
        work["walk_flops"] += sw * 10.0 * pr["interactions"]
        work["gather_bytes"] += sw * (32.0 * n + 8.0 * pr["nnz_S"])
        work["sort_bytes"] += sw * 4 * 16.0 * n
        rows.append({"level": l, "n": n, "sweeps": sw, "ms_per_sweep": round(sum(st.values()), 4),
                     "walk_ms": round(st["traverse"], 4), "gather_ms": round(st["gather"], 4),
                     "sort_ms": round(st["morton_hist"] + st["sort"], 4),
                     "interactions_per_vertex": round(pr["interactions"] / n, 1)})
    tot = sum(cls.values())
    out = {"levels": rows, "class_ms": {k: round(v, 3) for k, v in cls.items()},
           "class_share_of_multikernel_time": {k: round(v / tot, 4) for k, v in cls.items()}
           if tot > 0 else None,
           "note": "stage times from one-by-one profiled sweeps (events between stages); "
                   "inside the layout's CUDA graph the same kernels run back to back"}
    if cls["walk"] > 0:
        a = work["walk_flops"] / (cls["walk"] / 1e3) / 1e12
        out["walk_roofline"] = {"bound": "alu", "achieved": a, "peak": fp32_peak,
                                "unit": "TFLOP/s", "frac": a / fp32_peak, "peak_source": "measured"}
    if cls["gather"] > 0:
        a = work["gather_bytes"] / (cls["gather"] / 1e3) / 1e9
        out["gather_roofline"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                                  "frac": a / hbm, "peak_source": src}
    if cls["sort+keys"] > 0:
        a = work["sort_bytes"] / (cls["sort+keys"] / 1e3) / 1e9
        out["sort_roofline"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                                "frac": a / hbm, "peak_source": src}
    return out


def mpnn_roofline(mm, n, peaks):
    """The learned prolongation's two tensor-core kernels at the width of a
    hidden layer on this workload's n vertices (mm_net_gemm_profile, CUDA
    events): the layer product H W^T ([n x 128] x [128 x 64], BF16 out) and
    the weight-gradient partials Hcat^T dZ ([n x 128]^T x [n x 64], FP32
    partials).  Both do 2 n 128 64 flops; their algorithmic bytes are the
    BF16 operands read once and the output written once.  Tensor fraction
    against the measured BF16 GEMM rate (burst), HBM fraction against the
    measured copy bandwidth."""
    f_ms, b_ms = mm.net_gemm_profile(n, reps=20)
    flops = 2.0 * n * 128 * 64
    bf16 = peaks.get("bf16_tflops", 1900.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    parts = min(torch_sms(), max(1, (n + 63) // 64))
    out = {}
    for name, ms, nbytes in (("layer_product", f_ms, 2.0 * n * (128 + 64) + 2.0 * 64 * 128),
                             ("weight_gradient", b_ms, 2.0 * n * (128 + 64)
                              + 4.0 * parts * 128 * 64)):
        tf = flops / (ms / 1e3) / 1e12
        gb = nbytes / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "tflops": tf, "tensor_frac": tf / bf16, "gbs": gb,
                     "hbm_frac": gb / hbm, "n": n, "bound": "hbm"}
    out["peaks"] = {"bf16_tflops": bf16, "hbm_gbs": hbm, "source": "MEASURED_PEAKS.json"}
    return out


def torch_sms():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def side_table(mm, wname):
    """A second workload timed the same way as the headline (inputs resident,
    L2 flushed, CUDA events): layout time, vertex-updates/s, warm hierarchy
    build and time to layout."""
    import torch
    w = WORKLOADS[wname]
    rp, col = make_graph(w)[:2]
    kw = params_of(mm, w)
    p = mm.default_params(**kw)
    drp, dcol = torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()
    h = mm.build_hierarchy(drp, dcol, p)
    builds = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = mm.build_hierarchy(drp, dcol, p)
        torch.cuda.synchronize()
        builds.append((time.perf_counter() - t0) * 1e3)
        del hh
    x, st = mm.layout(h, p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    for _ in range(5):
        flush.fill_(1)
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        x, st = mm.layout(h, p, x_out=x)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    lay = statistics.median(ms)
    bms = statistics.median(builds)
    return {"workload": wname, "desc": w["desc"], "n": len(rp) - 1, "m": int(len(col) // 2),
            "levels": st["num_levels"], "level_n": st["level_n"],
            "level_sweeps": st["level_sweeps"],
            "level_rel_change": [round(v, 6) for v in st["level_rel_change"]],
            "layout_ms": lay, "value": st["vertex_updates"] / (lay / 1e3), "unit": UNIT,
            "hierarchy_build_ms": bms, "time_to_layout_s": (bms + lay) / 1e3}


# Source files whose kernels the stored ncu DRAM figures describe, with the
# SHA-256 prefix of the file when the capture was taken: a figure is reported
# only while its kernel's source is unchanged.
def _src_sha(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
