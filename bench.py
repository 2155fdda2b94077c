"""Benchmark of the data-driven (DD) hot path on GB300.

A step is one DD iteration z_{i+1} = P_D(P_C(z_i)) of a running solve
(assembly of E and S, FP64 CG for both systems, recovery, nearest-data
projection of every material point, convergence statistics) through the
library's C ABI.  `value` = material-point searches per second over the
timed steps (whole job, all ranks).  Under torchrun every rank runs an
independent replica (the search does not shard).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--mode tc|tc_topk|fp32|ann|knng|serve]

The default workload is the 32^3 cube with 4 load cases on 10^9 points with
the approximate tree search; the workloads are listed in dd_inputs.WORKLOADS
(the mode follows from the name unless given).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dd_inputs as I  # noqa: E402

METRIC = "DD searches/s & solve time at N=1e9 (ANN vs exact); p50/p99 serve latency"
UNIT = "searches/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
L2_BYTES = 129 * 2 ** 20

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the search's
# kernels, from one-kernel ncu captures of a smaller case of the same mode
# (profiles/dram_search_cube32_N3e7.md), keyed by the sha256 of the kernels'
# source file (a changed source reports null until it is captured again).
# The captured bytes split into the distinct data points the search read
# (48 B each) and a per-query part; a bench run scales the per-query part by
# its own query count and adds its own distinct points' bytes (a floor of the
# data part).
TRAFFIC = {
    # mode: ((source file under the package's csrc/, sha256), ...), DRAM bytes
    #        per search, distinct data bytes per search, queries per search
    "ann": ((("ann.cu", "b215ecd4527cb4aa091bd5db4d12157189d5e0570ca1156428f73788cf452cd5"),
             ("near_tc.cu", "7f925e5f2a22e2a025fadf2e822dc2bd4ed3b94324d0de05e0876f0e7fc0d7f4")),
            239.86e6, 307232 * 48.0, 262144),
}


# Captures of exactly the benched launch: (workload, mode): (source, sha256,
# DRAM bytes per launch); profiles/k_scan_tc_cube16_N1e6.md.
TRAFFIC_EXACT = {
    ("cube16_N1e6_exact", "tc"): ("search_tc.cu", "88f6e8471c848cf2a664b288412b49176e7e9d072215266d4cd5fdf669e3d7a7", 78.45e6),
}


def exact_traffic(workload: str, mode: str):
    t = TRAFFIC_EXACT.get((workload, mode))
    if t is None:
        return None
    path, sha, byts = t
    with open(os.path.join(ROOT, "paper_2012_00357_gb300", "csrc", path), "rb") as f:
        return byts if hashlib.sha256(f.read()).hexdigest() == sha else None


def captured_traffic(mode: str, queries_now: float, distinct_bytes_now: float):
    t = TRAFFIC.get(mode)
    if t is None:
        return None
    sources, byts, distinct, queries = t
    for path, sha in sources:
        with open(os.path.join(ROOT, "paper_2012_00357_gb300", "csrc", path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != sha:
                return None
    return (byts - distinct) / queries * queries_now + distinct_bytes_now


def load_peaks():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained"), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle's brute-force P_D on a bounded query sample
# ----------------------------------------------------------------------------
def oracle_searches_per_s(W: I.Workload, C, target_s: float = 12.0, max_queries: int = 4096,
                          max_points: int = 2_000_000):
    """Brute-force cost is linear in N: above max_points the oracle scans the
    first max_points points and the rate is scaled by max_points / N."""
    from oracle import metric, nn
    t0 = time.time()
    n_pts = min(W.N, max_points)
    data = I.make_dataset(n_pts, W.law, seed=W.seed)
    if C is None:       # the data-derived metric (Sec. 3.1) of the sample
        C = metric.pca_metric(data.astype(np.float64))
    Z = metric.to_z(data, C)
    gen_s = time.time() - t0
    y = I.make_states(max_queries, W.law, seed=99, spread=0.05)
    zq = metric.to_z(y, C)
    t = time.perf_counter()
    nn.nn_top2(Z, zq[:16])
    dt = time.perf_counter() - t
    rate = 16 / max(dt, 1e-9)
    n = int(min(max_queries, max(16, rate * target_s)))
    t = time.perf_counter()
    nn.nn_top2(Z, zq[:n])
    dt = time.perf_counter() - t
    scale = n_pts / W.N
    what = (f"{n} query states x all {W.N} data points" if n_pts == W.N else
            f"{n} query states x the first {n_pts} of {W.N} data points, rate scaled by {n_pts}/{W.N} "
            f"(extrapolated, brute force is linear in N)")
    return {"value": n / dt * scale, "unit": UNIT, "cores": nn.threads(), "kind": "oracle",
            "sample": f"{what}, brute-force FP64 scan (oracle/nn.c); data generation {gen_s:.1f}s not timed"}


def oracle_dd_iterations(W: I.Workload, C, target_s: float = 12.0):
    """The oracle's DD solve itself (Eq. 8: direct P_C, brute-force P_D over
    all N points) from the workload's initial association, iterated until it
    converges or target_s has passed: searches/s over whole DD iterations
    (for data sets the oracle scans in seconds)."""
    from oracle import dd as odd
    from oracle import nn
    data = I.make_dataset(W.N, W.law, seed=W.seed)
    load = I.load_case(*W.loads[0])
    t0 = time.perf_counter()
    prob = odd.DDProblem(data, C, W.n_el, load)
    setup_s = time.perf_counter() - t0
    idx = I.initial_association(W.m, W.N, seed=W.seed)
    t = time.perf_counter()
    it, converged = 0, False
    while True:
        u, eta, eps, sig = prob.project_C(idx)
        new, _, _ = prob.project_D(eps, sig)
        it += 1
        converged = bool(np.array_equal(new, idx))
        idx = new
        if converged or time.perf_counter() - t > target_s:
            break
    dt = time.perf_counter() - t
    return {"value": W.m * it / dt, "unit": UNIT, "cores": nn.threads(), "kind": "oracle",
            "sample": f"{it} full DD iterations of the oracle (direct P_C, brute-force FP64 P_D of all {W.m} "
                      f"material points over all {W.N} data points) from the random association"
                      f"{', converged' if converged else ''}; factorisation {setup_s:.1f}s not timed"}


# ----------------------------------------------------------------------------
def make_workload(name: str):
    W = I.WORKLOADS[name]
    return W


def run_ours(args, world, rank, local):
    import torch

    import paper_2012_00357_gb300 as P

    P.build()
    torch.cuda.set_device(local)
    W = make_workload(args.workload)
    C = I.isotropic_C(W.law.E, W.law.nu)
    mode = {"tc": P.DD_SEARCH_EXACT_TC, "tc_topk": P.DD_SEARCH_EXACT_TC, "fp32": P.DD_SEARCH_EXACT_FP32,
            "ann": P.DD_SEARCH_ANN, "knng": P.DD_SEARCH_KNNG}[args.mode]
    approx = mode in (P.DD_SEARCH_ANN, P.DD_SEARCH_KNNG)
    nlist = 0
    if approx:
        nlist = args.nlist or max(64, 1 << int(np.log2(max(W.N // 3000, 64))))
    certify = args.mode != "tc_topk"
    ctx = P.dd_create(local)
    raw = torch.empty((W.N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, W.law, C, seed=W.seed)
    t_build = time.perf_counter()
    if W.extra.get("metric") == "pca":
        C = P.dd_pca_metric(ctx, raw)          # the data-derived metric of Sec. 3.1
    levels = args.ann_levels or (2 if W.N >= 300_000_000 or mode == P.DD_SEARCH_KNNG else 1)
    if approx and levels == 2 and not args.nlist:
        # 2^24 asks for the finest tree the search handles, 4096 cells of 512
        # leaves (about 480 points per leaf at 10^9 points)
        nlist = 1 << 24 if W.N >= 300_000_000 else 1 << 17
    knn = dict(knn_k=args.knn_k, knn_fd=args.knn_fd) if mode == P.DD_SEARCH_KNNG else {}
    # the approximate modes also get the FP16 operands when the check below
    # times the certified tensor-core exact search on the same data set
    exact_tc = approx and (args.ann_check > 0 or args.exact_solve) and args.exact_tc
    ds = P.dd_load_dataset(ctx, raw, C, borrow=True, build_fp16=(mode == P.DD_SEARCH_EXACT_TC or exact_tc),
                           ann_nlist=nlist,
                           seed=1, ann_levels=levels, ann_alu=args.ann_alu, **knn)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t_build
    load = I.load_case(*W.loads[0])
    init = I.initial_association(W.m, W.N, seed=W.seed)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    data_bytes = W.N * (64 if mode == P.DD_SEARCH_EXACT_TC else 52 if mode == P.DD_SEARCH_EXACT_FP32 else 48)
    ann_kw = dict(f_d0=args.fd0, f_d_final=args.fd_final, ramp_iters=args.ramp_iters,
                  ann_budget=args.ann_budget, eq14=args.eq14) if mode == P.DD_SEARCH_ANN else {}
    if mode == P.DD_SEARCH_KNNG:
        ann_kw = dict(f_s=args.f_s)
    flush_l2 = data_bytes < 2 * L2_BYTES

    loads = [I.load_case(*lc) for lc in W.loads]
    nload = len(loads)

    def new_solver(k=0, kw=None):
        return P.dd_solver_create(ds, ctx, W.n_el, loads[k], mode=mode, certify=certify, init_idx=init,
                                  max_iter=100000, **(ann_kw if kw is None else kw))

    svs = [new_solver(k) for k in range(nload)]

    def step(svs=svs, kw=None):
        """One iteration of every load case (one batched call when there are several)."""
        for k in range(nload):
            if P.dd_solver_done(svs[k]):
                P.dd_solver_free(svs[k])
                svs[k] = new_solver(k, kw)
        if nload == 1:
            return [P.dd_solver_step(svs[0], ctx)]
        return P.dd_solvers_step(svs, ctx)

    for _ in range(args.warmup):
        step()

    barrier(world)
    torch.cuda.synchronize()
    step_ms, scan_ms, infos = [], [], []
    launches0 = P.dd_launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            if flush_l2:
                flush.fill_(1.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            info = step()[0]                     # synchronous; batched phases are shared
            step_ms.append((time.perf_counter() - t) * 1e3)
            scan_ms.append(info.scan_ms)
            infos.append(info)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    launches = P.dd_launch_count(ctx) - launches0

    # device time of the steps: the library brackets each step's kernels with
    # CUDA events on the stream it launches them on
    dev_ms = [i.cg_ms + i.other_ms + i.search_ms for i in infos]
    total_ms = sum(dev_ms)
    total_ms = max_over_ranks(total_ms, world)
    searches = W.m * nload * args.steps * world
    value = searches / (total_ms / 1e3)

    # the other Eq. (14) rule over the same iteration window (fresh solves,
    # the same warm-up and timed steps), reported beside the headline
    eq14_other = None
    if mode == P.DD_SEARCH_ANN and not args.no_eq14_compare:
        kw2 = dict(ann_kw, eq14=1 - args.eq14)
        svs2 = [new_solver(k, kw2) for k in range(nload)]
        for _ in range(args.warmup):
            step(svs2, kw2)
        infos2 = []
        for _ in range(args.steps):
            if flush_l2:
                flush.fill_(1.0)
            infos2.append(step(svs2, kw2)[0])
        for sv in svs2:
            P.dd_solver_free(sv)
        ms2 = sum(i.cg_ms + i.other_ms + i.search_ms for i in infos2)
        eq14_other = {"eq14": "certified second bound" if kw2["eq14"] == 0 else "second-closest point found",
                      "value": W.m * nload * args.steps / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2 / args.steps,
                      "scan_ms_per_step": statistics.mean(i.scan_ms for i in infos2),
                      "skipped": sum(i.skipped for i in infos2)}

    # full solve from the random association (all load cases together,
    # outside the timed steps) through the public call, host arrays in and
    # out: the end-to-end figure (wall clock, initial association copied in
    # from pinned memory, the solutions read back)
    init_pin = torch.from_numpy(init).pin_memory().numpy()
    torch.cuda.synchronize()
    t = time.perf_counter()
    if nload == 1:
        rs = [P.dd_solve(ds, ctx, W.n_el, loads[0], mode=mode, certify=certify, init_idx=init_pin, max_iter=200,
                         **ann_kw)]
    else:
        rs = P.dd_solve_batch(ds, ctx, [W.n_el] * nload, loads, mode=mode, certify=certify, init_idx=init_pin,
                              max_iter=200, **ann_kw)
    solve_s = max_over_ranks(time.perf_counter() - t, world)
    solve_iters = sum(rr.iters for rr in rs)
    solve_h2d = nload * W.m * 4
    solve_d2h = sum(rr.u.nbytes + rr.eta.nbytes + rr.eps.nbytes + rr.sig.nbytes + rr.idx.nbytes
                    + rr.iters * 32 for rr in rs)
    r = rs[0]
    accuracy = None
    if approx and args.ann_check > 0:
        # agreement of the approximate answers with the certified exact search
        # on a sample of the final states (tensor-core scan, or the FP32 scan,
        # + FP64 rescoring), and the exact search's rate on that sample
        ys = np.concatenate([np.concatenate([rr.eps, rr.sig], axis=1) for rr in rs])
        pick = np.random.default_rng(0).choice(len(ys), min(args.ann_check, len(ys)), replace=False)
        ysel = np.ascontiguousarray(ys[pick])
        prev = np.ascontiguousarray(np.concatenate([rr.idx for rr in rs])[pick])
        ia = np.empty(len(pick), np.int32)
        da = np.empty(len(pick))
        ie = np.empty(len(pick), np.int32)
        de = np.empty(len(pick))
        P.dd_project_nearest(ds, ctx, ysel, ia, da, mode=mode, f_d=args.fd_final, prev_idx=prev, f_s=args.f_s,
                             ann_budget=args.ann_budget)
        exact_mode = P.DD_SEARCH_EXACT_TC if exact_tc else P.DD_SEARCH_EXACT_FP32
        P.dd_project_nearest(ds, ctx, ysel[:256], ie[:256], de[:256], mode=exact_mode)   # tunes, warms up
        torch.cuda.synchronize()
        t_ex = time.perf_counter()
        st_ex = P.dd_project_nearest(ds, ctx, ysel, ie, de, mode=exact_mode)
        t_ex = time.perf_counter() - t_ex
        accuracy = {"sample": int(len(pick)), "same_index": float(np.mean(ia == ie)),
                    "mean_rel_distance_excess": float(np.mean((da - de) / np.maximum(de, 1e-300))),
                    **({"f_d": args.fd_final} if mode == P.DD_SEARCH_ANN else {"f_s": args.f_s, "k": args.knn_k}),
                    "exact": "tensor-core split-FP16 scan, certified" if exact_tc else "FP32 scan, certified",
                    "exact_searches_per_s": len(pick) / t_ex, "exact_uncertified": int(st_ex.uncertified)}

    # the metric's "solve time at N (ANN vs exact)": the first load case
    # solved by the approximate search and by the certified exact search
    # (tensor-core scan, FP64 rescoring; the few queries it cannot certify go
    # through the certified FP32 scan before any FP64 scan) from the same
    # random association, and, with --exact-start both, the exact iteration
    # started from the approximate solve's final association as well, which
    # descends to the exact fixed point next to it.  Opt-in: minutes.
    exact_solve = None
    if approx and args.exact_solve and exact_tc:
        torch.cuda.synchronize()
        t = time.perf_counter()
        ra1 = P.dd_solve(ds, ctx, W.n_el, loads[0], mode=mode, certify=certify, init_idx=init_pin, max_iter=200,
                         **ann_kw)
        ta1 = time.perf_counter() - t
        da1 = float(ra1.d2_pd[-1])

        def exact_run(start, init_idx):
            # stepwise, so that every iteration is logged (stderr) and a
            # wall-clock budget can end it
            sv = P.dd_solver_create(ds, ctx, W.n_el, loads[0], mode=P.DD_SEARCH_EXACT_TC, certify=True,
                                    init_idx=init_idx, max_iter=200)
            t0 = time.perf_counter()
            hist = []
            while not P.dd_solver_done(sv):
                info = P.dd_solver_step(sv, ctx)
                hist.append({"iter": info.iter, "d2_pd": info.d2_pd, "changed": int(info.changed),
                             "uncertified": int(info.uncertified), "search_ms": info.search_ms,
                             "cg_ms": info.cg_ms, "t_s": time.perf_counter() - t0})
                print(json.dumps({"exact_solve_iteration": {"start": start, **hist[-1]}}), file=sys.stderr,
                      flush=True)
                if hist[-1]["t_s"] > args.exact_budget_s:
                    break
            tx = time.perf_counter() - t0
            done = bool(P.dd_solver_done(sv))
            P.dd_solver_free(sv)
            dx = hist[-1]["d2_pd"]
            return {"start": start, "exact_solve_s": tx, "exact_iters": len(hist), "exact_converged": done,
                    "exact_d2": dx, "exact_changed_last": hist[-1]["changed"],
                    "exact_uncertified": sum(h["uncertified"] for h in hist),
                    "exact_searches_per_s": W.m * len(hist) / (sum(h["search_ms"] for h in hist) / 1e3),
                    "ann_rel_d2_vs_exact": (da1 - dx) / dx, "speedup": tx / ta1, "history": hist}

        runs = []
        if args.exact_start in ("random", "both"):
            runs.append(exact_run("the random association of the approximate solve", init_pin))
        if args.exact_start in ("ann", "both"):
            runs.append(exact_run("the approximate solve's final association", np.ascontiguousarray(ra1.idx)))
        exact_solve = {"load": W.loads[0][0], "exact": "tensor-core split-FP16 scan + FP64 rescoring, certified",
                       "exact_budget_s": args.exact_budget_s, "ann_solve_s": ta1, "ann_iters": ra1.iters,
                       "ann_d2": da1, "runs": runs}

    # end-to-end through the public API with host buffers (pinned): one
    # projection of the step's m states per call, copies inside the timed region
    m_e2e = W.m * nload
    y = torch.from_numpy(I.make_states(m_e2e, W.law, seed=7, spread=0.05)).pin_memory()
    idx_h = torch.empty(m_e2e, dtype=torch.int32).pin_memory()
    d2_h = torch.empty(m_e2e, dtype=torch.float64).pin_memory()
    e2e_kw = dict(mode=mode, certify=certify, f_d=args.fd_final, f_s=args.f_s, ann_budget=args.ann_budget)
    P.dd_project_nearest(ds, ctx, y.numpy(), idx_h.numpy(), d2_h.numpy(), **e2e_kw)
    reps = max(3, args.steps)
    t = time.perf_counter()
    for _ in range(reps):
        P.dd_project_nearest(ds, ctx, y.numpy(), idx_h.numpy(), d2_h.numpy(), **e2e_kw)
    e2e_s = max_over_ranks((time.perf_counter() - t) / reps, world)

    peaks = load_peaks()
    kc = 3 if (mode == P.DD_SEARCH_EXACT_TC and certify) else 1
    scan_avg = statistics.mean(scan_ms)
    clk_sum = clk.summary()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = clk_sum.get("sm_mhz") or 1920.0
    # FP32 lane operations per second of the device (one FFMA or FADD per
    # lane per clock), from its SM count and the clock sampled while timing
    alu_peak = n_sm * 128 * clk_mhz * 1e6
    alu_src = f"{n_sm} SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz (median SM clock sampled while timing)"
    if mode == P.DD_SEARCH_ANN:
        # The search is bound by SM work, not by HBM: per step it evaluates
        # ~10^4 distances per query, most of them on leaves that L1/L2 serve.
        # FP32 lane operations: 12 per distance to a data point (the 12 FMA
        # of the leaf-frame expanded form of the leaf-major scan; the in-warp
        # probe's direct form takes 24, so this undercounts its share), 24 per
        # leaf-centroid distance (12 differences, 12 FMA), and, when the cells
        # are ranked on the ALU, 12 per coarse-cell distance; ranked on the
        # tensor cores (the default) those are MMA work and are not counted.
        # The survey's HBM figure (48 B per probed point) and the measured
        # DRAM traffic are reported beside it.
        nq = W.m * nload
        Lr = P.dd_dataset_ann_cells(ds, ctx)[1].shape[0] if levels == 2 else nlist
        points = statistics.mean(i.points for i in infos)
        dists = statistics.mean(i.distances for i in infos)
        cells = statistics.mean((nq - i.skipped) * Lr for i in infos)
        leafc = max(0.0, dists - points - cells)
        tc_rank = not args.ann_alu and 16 <= Lr <= 4096
        lane_ops = 12 * points + 24 * leafc + (0 if tc_rank else 12 * cells)
        achieved = lane_ops / (scan_avg / 1e3)
        byts = points * 48 + nq * 48
        traffic = captured_traffic(args.mode, nq, statistics.mean(i.unique_points for i in infos) * 48)
        rank_k = "k_near_tc<0>" if tc_rank else "k_rank_small"
        roof = {"kernel": (f"k_ann_gate + {rank_k} + k_ann_probe2 + k_leaf_scan (one search per step)"
                           if levels == 2 else "k_ann_probe + centroid ranking (one search per step)"),
                "bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12, "unit": "T FP32 lane-ops/s",
                "frac": achieved / alu_peak, "traffic": traffic, "peak_source": alu_src,
                "algorithmic": ("12 lane-ops per point distance + 24 per leaf-centroid distance, per search (the "
                                "step's one launch sequence); the coarse-cell distances run on the tensor cores"
                                if tc_rank else
                                "12 lane-ops per point distance + 24 per leaf-centroid distance + 12 per coarse-cell "
                                "distance, per search (the step's one launch sequence)"),
                "lane_ops_direct_form": 24 * (points + leafc),
                "lane_ops": lane_ops, "distances": {"points": points, "leaf_centroids": leafc, "cells": cells},
                "hbm": {"algorithmic_bytes": byts,
                        "algorithmic": "48 B x points of the clusters each non-skipped query probed + 48 B x "
                                       "queries (most served by L1/L2, so not an HBM rate)",
                        "algorithmic_gbs": byts / (scan_avg / 1e3) / 1e9,
                        "dram_gbs": None if traffic is None else traffic / (scan_avg / 1e3) / 1e9,
                        "dram_frac": None if traffic is None else traffic / (scan_avg / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "peak": peaks["hbm_gbs"], "peak_source": f"{peaks['source']} copy bandwidth",
                        "distinct_gbs": (statistics.mean(i.unique_points for i in infos) * 48 + nq * 48 + nlist * 52)
                                        / (scan_avg / 1e3) / 1e9}}
    elif mode == P.DD_SEARCH_KNNG:
        # greedy walks: every evaluated neighbour costs its 4 B index and its
        # 48 B row, every query its 48 B record
        evals = statistics.mean(i.points for i in infos)
        byts = evals * 52 + W.m * nload * 48
        achieved = byts / (scan_avg / 1e3) / 1e9
        roof = {"kernel": "k_knng_walk", "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_source": f"{peaks['source']} copy bandwidth",
                "algorithmic": "52 B x neighbours evaluated + 48 B x queries, per launch", "algorithmic_bytes": byts}
    elif mode == P.DD_SEARCH_EXACT_TC:
        # method work: one K = 16 product per (query, point) distance; the
        # split-FP16 form issues three of them (reported beside it)
        long_scan = scan_avg > 100.0
        peak = peaks["bf16_tflops_sustained"] if long_scan and peaks.get("bf16_tflops_sustained") else peaks["bf16_tflops"]
        flops = 2.0 * W.m * nload * W.N * 16
        achieved = flops / (scan_avg / 1e3) / 1e12
        roof = {"kernel": f"k_scan_tc<{kc}>", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": exact_traffic(W.name, args.mode), "peak_source":
                    f"{peaks['source']} bf16 dense {'sustained' if long_scan else 'burst'} (fp16 runs at the same rate)",
                "algorithmic": "2*m*N*16 flops per launch (one K = 16 product per distance)",
                "issued_tflops": achieved * kc, "issued": f"{kc} FP16 products per distance (split-FP16 operands)"
                if kc == 3 else "1 FP16 product per distance"}
    else:
        # FP32 CUDA-core scan: 12 FFMA per (query, point) on the expanded form
        flops = 2.0 * 12 * W.m * nload * W.N
        achieved = flops / (scan_avg / 1e3) / 1e12
        peak_tflops = 2 * alu_peak / 1e12
        roof = {"kernel": "k_scan_fp32", "bound": "alu", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": None,
                "peak_source": alu_src + ", 2 flop per FFMA",
                "algorithmic": "2*12*m*N flops per launch (12 FFMA per pair)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (P_C, rescoring) + " + ("fp16 split, f32 accum" if kc == 3 and mode == 1
                                                                    else "fp16, f32 accum" if mode == 1 else "f32"),
        "data": "synthetic (dd_inputs generator, made on device)",
        "config": {"workload": W.name, "mesh": f"{W.n_el}^3 hex, 2x2x2 Gauss", "material_points": W.m * nload,
                   "data_points": W.N, "law": W.law.kind, "metric": W.extra.get("metric", "isotropic C of the law"),
                   "load": W.loads[0][0], "search": args.mode,
                   "l2": "flushed before every step" if flush_l2 else "inputs larger than L2",
                   "parallelism": f"replicas x{world}",
                   **({"f_d": f"{args.fd0} -> {args.fd_final} over {args.ramp_iters} iterations",
                       "leaves": P.dd_dataset_ann_nlist(ds), "ann_levels": levels,
                       "eq14": "certified second bound" if args.eq14 == 0 else "second-closest point found"}
                      if mode == P.DD_SEARCH_ANN else {}),
                   **({"knn_k": args.knn_k, "knn_fd": args.knn_fd, "f_s": args.f_s, "nlist": nlist}
                      if mode == P.DD_SEARCH_KNNG else {})},
        "roofline": roof,
        "e2e": {"value": W.m * solve_iters * world / solve_s, "unit": UNIT,
                "h2d_bytes_per_step": solve_h2d / max(1, max(rr.iters for rr in rs)),
                "d2h_bytes_per_step": solve_d2h / max(1, max(rr.iters for rr in rs)),
                "what": (f"dd_solve_batch of the {nload} load case(s) from the random initial association, wall "
                         f"clock: {solve_iters} DD iterations x {W.m} searches in {solve_s:.3f} s, initial "
                         f"association in from pinned memory ({solve_h2d} B), solutions read back ({solve_d2h} B); "
                         f"bytes per step = per solve / its iterations"),
                "projection": {"value": m_e2e * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": m_e2e * 96,
                               "d2h_bytes_per_step": m_e2e * 12,
                               "what": "dd_project_nearest of fresh states (no warm start) with pinned host "
                                       "buffers (states in, indices + distances out)"}},
        "gpu_launches": launches,
        "clocks": clk_sum,
        "detail": {
            "device_ms_per_step": statistics.mean(dev_ms), "scan_ms_per_step": scan_avg,
            "cg_ms_per_step": statistics.mean(i.cg_ms for i in infos),
            "search_ms_per_step": statistics.mean(i.search_ms for i in infos),
            "cg_iters": [i.cg_iters for i in infos][:8], "uncertified": sum(i.uncertified for i in infos),
            "dd_iterations_per_s": args.steps * world / (total_ms / 1e3), "wall_s": wall,
            "wall_ms_per_step": statistics.mean(step_ms),
            "solve_s": solve_s, "solve_iters": r.iters, "solve_converged": r.converged,
            "solve_search_ms": r.search_ms, "solve_cg_ms": r.cg_ms, "solve_d2": float(r.d2_pd[-1]),
            "index_build_s": build_s, "nlist": nlist, "ann_levels": levels, "ann_vs_exact": accuracy,
            "centroid_passes": ("ALU" if args.ann_alu else "tensor cores, answers equal to the ALU kernels'"),
            "index_build_fallback_rows": P.dd_dataset_ann_build_fallback(ds) if approx else 0,
            "load_cases": [lc[0] for lc in W.loads],
            "solve_d2_all": [float(rr.d2_pd[-1]) for rr in rs], "solve_iters_all": [rr.iters for rr in rs],
            "skipped": sum(getattr(i, "skipped", 0) for i in infos),
            "distances_per_query": statistics.mean(i.distances for i in infos) / (W.m * nload),
            "points_per_query": statistics.mean(i.points for i in infos) / (W.m * nload),
            "distinct_points_per_step": statistics.mean(i.unique_points for i in infos),
            "walk_moves_per_query": statistics.mean(i.moves for i in infos) / (W.m * nload),
            "solve_at_N_ann_vs_exact": exact_solve,
            "eq14_other_rule": eq14_other,
        },
    }
    for sv in svs:
        P.dd_solver_free(sv)
    P.dd_free_dataset(ds)
    del raw
    torch.cuda.empty_cache()
    if args.serve_requests > 0 and W.name != "serve_N1e7":
        # the metric's p50/p99 serve latency: a short run of the serving
        # configuration (resident 10^7-point data set, Poisson arrivals)
        line["detail"]["serve"] = serve_leg(P, ctx, I.WORKLOADS["serve_N1e7"], args, args.serve_requests)
    P.dd_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        # whole oracle DD iterations where it scans the data set in seconds,
        # else its brute-force P_D on a bounded query sample
        line["cpu_baseline"] = (oracle_dd_iterations(W, C, target_s=args.cpu_seconds) if W.N <= 2_000_000
                                else oracle_searches_per_s(W, C, target_s=args.cpu_seconds))
    return line


def serve_leg(P, ctx, W, args, n_req, clk=None):
    """Serving (BASELINE's serving configuration): one resident data set,
    Poisson arrivals at 0.8 x the service rate measured by a closed-loop
    burst, admission by a device-memory budget, continuous batching.
    Returns the figures of the measured stream."""
    import threading as th

    import torch

    C = I.isotropic_C(W.law.E, W.law.nu)
    ex = W.extra
    raw = torch.empty((W.N, 12), dtype=torch.float32, device="cuda")
    P.dd_synth_dataset(ctx, raw, W.law, C, seed=W.seed)
    nlist = args.nlist or max(64, 1 << int(np.log2(max(W.N // 3000, 64))))
    ds = P.dd_load_dataset(ctx, raw, C, borrow=True, ann_nlist=nlist, seed=1)
    kw = dict(mode=P.DD_SEARCH_ANN, f_d0=args.fd0, f_d_final=args.fd_final, ramp_iters=args.ramp_iters, max_iter=200,
              eq14=args.eq14)

    def serve(reqs, budget):
        srv = P.dd_server_start(ds, ctx, state_budget=budget, max_batch=args.max_batch, **kw)
        tickets, lat, iters, m_tot = [None] * len(reqs), [None] * len(reqs), [0] * len(reqs), [0] * len(reqs)
        t0 = time.perf_counter()

        def submitter():
            for r, (edge, load, at, seed) in enumerate(reqs):
                dt = t0 + at - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[r] = P.dd_server_submit(srv, edge, load, seed=seed)

        th_sub = th.Thread(target=submitter)
        th_sub.start()
        for r in range(len(reqs)):
            while tickets[r] is None:
                time.sleep(0.0005)
            res, lat[r] = P.dd_server_poll(srv, ctx, tickets[r], timeout_s=600.0)
            iters[r], m_tot[r] = res.iters, res.n_gp
        th_sub.join()
        makespan = time.perf_counter() - t0
        st = P.dd_server_get_stats(srv)
        P.dd_server_stop(srv)
        return lat, iters, m_tot, makespan, st

    budget = int(args.serve_budget_gb * 2 ** 30)
    # calibration: a closed-loop burst gives the service rate
    burst = [(e, L, 0.0, s) for (e, L, _, s) in I.serve_requests(W.seed + 1, 48, ex["edge_min"], ex["edge_max"],
                                                                 ex["t_min"], ex["t_max"], 1.0)]
    _, _, _, mk, _ = serve(burst, budget)
    rate = 0.8 * len(burst) / mk
    reqs = I.serve_requests(W.seed, n_req, ex["edge_min"], ex["edge_max"], ex["t_min"], ex["t_max"], rate)
    if clk is not None:
        with clk:
            lat, iters, m_tot, makespan, st = serve(reqs, budget)
    else:
        lat, iters, m_tot, makespan, st = serve(reqs, budget)
    P.dd_free_dataset(ds)
    del raw
    lat_s = sorted(lat)
    return {"workload": W.name, "requests": n_req, "data_points": W.N, "nlist": nlist,
            "p50_ms": float(np.percentile(lat_s, 50)), "p99_ms": float(np.percentile(lat_s, 99)),
            "mean_ms": float(np.mean(lat_s)), "solves_per_s": n_req / makespan, "makespan_s": makespan,
            "searches_per_s": sum(i * m for i, m in zip(iters, m_tot)) / makespan,
            "lambda_per_s": rate, "arrivals": f"Poisson, rate {rate:.2f}/s = 0.8 x calibrated service rate",
            "max_active": int(st.max_active), "batched_steps": int(st.steps),
            "mean_iterations": float(np.mean(iters)),
            "step_ms": {"busy": st.busy_ms / max(1, st.steps), "cg": st.cg_ms / max(1, st.steps),
                        "search": st.search_ms / max(1, st.steps), "other": st.other_ms / max(1, st.steps)},
            "graph_steps": int(st.graph_steps), "state_budget_gb": args.serve_budget_gb,
            "eq14": "certified second bound" if args.eq14 == 0 else "second-closest point found",
            "f_d": f"{args.fd0} -> {args.fd_final} over {args.ramp_iters} iterations",
            "edges": f"U{{{ex['edge_min']}..{ex['edge_max']}}}",
            "traction": f"U[{ex['t_min']}, {ex['t_max']}] random direction"}


def run_serve(args, world, rank, local):
    """Serving: resident data set, Poisson arrivals, continuous batching."""
    import torch

    import paper_2012_00357_gb300 as P

    P.build()
    torch.cuda.set_device(local)
    W = make_workload(args.workload)
    ctx = P.dd_create(local)
    clk = ClockSampler(local)
    sv = serve_leg(P, ctx, W, args, W.extra["requests"], clk=clk)
    n_req = sv["requests"]
    line = {
        "metric": METRIC, "value": sv["searches_per_s"], "unit": UNIT, "n_gpus": 1, "steps": n_req, "warmup": 48,
        "ms_per_step": sv["makespan_s"] * 1e3 / n_req, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (P_C refinement, rescoring) + f32",
        "data": "synthetic (dd_inputs generator, made on device)",
        "config": {"workload": W.name, "data_points": W.N, "requests": n_req, "edges": sv["edges"],
                   "traction": sv["traction"], "search": "ann", "f_d": sv["f_d"], "nlist": sv["nlist"],
                   "state_budget_gb": args.serve_budget_gb, "arrivals": sv["arrivals"],
                   "l2": "inputs larger than L2", "parallelism": "replicas x1"},
        "serve": {k: v for k, v in sv.items() if k not in ("workload", "edges", "traction", "f_d", "arrivals")},
        "gpu_launches": int(P.dd_launch_count(ctx)),
        "clocks": clk.summary(),
    }
    P.dd_destroy(ctx)
    return line


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, same workload and metric."""
    if rank != 0:
        return None
    W = make_workload(args.workload)
    C = None if W.extra.get("metric") == "pca" else I.isotropic_C(W.law.E, W.law.nu)
    per_step = max(4.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        if info is None or i == args.warmup:
            info = (oracle_dd_iterations(W, C, target_s=per_step) if W.N <= 2_000_000 and C is not None
                    else oracle_searches_per_s(W, C, target_s=per_step))
        if i >= args.warmup:
            vals.append(info["value"])
    v = statistics.mean(vals)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (dd_inputs)",
            "config": {"workload": W.name, "mesh": f"{W.n_el}^3 hex, 2x2x2 Gauss",
                       "material_points": W.m * max(1, len(W.loads)), "data_points": W.N, "law": W.law.kind,
                       "metric": W.extra.get("metric", "isotropic C of the law"), "load": W.loads[0][0],
                       "search": "exact FP64 brute force (the oracle) on a bounded query sample",
                       "parallelism": "host cores of rank 0"},
            "cpu_baseline": {**info, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # the headline metric is quoted at N = 10^9: the 32^3 cube with 4 load
    # cases on 10^9 points, approximate search (the other workloads by flag)
    ap.add_argument("--workload", default="cube32_N1e9_ann_4loads")
    ap.add_argument("--mode", default=None, choices=["tc", "tc_topk", "fp32", "ann", "knng", "serve"],
                    help="search mode (default: ann for *_ann workloads, serve for serve_*, else tc)")
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    # accuracy schedule of the approximate search: f_d from 0.3 to 0.8 over 5
    # iterations keeps the DD solution within 1e-3 of the exact-search one at
    # 10^8 and 10^9 points (the paper's ramp from 0, or a lower final f_d,
    # ends at a worse fixed point on these workloads: 0.7 is 6.5e-3 above at
    # 10^9)
    ap.add_argument("--fd-final", type=float, default=None,
                    help="final f_d of the approximate search (default: the workload's schedule, else 0.8)")
    ap.add_argument("--fd0", type=float, default=None, help="f_d of the first iteration (default: workload's, else 0.3)")
    ap.add_argument("--ramp-iters", type=int, default=None, help="iterations of the f_d ramp (default: workload's, else 5)")
    ap.add_argument("--nlist", type=int, default=0)
    ap.add_argument("--ann-levels", type=int, default=0)
    ap.add_argument("--ann-check", type=int, default=8192,
                    help="final states checked against the certified exact search (0: none)")
    ap.add_argument("--ann-alu", action="store_true",
                    help="nearest-centroid passes of the tree build and the cell ranking on the ALU only (the "
                         "tensor-core passes, the default, give the same answers)")
    ap.add_argument("--no-exact-tc", dest="exact_tc", action="store_false",
                    help="check with the FP32 exact scan instead of the tensor-core one (no FP16 copy)")
    ap.add_argument("--eq14", type=int, default=1, choices=[0, 1],
                    help="second distance of the Eq. (14) skip: 1 the second-closest point found (the paper's "
                         "estimate, used below f_d = 1; the default here), 0 the certified bound (the library's "
                         "default); the other rule is timed over the same steps and reported in detail")
    ap.add_argument("--no-eq14-compare", action="store_true", help="do not time the other Eq. (14) rule")
    ap.add_argument("--ann-budget", type=int, default=0,
                    help="leaves a query's warp scans before the leaf-major pass (0: library default, -1: all)")
    ap.add_argument("--knn-k", type=int, default=None, help="k of the k-NN graph (default: the workload's, else 128)")
    ap.add_argument("--knn-fd", type=float, default=None, help="f_d of the graph build (default: workload's, else 0.8)")
    ap.add_argument("--f-s", type=int, default=None, help="node-change bound of the graph walk (0: none; default: "
                    "the workload's, else 2)")
    ap.add_argument("--exact-solve", action="store_true",
                    help="also solve the first load case with the certified tensor-core exact search and with the "
                         "approximate search alone (solve time and distance at N, ANN vs exact; minutes at 10^9)")
    ap.add_argument("--exact-start", choices=("random", "ann", "both"), default="random",
                    help="association the exact solve of --exact-solve starts from: the approximate solve's random "
                         "one, its final one, or both runs")
    ap.add_argument("--exact-budget-s", type=float, default=900.0,
                    help="wall-clock budget of each exact solve of --exact-solve (it stops after the iteration that "
                         "passes it and reports whether it had converged)")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the short serving run reported in detail.serve (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.mode is None:
        args.mode = ("serve" if args.workload.startswith("serve") else "ann" if "_ann" in args.workload
                     else "knng" if "_knng" in args.workload else "tc")
    # f_d schedule of the approximate search: the workload's, unless given
    sched = I.WORKLOADS[args.workload].extra.get("schedule", (0.3, 0.8, 5))
    args.fd0 = sched[0] if args.fd0 is None else args.fd0
    args.fd_final = sched[1] if args.fd_final is None else args.fd_final
    args.ramp_iters = sched[2] if args.ramp_iters is None else args.ramp_iters
    ex = I.WORKLOADS[args.workload].extra
    args.knn_k = ex.get("knn_k", 128) if args.knn_k is None else args.knn_k
    args.knn_fd = ex.get("knn_fd", 0.8) if args.knn_fd is None else args.knn_fd
    args.f_s = ex.get("f_s", 2) if args.f_s is None else args.f_s
    world, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    elif args.mode == "serve":
        line = run_serve(args, world, rank, local)
    else:
        line = run_ours(args, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
