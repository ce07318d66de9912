#!/usr/bin/env python
"""Benchmark of the GATE TE iteration engine on one B300.

A step is one cold-start solve of the max-min TE problem on the workload to
within 1% of the optimum: te_reset (initial rates of Algorithm 1), te_solve
for K iterations (one persistent kernel launch running the whole iteration
loop), and te_allocation with a feasibility step.  The solver runs with the
paper's rule (default options).

Optimality is the metric of Section 4.1, mean_d min(S_d / max(OPT_d, theta), 1)
with theta = 1e-6 max_e C_e.  OPT comes from a stricter reference rule run in
the same process: the solver with beta bounded at --ref-beta-max times beta0
(residual balancing cannot freeze the iterate after the alpha increments),
--ref-gamma, for --ref-iters iterations, made feasible by proportional
scaling.  An exact max-min (a sequence of LPs over 36M paths) is out of
reach, so the same run measures the reference rule, and the default rule,
against the exact max-min of the workload's k = 1 variant (every demand's
first path; progressive filling on the host) and reports both.  K is the
first iteration count whose proportionally scaled allocation reaches
optimality >= 0.99 against OPT (probed every --probe-every iterations, then
refined in steps of --refine-every).  Algorithm 2 (the paper's projection) is
probed at the same points and reported beside: it trims whole paths, so where
an edge is far over capacity it empties demands.

roofline.achieved counts the method's algorithmic bytes with int32 edge ids
(4 B per incidence, 12 B per path, 8 B per demand, 8 B per edge per CTA) over
the iteration kernel's time; layout_achieved counts what the sliced layout
moves (16-bit ids).  The oracle numbers of cpu_baseline are extrapolated from
a timed sample (and say so), beside one full oracle solve of the 200-node
workload timed for real.

Default workload: the 1500-node synthetic WAN (10,056 directed edges, all
2,248,500 ordered pairs as gravity demands, k = 16 paths, 36M paths, 215M
path-edge incidences).  Inputs stay resident; each iteration streams 0.80 GB
(> the 126 MB L2) so no extra L2 flush is needed.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead.  Under torchrun every rank solves its own
replica (the method needs no collective on one instance per GPU).
"""
import argparse
import hashlib
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

METRIC = "ms to within 1% of optimal fairness objective (max-min, optimality >= 0.99); iter/s; % HBM peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large", choices=["tiny", "medium", "large", "wan3000"])
    ap.add_argument("--ref-iters", type=int, default=40000)
    ap.add_argument("--ref-alpha-max", type=float, default=32.0,
                    help="alpha cap of the OPT reference run")
    ap.add_argument("--ref-gamma", type=float, default=1e-3, help="gamma of the OPT reference run")
    ap.add_argument("--ref-gamma-max", type=float, default=0.0,
                    help="max-norm primal residual bar of the OPT reference run (0: off)")
    ap.add_argument("--ref-beta-max", type=float, default=4096.0,
                    help="bound on beta of the OPT reference run, times beta0")
    ap.add_argument("--ref-k", type=int, default=7975,
                    help="reference arm on the large workload: iterations the oracle is extrapolated to "
                         "(the CUDA arm's measured count to 1%%)")
    ap.add_argument("--no-k1-check", action="store_true",
                    help="skip the reference rule's accuracy check on the k = 1 variant")
    ap.add_argument("--no-medium-oracle", action="store_true",
                    help="skip the measured oracle solve of the 200-node workload")
    ap.add_argument("--probe-every", type=int, default=250)
    ap.add_argument("--refine-every", type=int, default=25)
    ap.add_argument("--target", type=float, default=0.99)
    ap.add_argument("--oracle-sample-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ablation", action="store_true",
                    help="iterations to 1%% with and without adaptive beta, and cold versus warm re-solves "
                         "after a demand change (Section 4 factor analysis), one JSON line")
    ap.add_argument("--batch", type=int, default=0, metavar="SCENARIOS",
                    help="what-if batch on the 500-node WAN: SCENARIOS failure scenarios x 4 demand matrices, "
                         "the batch engine against a loop of single-instance solves, one JSON line")
    ap.add_argument("--batch-iters", type=int, default=2000)
    ap.add_argument("--exact-k1", action="store_true",
                    help="the solver's max-min on the single-path (k = 1) variants of the 200- and 1500-node "
                         "workloads against their exact max-min (progressive filling), one JSON line each")
    ap.add_argument("--steady", default="", metavar="ALPHAS",
                    help="steady-state us per iteration at these fixed alphas (comma separated), one JSON line")
    ap.add_argument("--feasibility", type=int, default=0, metavar="K",
                    help="time the two feasibility steps (Algorithm 2 and proportional scaling, device output) "
                         "on the iterate after K iterations of the default solver, one JSON line")
    ap.add_argument("--literal", type=int, default=0, metavar="ITERS",
                    help="time the printed multi-block iteration (te_literal_run) and report the "
                         "capacity overload it leaves")
    ap.add_argument("--edge-mode", choices=["auto", "global"], default="auto",
                    help="the timed handle's (and --steady's) per-edge arrays of the iteration kernel: in "
                         "shared memory when they fit (auto) or always in global memory")
    ap.add_argument("--alpha-fair", default="", metavar="ALPHAS",
                    help="time to a duality-gap certificate of --cert-eps at each fixed alpha (e.g. 1,2)")
    ap.add_argument("--cert-eps", type=float, default=1e-3)
    ap.add_argument("--no-alpha-fair-check", action="store_true",
                    help="leave the certified alpha = 1 measurement out of the default line")
    ap.add_argument("--iters", type=int, default=0,
                    help="profiling runs only: use this K and skip the reference run and the probe")
    return ap.parse_args()


def dist_setup(backend: str = "nccl"):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE).  The
    ranks solve independent replicas: the only collectives are the barriers
    around the timed region and the maximum of the timings."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
        return ws, rank, local, dist
    return 1, 0, local, None


def max_over_ranks(values, dist, device=None):
    """Elementwise maximum of a list of floats over all ranks (the values
    themselves with one rank)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def shard(n: int, rank: int, world: int) -> list:
    """Instances of a what-if batch that rank takes: i = rank, rank + world,
    ... (no exchange between ranks)."""
    return list(range(rank, n, world))


def workload_desc(inst) -> str:
    s = inst.summary()
    return (f"{inst.name}: {s['nodes']}-node synthetic WAN, {s['edges']} directed edges, {s['demands']} demands, "
            f"{s['paths']} paths (k={s['k']}), {s['nnz']} path-edge incidences, mean {s['mean_hops']:.2f} hops")


class Optimality:
    """Section 4.1's optimality, mean_d min(S_d / max(OPT_d, theta), 1), of an
    allocation held on the device (evaluation only; torch ops)."""

    def __init__(self, inst, dev):
        import numpy as np
        import torch
        self.torch = torch
        self.K = inst.n_demands
        self.idx = torch.from_numpy(np.repeat(np.arange(inst.n_demands, dtype=np.int64),
                                              np.diff(inst.demand_path_off))).to(dev)
        self.theta = 1e-6 * float(inst.capacity.max())
        self.opt = None

    def totals(self, x):
        S = self.torch.zeros(self.K, dtype=self.torch.float64, device=x.device)
        S.index_add_(0, self.idx, x.to(self.torch.float64))
        return S

    def set_reference(self, x):
        self.opt = self.totals(x).clamp_min(self.theta)

    def __call__(self, x):
        return float(self.torch.minimum(self.totals(x) / self.opt, self.torch.ones_like(self.opt)).mean())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = [os.path.join(ROOT, "paper_2605_01748_b300", "csrc", f)
                  for f in ("te_iter.cu", "te_kernels.cuh", "te_internal.cuh")]


def kernel_hash() -> str:
    """Hash of the iteration kernel's sources (the kernel and its shared device code)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


# DRAM traffic of the iteration kernel from one ncu capture (written by hand
# from the capture's dram__bytes_read.sum + dram__bytes_write.sum): a JSON
# object with the workload, the bytes per iteration and the hash of the
# kernel sources it was taken on.  The traffic is reported only while the
# sources are unchanged and the workload is the captured one.
NCU_TRAFFIC_JSON = os.path.join(ROOT, "profiles", "k_iter_large_traffic.json")


def ncu_traffic(workload: str):
    """(DRAM bytes per iteration, source) of the captured workload, or
    (None, reason)."""
    if not os.path.exists(NCU_TRAFFIC_JSON):
        return None, "no capture recorded"
    rec = json.load(open(NCU_TRAFFIC_JSON))
    if rec.get("workload") != workload:
        return None, f"the capture is of the {rec.get('workload')} workload"
    if rec.get("kernel_source_sha256_16") != kernel_hash():
        return None, "the kernel changed since the capture"
    return float(rec["dram_bytes_per_iteration"]), os.path.relpath(NCU_TRAFFIC_JSON, ROOT)


def method_bytes(inst, grid: int) -> int:
    """Algorithmic bytes of one iteration by the per-unit figures of the
    method's traffic with int32 edge ids: 4 B per incidence (the path-edge
    ids), 12 B per path (its rate read and written, its offset), 8 B per
    demand (demand and multiplier) and 8 B per edge per CTA (the partial
    loads)."""
    return int(4 * inst.nnz + 12 * inst.n_paths + 8 * inst.n_demands + 8 * grid * inst.n_edges)


def ref_options(a) -> dict:
    """Options of the OPT reference run (a stricter rule than the default):
    beta bounded by --ref-beta-max times beta0, so that the balancing cannot
    freeze the iterate after the alpha increments."""
    return dict(alpha_max=a.ref_alpha_max, gamma=a.ref_gamma, gamma_max=a.ref_gamma_max, beta_max=a.ref_beta_max)


def first_path_variant(inst):
    """The k = 1 variant: every demand keeps only its first path."""
    import numpy as np
    from paper_2605_01748_b300 import instances
    keep = np.zeros(inst.n_paths, dtype=bool)
    keep[inst.demand_path_off[:-1]] = True
    v = instances.drop_paths(inst, keep, name=inst.name + "-k1")
    v.meta["k"] = 1
    return v


def exact_maxmin_k1(inst1):
    """Host reference leg: the exact max-min rates of single-path demands by
    progressive filling (the FP64 oracle's), and the host time it took."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    exact = O.maxmin_single_path(inst1)
    return exact, time.perf_counter() - t0


def run_rule_on(te, inst, dev, stream, opts, opt_eval, iters, every=0):
    """Runs the solver with `opts` on `inst` for up to `iters` iterations
    (stopping where its rule fires) and returns (result, optimality of the
    proportionally scaled allocation, first iteration count probed at
    `every` whose optimality reached 0.99 or None)."""
    import torch
    x = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
    t = te.TE(inst, cuda_stream=stream.cuda_stream, **opts)
    first = None
    if every > 0:
        while True:
            r = t.solve(every)
            te.te_allocation(t.h, x, te.PROJECT_SCALE)
            if first is None and opt_eval(x) >= 0.99:
                first = r["total_iters"]
            if r["converged"] or r["total_iters"] >= iters:
                break
    else:
        r = t.solve(iters)
    te.te_allocation(t.h, x, te.PROJECT_SCALE)
    q = opt_eval(x)
    t.close()
    return r, q, first


def run_ours(a, ws, rank, local, dist):
    import numpy as np
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    stream = torch.cuda.current_stream(dev)
    edge_mode = te.EDGES_GLOBAL if a.edge_mode == "global" else te.EDGES_AUTO
    t = te.TE(inst, cuda_stream=stream.cuda_stream, edge_mode=edge_mode)
    lay = t.layout()
    xdev = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
    opt = Optimality(inst, dev)

    SCALE, ALG2 = te.PROJECT_SCALE, te.PROJECT_ALG2
    ref_desc, ref_k1 = None, None
    if a.iters <= 0:
        # OPT: the stricter reference rule run from the cold start, made
        # feasible by proportional scaling
        ropts = ref_options(a)
        tr = te.TE(inst, cuda_stream=stream.cuda_stream, **ropts)
        ref_res = tr.solve(a.ref_iters)
        te.te_allocation(tr.h, xdev, SCALE)
        opt.set_reference(xdev)
        te.te_allocation(tr.h, xdev, ALG2)
        alg2_at_ref = opt(xdev)
        tr.close()
        ref_desc = (f"the solver under the reference rule {ropts} from the cold start, {ref_res['total_iters']} "
                    f"iterations (alpha {ref_res['alpha']:g}; "
                    f"{'stopped by its rule' if ref_res['converged'] else 'iteration cap'}), proportionally "
                    f"scaled; theta = 1e-6 max C_e")
        if rank == 0 and not a.no_k1_check:
            # accuracy of that rule against an exact optimum: the k = 1
            # variant of this workload, whose exact max-min is progressive filling
            inst1 = first_path_variant(inst)
            exact, ex_s = exact_maxmin_k1(inst1)
            ev1 = Optimality(inst1, dev)
            ev1.opt = torch.from_numpy(np.maximum(exact, ev1.theta)).to(dev)
            r1, q1, _ = run_rule_on(te, inst1, dev, stream, ropts, ev1, a.ref_iters)
            rd, qd, _ = run_rule_on(te, inst1, dev, stream, {}, ev1, a.ref_iters)
            ref_k1 = {"workload": workload_desc(inst1),
                      "reference_rule": {"optimality": round(q1, 5), "iters": r1["total_iters"],
                                         "alpha": r1["alpha"]},
                      "default_rule": {"optimality": round(qd, 5), "iters": rd["total_iters"], "alpha": rd["alpha"]},
                      "exact": f"progressive filling on the host ({ex_s:.1f} s)"}

    def probe_at(n):
        """Runs to total iteration n; returns (result, optimality scaled, optimality Algorithm 2)."""
        r = t.solve(n - t.solve(0)["total_iters"])
        te.te_allocation(t.h, xdev, SCALE)
        q = opt(xdev)
        te.te_allocation(t.h, xdev, ALG2)
        return r, q, opt(xdev)

    # probe: first K whose scaled allocation is within 1% of OPT, coarse then fine
    K, trace = (a.iters if a.iters > 0 else None), []
    alg2_best = (0.0, 0)
    stop_iters = None
    if K is None:
        t.reset()
        n, lo = 0, 0
        while n < a.ref_iters:
            r, q, q2 = probe_at(n + a.probe_every)
            n = r["total_iters"]
            trace.append((n, r["alpha"], round(q, 5), round(q2, 5)))
            if q2 > alg2_best[0]:
                alg2_best = (q2, n)
            if q >= a.target:
                K = n
                break
            if r["converged"]:
                stop_iters = n
                break
            lo = n
        if K is not None and K - lo > a.refine_every:
            t.reset()
            t.solve(lo)
            n = lo
            while n < K:
                n += a.refine_every
                r, q, q2 = probe_at(n)
                if q >= a.target:
                    trace.append((n, r["alpha"], round(q, 5), round(q2, 5)))
                    K = n
                    break
        if K is None:
            K = stop_iters or a.ref_iters
    q_at_K = trace[-1][2] if trace else None
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.warmup + a.steps)]
    launches0 = None
    for i in range(a.warmup + a.steps):
        if i == a.warmup:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            launches0 = t.layout()["kernel_launches"]
            clocks = ClockSampler(str(torch.cuda.get_device_properties(dev).uuid))
            clocks.__enter__()
            wall0 = time.perf_counter()
        e = ev[i]
        e[0].record(stream)
        t.reset()
        e[1].record(stream)
        t.solve(K)
        e[2].record(stream)
        te.te_allocation(t.h, xdev, SCALE)
        e[3].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks.__exit__(None, None, None)
    launches = t.layout()["kernel_launches"] - launches0
    timed = ev[a.warmup:]
    step_ms = [e[0].elapsed_time(e[3]) for e in timed]
    solve_ms = [e[1].elapsed_time(e[2]) for e in timed]
    total_ms = sum(step_ms)
    opt_check = opt(xdev) if opt.opt is not None else None

    # end to end through the public API with host buffers: demands in from
    # pinned host memory, allocation out to pinned host memory
    d_host = torch.from_numpy(inst.demand.astype(np.float64)).pin_memory()
    x_host = torch.empty(inst.n_paths, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for i in range(max(1, min(a.steps, 3))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t.set_demands(d_host)
        t.reset()
        t.solve(K)
        te.te_allocation(t.h, x_host, SCALE)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))

    # maximum over ranks
    ms_step = total_ms / a.steps
    ms_step, e2e_mean = max_over_ranks([ms_step, statistics.mean(e2e_ms)], dist, dev)

    solve_mean = statistics.mean(solve_ms)
    alg_bytes = method_bytes(inst, lay["grid"])
    achieved = alg_bytes * K / (solve_mean * 1e-3) / 1e9
    moved = lay["bytes_per_iter"] * K / (solve_mean * 1e-3) / 1e9
    traffic_iter, traffic_src = ncu_traffic(a.workload)
    if a.edge_mode == "global":
        traffic_iter, traffic_src = None, "the capture is of the shared-memory edge arrays"
    l2_resident = lay["bytes_per_iter"] < 126e6
    out = {
        "metric": METRIC,
        "value": round(ms_step, 4),
        "unit": "ms",
        "n_gpus": ws,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": workload_desc(inst),
            "objective": "max-min via alpha-continuation (alpha from 0, +1 per convergence, gamma 1e-3)",
            "iters_to_1pct": K,
            "k_source": "--iters" if a.iters > 0 else "probe of this run",
            "optimality_at_K": q_at_K,
            "optimality_timed_output": None if opt_check is None else round(opt_check, 5),
            "feasibility_step": "proportional scaling (te_allocation PROJECT_SCALE; not in the paper)",
            "opt_reference": ref_desc,
            "opt_reference_accuracy_k1": ref_k1,
            "algorithm2": None if ref_desc is None else {
                "best_optimality_probed": round(alg2_best[0], 5), "at_iters": alg2_best[1],
                "optimality_at_reference": round(alg2_at_ref, 5),
                "note": "the paper's projection on the same iterates; whole-path trims empty "
                        "the demands on edges far over capacity"},
            "probe_trace_tail": trace[-4:],
            "l2": (f"L2-resident: {lay['bytes_per_iter'] / 1e6:.1f} MB per iteration (< 126 MB L2), no flush; "
                   f"a step is one launch of K iterations over the same data") if l2_resident else
                  "no flush: every iteration streams the sliced incidence (> 126 MB L2)",
            "parallelism": "replicas" if ws > 1 else "single GPU",
            "step": "te_reset + te_solve(K) (one persistent launch) + te_allocation(PROJECT_SCALE, device out)",
            "edge_arrays": "global memory (edge_mode)" if a.edge_mode == "global" else "shared memory",
        },
        "iters_per_s": round(K / (solve_mean * 1e-3), 1),
        "solve_ms": round(solve_mean, 4),
        "us_per_iter": round(1e3 * solve_mean / K, 3),
        "projection_ms": round(statistics.mean([e[2].elapsed_time(e[3]) for e in timed]), 4),
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": hbm_peak,
            "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4),
            "traffic": None if traffic_iter is None else int(traffic_iter * K),
            "traffic_source": traffic_src,
            "kernel": "k_iter (persistent; one launch = K iterations)",
            "algorithmic_bytes_per_iter": alg_bytes,
            "algorithmic_bytes_rule": "4 B per incidence (int32 id) + 12 B per path + 8 B per demand "
                                      "+ 8 B per edge per CTA",
            "layout_bytes_per_iter": lay["bytes_per_iter"],
            "layout_achieved": round(moved, 1),
            "layout_frac": round(moved / hbm_peak, 4),
            "peak_source": peak_src,
            **({"note": "L2-resident workload: bound by latency and the grid barriers, not HBM"}
               if l2_resident else {}),
        },
        "e2e": {"value": round(e2e_mean, 4), "unit": "ms", "h2d_bytes_per_step": int(inst.n_demands * 8),
                "d2h_bytes_per_step": int(inst.n_paths * 4)},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
        "wall_s_timed": round(wall, 3),
    }
    # FP64 oracle beside it (host cores): a bounded sample of iterations of
    # the same workload, extrapolated to K, the GPU's error against it after
    # those iterations, and one full oracle solve of the 200-node workload
    # timed for real beside the same solve on the GPU
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        out.update(cpu_legs(a, inst, t, K, te, dev, stream))
    # the alpha-fair objective at alpha = 1 (proportional fairness) against
    # its exact optimum on the same workload, by the duality-gap certificate
    # (outside the timed region; the full mode is --alpha-fair)
    if rank == 0 and a.iters <= 0 and not a.no_alpha_fair_check:
        row = alpha_fair_row(a, te, inst, 1.0, stream, xdev, False)
        out["alpha_fair_certified"] = {"alpha": 1.0, "target": a.cert_eps, "certificate": CERT_DESC,
                                       "iters": row["iters"], "ms": row["value"],
                                       "certified_eps": row.get("certified_eps"),
                                       "paper_stop_rule": row["paper_stop_rule"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    t.close()


def cpu_legs(a, inst, t, K, te, dev, stream):
    """The oracle's baseline numbers and the GPU's error against it."""
    import numpy as np
    from oracle import oracle as O
    from paper_2605_01748_b300 import instances
    n = a.oracle_sample_iters
    cores = os.cpu_count() or 1
    s = O.OracleSolver(inst, threads=cores)
    t0 = time.perf_counter()
    s.run(n)
    dt = time.perf_counter() - t0
    per_iter = dt / n
    t1 = time.perf_counter()
    O.project_scale(inst, s.allocation())
    dp = time.perf_counter() - t1
    t.reset()
    t.solve(n)
    xg = t.allocation(project=False).astype(np.float64)
    xo = s.allocation()
    err = float(np.max(np.abs(xg - xo)) / max(np.max(np.abs(xo)), 1e-300))
    s1 = O.OracleSolver(inst, threads=1)
    t2 = time.perf_counter()
    s1.run(1)
    d1 = time.perf_counter() - t2
    del s1, s
    base = {"value": round((per_iter * K + dp) * 1e3, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "extrapolated": True,
            "sample": f"{n} FP64 oracle iterations of the same workload in one call ({dt:.2f} s, incl. its "
                      f"edge->path transpose), extrapolated to K={K} iterations, plus one proportional scaling "
                      f"({dp:.2f} s)",
            "s_per_iter": round(per_iter, 4), "s_per_iter_1_thread": round(d1, 4)}
    errs = {"max_rel_err_after_sample_iters": err, "iters": n}
    if a.workload != "medium" and not a.no_medium_oracle:
        # measured, not extrapolated: the 200-node workload solved to the stop
        # rule by the oracle on all host cores and by the GPU
        med = instances.make("medium", threads=cores)
        so = O.OracleSolver(med, threads=cores)
        t3 = time.perf_counter()
        so.run(a.ref_iters)
        xo_s = O.project_scale(med, so.allocation())
        d_or = time.perf_counter() - t3
        import torch
        tg = te.TE(med, cuda_stream=stream.cuda_stream)
        x = torch.empty(med.n_paths, dtype=torch.float32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tg.solve(10)
        tg.reset()
        torch.cuda.synchronize()
        e0.record(stream)
        rg = tg.solve(a.ref_iters)
        te.te_allocation(tg.h, x, te.PROJECT_SCALE)
        e1.record(stream)
        torch.cuda.synchronize()
        xg_s = x.cpu().numpy().astype(np.float64)
        tg.close()
        Sg, So = O.demand_totals(med, xg_s), O.demand_totals(med, xo_s)
        base["measured_medium"] = {
            "workload": workload_desc(med), "oracle_ms": round(d_or * 1e3, 1), "oracle_iters": so.iters,
            "gpu_ms": round(e0.elapsed_time(e1), 3), "gpu_iters": rg["total_iters"], "cores": cores,
            "step": "cold start to the stop rule (default options) plus proportional scaling, not extrapolated"}
        errs["medium_full_solve"] = {
            "same_stop_iteration": bool(so.iters == rg["total_iters"]),
            "max_rel_err_demand_totals": float(np.max(np.abs(Sg - So)) / max(So.max(), 1e-300))}
    return {"cpu_baseline": base, "error_vs_oracle": errs}


def oracle_k(inst, O, target: float, every: int, cap: int, threads: int):
    """The oracle's own iteration count to 1% (the same definition as the
    CUDA arm: OPT = the run to its stop rule, proportionally scaled); only
    affordable on the small workloads."""
    import numpy as np
    theta = 1e-6 * float(inst.capacity.max())
    s = O.OracleSolver(inst, threads=threads)
    s.run(cap)
    opt_S = O.demand_totals(inst, O.project_scale(inst, s.allocation()))
    s = O.OracleSolver(inst, threads=threads)
    while s.iters < cap:
        s.run(every)
        q = O.optimality(O.demand_totals(inst, O.project_scale(inst, s.allocation())), opt_S, theta)
        if q >= target or s.converged:
            return s.iters
    return s.iters


def run_ablation(a):
    """Iterations (and device time) to optimality >= 0.99 for: the default
    solver; residual balancing off (fixed beta0); and, after every demand is
    scaled by a seeded factor in [0.8, 1.2], a cold start, the paper's warm
    start (previous rates, duals and alpha reset, Algorithm 1's optional x^0)
    and a full warm start (rates, prices, beta and alpha kept).  OPT of each
    demand matrix: its own run to the stop rule, proportionally scaled."""
    import numpy as np
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    xdev = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
    SCALE = te.PROJECT_SCALE

    def reference(t):
        t.reset()
        r = t.solve(a.ref_iters)
        te.te_allocation(t.h, xdev, SCALE)
        return r

    def probe(t, opt, start_iters, cap):
        """Iterations beyond start_iters to reach the target (coarse, then fine)."""
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n, lo, ms = 0, 0, 0.0
        while n < cap:
            ev0.record(stream)
            r = t.solve(a.probe_every)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            n = t.solve(0)["total_iters"] - start_iters
            te.te_allocation(t.h, xdev, SCALE)
            q = opt(xdev)
            if q >= a.target:
                return n, round(q, 5), round(ms, 1)
            if r["converged"]:
                return None, round(q, 5), round(ms, 1)
        return None, round(q, 5), round(ms, 1)

    out = {"mode": "ablation", "workload": workload_desc(inst), "target": a.target,
           "probe_every": a.probe_every, "unit": "iterations (device ms of those iterations)"}
    base = te.TE(inst, cuda_stream=stream.cuda_stream)
    opt = Optimality(inst, dev)
    rr = reference(base)
    opt.set_reference(xdev)
    out["reference_iters"] = rr["total_iters"]
    base.reset()
    K, q, ms = probe(base, opt, 0, rr["total_iters"])
    out["default"] = {"iters": K, "optimality": q, "ms": ms}
    x_at_K = torch.empty_like(xdev)
    te.te_allocation(base.h, x_at_K, te.PROJECT_NONE)
    # residual balancing off: beta stays at beta0
    fixed = te.TE(inst, adapt_beta=0, cuda_stream=stream.cuda_stream)
    Kf, qf, msf = probe(fixed, opt, 0, 3 * (K or rr["total_iters"]))
    out["fixed_beta"] = {"iters": Kf, "optimality": qf, "ms": msf,
                         "note": None if Kf else f"not reached within {3 * (K or rr['total_iters'])} iterations"}
    fixed.close()
    # demand change
    rng = np.random.default_rng(20260)
    D2 = inst.demand * np.exp(rng.uniform(np.log(0.8), np.log(1.2), inst.n_demands))
    new = te.TE(instances.Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst, inst.capacity,
                                   inst.demand_src, inst.demand_dst, D2, inst.demand_path_off,
                                   inst.path_edge_off, inst.path_edges, dict(inst.meta)),
                cuda_stream=stream.cuda_stream)
    opt2 = Optimality(inst, dev)
    rr2 = reference(new)
    opt2.set_reference(xdev)
    new.reset()
    Kc, qc, msc = probe(new, opt2, 0, rr2["total_iters"])
    out["changed_demands"] = {"reference_iters": rr2["total_iters"],
                              "cold": {"iters": Kc, "optimality": qc, "ms": msc}}
    new.close()
    # warm starts from the base solution at its K (the allocation in service)
    d2 = torch.from_numpy(D2).to(dev)
    for name, keep in (("warm_paper", False), ("warm_full", True)):
        base.reset()
        base.solve(K or rr["total_iters"])
        base.set_demands(d2)
        if not keep:
            base.warm_start(x_at_K, keep_duals=False)
        start = base.solve(0)["total_iters"]
        Kw, qw, msw = probe(base, opt2, start, rr2["total_iters"])
        out["changed_demands"][name] = {"iters": Kw, "optimality": qw, "ms": msw}
    # error against the FP64 oracle after a short sample of the default solve
    from oracle import oracle as O
    n_err = 3
    base.set_demands(inst.demand)  # the warm starts above changed them
    base.reset()
    base.solve(n_err)
    so = O.OracleSolver(inst, threads=os.cpu_count() or 0)
    so.run(n_err)
    xo = so.allocation()
    xg = base.allocation(project=te.PROJECT_NONE).astype(np.float64)
    out["error_vs_oracle"] = {"max_rel_err": float(np.max(np.abs(xg - xo)) / max(np.max(np.abs(xo)), 1e-300)),
                              "iters": n_err}
    base.close()
    print(json.dumps(out), flush=True)


def run_batch(a, ws=1, rank=0, dist=None):
    """The batch engine against the plain loop on the same GPU: every
    instance of the what-if batch (a.batch failure scenarios of the 500-node
    WAN, each removing 1-3 links, x 4 demand matrices perturbed by a clipped
    lognormal factor) runs --batch-iters iterations with the same options
    (no early stop), once as one batch launch and once as one te_solve per
    instance (one handle per scenario, te_set_demands + te_reset per matrix).
    Device time by CUDA events; the batch's first call includes its CTA-shape
    timing, so the batch is timed on a second solve after te_batch_reset."""
    import numpy as np
    import torch
    from paper_2605_01748_b300 import instances, te

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    base = instances.make_batch_base(threads=os.cpu_count() or 0)
    W_all = instances.make_what_if(base, a.batch, 4, seed=0)
    # under torchrun each rank takes its share of the instances (no exchange)
    mine = shard(len(W_all), rank, ws)
    W = [W_all[i] for i in mine]
    gen_s = time.time() - t0
    K = a.batch_iters
    opts = dict(gamma=-1.0)
    t0 = time.time()
    b = te.TEBatch(W, cuda_stream=stream.cuda_stream, **opts)
    create_s = time.time() - t0
    b.solve(K)  # includes the CTA-shape timing
    b.reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = b.solve(K)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)
    info = b.info()
    # error against the FP64 oracle: the first and the last instance after a
    # short run of the same options (the oracle takes ~0.1 s per iteration here)
    b.reset()
    n_err = 20
    b.solve(n_err)
    batch_err = {}
    if rank == 0:
        from oracle import oracle as O
        for j in sorted({0, len(W) - 1}):
            so = O.OracleSolver(W[j], threads=os.cpu_count() or 0, **opts)
            so.run(n_err)
            xo = so.allocation()
            xg = b.allocation(j, project=te.PROJECT_NONE).astype(np.float64)
            batch_err[f"instance_{mine[j]}"] = float(np.max(np.abs(xg - xo)) / max(np.max(np.abs(xo)), 1e-300))
    b.close()
    assert all(r["iters"] == K for r in res)
    loop_ms = 0.0
    first = {}
    for i in mine:  # one handle per scenario, its matrices through te_set_demands
        first.setdefault(i // 4, i)
    for sidx, i0 in first.items():
        t = te.TE(W_all[i0], cuda_stream=stream.cuda_stream, **opts)
        for i in [i for i in mine if i // 4 == sidx]:
            t.set_demands(W_all[i].demand)
            t.reset()
            e0.record(stream)
            t.solve(K)
            e1.record(stream)
            torch.cuda.synchronize()
            loop_ms += e0.elapsed_time(e1)
        t.close()
    batch_ms, loop_ms = max_over_ranks([batch_ms, loop_ms], dist, torch.device("cuda", local))
    if rank != 0:
        return
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    n = len(W_all)
    # the method's bytes (the headline's per-unit rule, summed over the
    # instances; per-CTA partial loads for the CTAs an instance runs on) and
    # the bytes this layout moves
    cpi = max(1, int(info.get("ctas_per_instance", 1) or 1))
    method = sum(method_bytes(w, cpi) for w in W_all)
    achieved = method * K / (batch_ms * 1e-3) / 1e9
    layout_achieved = info["bytes_per_iter"] * ws * K / (batch_ms * 1e-3) / 1e9
    out = {"mode": "batch", "workload": f"what-if batch: {a.batch} failure scenarios x 4 demand matrices = {n} "
                                         f"instances of the 500-node WAN ({base.n_edges} directed edges, "
                                         f"{base.n_demands} demands, k=8, {info['n_paths']} paths in all)",
           "iterations_per_instance": K, "batch_ms": round(batch_ms, 1), "loop_ms": round(loop_ms, 1),
           "speedup": round(loop_ms / batch_ms, 2),
           "instance_iters_per_s": {"batch": round(n * K / (batch_ms * 1e-3), 1),
                                    "loop": round(n * K / (loop_ms * 1e-3), 1)},
           "batch_roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(achieved / hbm, 4), "algorithmic_bytes_per_iter": method,
                              "algorithmic_bytes_rule": "4 B per incidence (int32 id) + 12 B per path + 8 B per "
                                                        "demand + 8 B per edge per CTA, summed over the instances",
                              "layout_bytes_per_iter": info["bytes_per_iter"] * ws,
                              "layout_achieved": round(layout_achieved, 1),
                              "layout_frac": round(layout_achieved / hbm, 4)},
           "batch_shape": {"warps_per_cta": info["warps_per_cta"], "ctas_per_sm": info["ctas_per_sm"],
                           "lanes_per_demand": info["lanes_per_demand"]},
           "host_s": {"generate": round(gen_s, 1), "batch_create": round(create_s, 1)},
           "options": "alpha-continuation and residual balancing as default, no early stop (gamma < 0)",
           "error_vs_oracle": {"max_rel_err": batch_err, "iters": n_err}}
    print(json.dumps(out), flush=True)


def run_exact_k1(a):
    """Against an exact optimum: the single-path (k = 1) variants of the 200-
    and 1500-node workloads, whose exact max-min rates come from progressive
    filling (host reference leg).  For each: the solver under the default
    options and under the reference rule, probed every --probe-every
    iterations until its rule fires; the first iteration count whose
    proportionally scaled allocation is within 1% of the exact optimum (then
    refined), and that many iterations timed like the headline step (reset,
    solve, feasibility step).  One JSON line per variant."""
    import numpy as np
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for name in ("medium", "large"):
        inst = first_path_variant(instances.make(name, threads=os.cpu_count() or 0))
        exact, wf_s = exact_maxmin_k1(inst)
        ev = Optimality(inst, dev)
        ev.opt = torch.from_numpy(np.maximum(exact, ev.theta)).to(dev)
        x = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
        line = {"mode": "exact-k1", "workload": workload_desc(inst), "exact_host_s": round(wf_s, 1),
                "metric": "ms to within 1% of the exact max-min (optimality >= 0.99)", "unit": "ms"}
        for label, opts in (("default", {}), ("reference_rule", ref_options(a))):
            t = te.TE(inst, cuda_stream=stream.cuda_stream, **opts)
            rows, first, lo, best = [], None, 0, 0.0
            while True:
                r = t.solve(a.probe_every)
                te.te_allocation(t.h, x, te.PROJECT_SCALE)
                q = ev(x)
                best = max(best, q)
                rows.append((r["total_iters"], r["alpha"], round(q, 5)))
                if first is None and q >= a.target:
                    first = r["total_iters"]
                    break
                if r["converged"] or r["total_iters"] >= a.ref_iters:
                    break
                lo = r["total_iters"]
            res = {"stop_or_hit": rows[-1], "best_optimality": round(best, 5), "trace_tail": rows[-4:]}
            if first is not None:
                t.reset()
                t.solve(lo)
                n = lo
                while n < first:
                    n += a.refine_every
                    t.solve(a.refine_every)
                    te.te_allocation(t.h, x, te.PROJECT_SCALE)
                    if ev(x) >= a.target:
                        first = n
                        break
                ms = []
                for i in range(a.warmup + a.steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    t.reset()
                    t.solve(first)
                    te.te_allocation(t.h, x, te.PROJECT_SCALE)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if i >= a.warmup:
                        ms.append(e0.elapsed_time(e1))
                res.update({"iters_to_1pct": first, "value": round(statistics.mean(ms), 4),
                            "optimality_timed_output": round(ev(x), 5)})
            else:
                res.update({"iters_to_1pct": None, "value": None})
            line[label] = res
            t.close()
        line["reference_rule_options"] = ref_options(a)
        print(json.dumps(line), flush=True)


def run_reference(a, ws, rank):
    """The FP64 CPU oracle as it stands, on the host cores, same workload and
    metric.  Each step runs a bounded sample of oracle iterations on the full
    workload, scales it to K iterations and adds one proportional scaling of
    the result.  K: on tiny and medium the oracle's own count to 1%; on large
    (about 20,000 FP64 iterations of 1 s each would be needed to find it) the
    count given by --ref-k (the CUDA arm's measured count); both arms run the
    same iteration, equal within 1e-4 at equal counts.  The value is an
    extrapolation from the timed sample and says so."""
    from oracle import oracle as O
    from paper_2605_01748_b300 import instances

    if rank != 0:
        return
    cores = os.cpu_count() or 1
    inst = instances.make(a.workload, threads=cores)
    if a.iters > 0:
        K, k_src = a.iters, "--iters"
    elif a.workload in ("tiny", "medium"):
        K = oracle_k(inst, O, a.target, a.refine_every, a.ref_iters, cores)
        k_src = "the oracle's own probe (stop-rule reference, proportional scaling)"
    else:
        K, k_src = a.ref_k, ("--ref-k: the iteration count to 1% that the CUDA arm measures on this workload "
                             "(finding it with the oracle would take about 20,000 FP64 iterations of ~1 s)")
    n = a.oracle_sample_iters
    times, proj, steps_ms = [], [], []
    for i in range(a.warmup + a.steps):
        s = O.OracleSolver(inst, threads=cores)
        t0 = time.perf_counter()
        s.run(n)
        dt = time.perf_counter() - t0
        t1 = time.perf_counter()
        O.project_scale(inst, s.allocation())
        dp = time.perf_counter() - t1
        if i >= a.warmup:
            times.append((dt / n * K + dp) * 1e3)
            proj.append(dp * 1e3)
            steps_ms.append((dt + dp) * 1e3)
    v = statistics.mean(times)
    # ms_per_step: the wall time of one timed step as run (the bounded sample);
    # value: the metric, extrapolated from that sample to K iterations
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": ws,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(statistics.mean(steps_ms), 1),
           "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(inst), "iters_to_1pct": K, "k_source": k_src,
                      "extrapolated": True,
                      "feasibility_step": "proportional scaling (oracle project_scale)"},
           "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle", "extrapolated": True,
                            "sample": f"per step: {n} FP64 oracle iterations of the full workload from the cold "
                                      f"start, scaled to K={K}, plus one proportional scaling "
                                      f"({statistics.mean(proj):.0f} ms)"},
           "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def certified_eps(gap: float, primal: float, dual: float, alpha: float, n_demands: int) -> float:
    """Unit-free bound on the distance of a feasible allocation to the exact
    alpha-fair optimum U*, from the weak-duality bracket primal <= U* <= dual
    (te_gap_projected).  alpha = 1: gap / n_demands bounds the mean of
    log(S*_c / S_c) over demands (U is a sum of logarithms, so only its
    differences are free of units).  alpha != 1: U_alpha(S) = (S^(1-alpha) -
    1) / (1 - alpha) carries a constant -1 / (1 - alpha) per demand, which
    the gap does not see; without it the objective is homogeneous in the
    rates, so gap / min(|primal_h|, |dual_h|) with that constant removed
    bounds (U*_h - U_h) / |U*_h| whatever the units (U_h and the bracket
    share one sign)."""
    if not math.isfinite(gap):
        return math.inf
    if alpha == 1.0:
        return gap / max(n_demands, 1)
    shift = n_demands / (1.0 - alpha)
    lo, hi = primal + shift, dual + shift
    if lo * hi <= 0.0:
        return math.inf
    return gap / min(abs(lo), abs(hi))


CERT_DESC = ("alpha = 1: gap / n_demands (mean log-ratio to the optimum); else gap / min(|primal_h|, |dual_h|), "
             "_h: without U_alpha's constant -1/(1-alpha) per demand (relative objective)")


def alpha_fair_row(a, te, inst, alpha, st, x, with_oracle):
    """One alpha of the certified measurement (see run_alpha_fair): what the
    paper's stop rule leaves, then the iterations and device time to a
    certificate of --cert-eps, and (with_oracle) the FP64 oracle run for the
    same number of iterations."""
    import numpy as np
    import torch

    fixed = dict(alpha_target=alpha, alpha_start=alpha, continuation=0)

    def cert(t):
        g, pr, du = t.gap(project=te.PROJECT_SCALE)
        return certified_eps(g, pr, du, alpha, inst.n_demands), (g, pr, du)

    row = {}
    t = te.TE(inst, cuda_stream=st.cuda_stream, **fixed)
    r = t.solve(a.ref_iters)
    e_stop, _ = cert(t)
    row["paper_stop_rule"] = {"iters": r["iters"], "converged": bool(r["converged"]), "certified_eps": e_stop}
    t.close()
    t = te.TE(inst, cuda_stream=st.cuda_stream, gamma=-1.0, **fixed)
    first, lo, trace = None, 0, []
    while True:
        n = int(t.solve(a.probe_every)["total_iters"])
        e, _ = cert(t)
        trace.append((n, e))
        if e <= a.cert_eps:
            first = n
            break
        lo = n
        if n >= a.ref_iters:
            break
    row["probe_tail"] = trace[-3:]
    if first is not None:
        t.reset()
        t.solve(lo)
        n = lo
        while n < first:
            n += a.refine_every
            t.solve(a.refine_every)
            if cert(t)[0] <= a.cert_eps:
                first = n
                break
        ms = []
        for i in range(a.warmup + a.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            t.reset()
            rr = t.solve(first)
            t.allocation(project=te.PROJECT_SCALE, out=x)
            e, bracket = cert(t)
            e1.record(st)
            torch.cuda.synchronize()
            if i >= a.warmup:
                ms.append(e0.elapsed_time(e1))
        v = statistics.mean(ms)
        row.update({"iters": first, "value": round(v, 3), "certified_eps": e,
                    "gap_primal_dual": bracket, "iters_per_s": round(first / (v / 1e3), 1)})
        if with_oracle:
            from oracle import oracle as O
            s = O.OracleSolver(inst, gamma=-1.0, threads=os.cpu_count() or 0, **fixed)
            s.run(first)
            xo = O.project_scale(inst, s.allocation())
            go, pro, duo = O.gap(inst, xo, s.prices(), alpha)
            xg = x.cpu().numpy().astype(np.float64)
            Sg, So = O.demand_totals(inst, xg), O.demand_totals(inst, xo)
            row["oracle_same_iters"] = {
                "certified_eps": certified_eps(go, pro, duo, alpha, inst.n_demands),
                "max_rel_err_rates": float(np.max(np.abs(xg - xo)) / max(np.max(np.abs(xo)), 1e-300)),
                "max_rel_err_demand_totals": float(np.max(np.abs(Sg - So)) / max(np.max(So), 1e-300)),
                "beta_gpu_oracle": [rr["beta"], s.beta]}
    else:
        row.update({"iters": None, "value": None})
    t.close()
    return row


def run_alpha_fair(a):
    """alpha-fair objectives at fixed alpha (Eq. 4; no continuation) against
    their exact optimum, certified by the duality gap: the Lagrangian dual at
    the solver's prices bounds U* from above and the proportionally scaled
    allocation from below, so certified_eps is an upper bound on the
    distance to the exact optimum that needs no reference solve.  For each
    alpha: the default solver with the stop rule off, probed every
    --probe-every iterations (te_gap_projected) until certified_eps <=
    --cert-eps, refined in steps of --refine-every, and that many iterations
    timed as one step (te_reset, te_solve(K), te_allocation with scaling into
    device memory, te_gap_projected: the certificate is part of the result);
    beside it what the paper's stop rule (gamma 1e-3) leaves.  On the 200-node
    and smaller workloads the FP64 oracle runs the same K iterations and its
    certificate and allocation are compared.  One JSON line."""
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    x = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
    line = {"mode": "alpha-fair", "workload": workload_desc(inst),
            "metric": f"ms to a duality-gap certificate within {a.cert_eps:g} of the exact alpha-fair optimum",
            "unit": "ms", "certificate": CERT_DESC}
    for alpha in [float(v) for v in a.alpha_fair.split(",")]:
        line[f"alpha={alpha:g}"] = alpha_fair_row(a, te, inst, alpha, st, x, inst.n_paths <= 1_000_000)
    print(json.dumps(line), flush=True)


def run_literal(a):
    """The printed multi-block update equations on the device (te_literal_run,
    an ablation): device time per iteration from two runs of different
    length (the difference removes the per-call set-up), and what the
    iterate looks like after --literal iterations at alpha = 1, beta = 1
    (normalised units): the largest relative capacity overload and the share
    of edges over capacity, against the two-block iteration of te_solve run
    to its stop rule and made feasible by proportional scaling.  One JSON
    line."""
    import numpy as np
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    n2 = a.literal
    n1 = max(1, n2 // 5)
    times = {}
    for n in (n1, n2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = te.te_literal_run(inst, 1.0, 1.0, n)
        times[n] = time.perf_counter() - t0
    plen = np.diff(inst.path_edge_off)
    L = np.bincount(inst.path_edges, weights=np.repeat(np.maximum(x, 0.0), plen), minlength=inst.n_edges)
    over = (L - inst.capacity) / inst.capacity
    t = te.TE(inst, alpha_target=1.0, alpha_start=1.0, continuation=0)
    r = t.solve(a.ref_iters)
    xs = t.allocation(project=te.PROJECT_SCALE).astype(np.float64)
    Ls = np.bincount(inst.path_edges, weights=np.repeat(xs, plen), minlength=inst.n_edges)
    t.close()
    per_iter_ms = (times[n2] - times[n1]) / (n2 - n1) * 1e3
    print(json.dumps({"mode": "literal", "workload": workload_desc(inst), "alpha": 1.0, "beta": 1.0,
                      "iters": n2, "ms_per_iter": round(per_iter_ms, 3),
                      "call_s": {str(n1): round(times[n1], 3), str(n2): round(times[n2], 3)},
                      "literal": {"max_overload": float(over.max()),
                                  "edges_over_capacity": float((over > 1e-6).mean()),
                                  "min_rate": float(x.min())},
                      "two_block": {"iters": r["iters"], "converged": bool(r["converged"]),
                                    "max_overload_after_scaling": float(((Ls - inst.capacity) / inst.capacity).max())}}),
          flush=True)


def run_steady(a):
    """Steady-state time per iteration of the iteration kernel at fixed
    alphas (no continuation, no stop, adaptive beta): CUDA events around
    te_solve on the launching stream, best of 3 x 300 iterations after 60
    warm-up iterations; one JSON line."""
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    row = {}
    for alpha in [float(v) for v in a.steady.split(",")]:
        t = te.TE(inst, alpha_target=alpha, alpha_start=alpha, gamma=-1.0, cuda_stream=st.cuda_stream,
                  edge_mode=te.EDGES_GLOBAL if a.edge_mode == "global" else te.EDGES_AUTO)
        lay = t.layout()
        grid, edges_global = lay["grid"], lay["edges_global"]
        t.solve(60)
        best = math.inf
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            r = t.solve(300)
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e3 / r["iters"])
        row[f"{alpha:g}"] = round(best, 1)
        t.close()
    # the method's bytes per iteration (the headline's per-unit rule) over the
    # best time per iteration, against the measured peak
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    mb = method_bytes(inst, grid)
    frac = {k: round(mb / (v * 1e-6) / 1e9 / hbm, 4) for k, v in row.items()}
    print(json.dumps({"mode": "steady", "workload": workload_desc(inst), "edge_mode": a.edge_mode,
                      "edges_global": bool(edges_global), "us_per_iter": row, "method_bytes_per_iter": mb,
                      "frac_of_measured_hbm": frac}), flush=True)


def run_feasibility(a):
    """Time of te_allocation with each feasibility step on one iterate (the
    default solver after a.feasibility iterations): CUDA events on the
    handle's stream around one call, best of 5 after one warm-up call;
    device output, so no host copy is timed.  One JSON line."""
    import torch
    from paper_2605_01748_b300 import instances, te

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    inst = instances.make(a.workload, threads=os.cpu_count() or 0)
    t = te.TE(inst, cuda_stream=st.cuda_stream)
    r = t.solve(a.feasibility)
    out = torch.empty(t.n_paths, dtype=torch.float32, device=dev)
    row = {"mode": "feasibility", "workload": workload_desc(inst), "iters": r["iters"], "alpha": r["alpha"]}
    for name, proj in (("algorithm2", te.PROJECT_ALG2), ("scaling", te.PROJECT_SCALE)):
        t.allocation(project=proj, out=out)
        best = math.inf
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            t.allocation(project=proj, out=out)
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        row[name] = {"ms": round(best, 3), "sum_of_rates": float(out.double().sum())}
    t.close()
    print(json.dumps(row), flush=True)


def main():
    a = parse()
    ws, rank, local, dist = dist_setup()
    if a.steady:
        run_steady(a)
    elif a.feasibility > 0:
        run_feasibility(a)
    elif a.exact_k1:
        run_exact_k1(a)
    elif a.alpha_fair:
        run_alpha_fair(a)
    elif a.literal > 0:
        run_literal(a)
    elif a.batch > 0:
        run_batch(a, ws, rank, dist)
    elif a.ablation:
        run_ablation(a)
    elif a.impl == "reference":
        run_reference(a, ws, rank)
    else:
        run_ours(a, ws, rank, local, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
