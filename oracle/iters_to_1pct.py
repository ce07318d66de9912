"""Iterations the FP64 oracle needs to come within 1% of the max-min optimum
(optimality metric of Section 4.1) on a workload -- TEST/BENCH INFRASTRUCTURE.

Writes oracle/iters_to_1pct_<workload>.json, which the benchmark's CPU
reference leg uses to turn its timed sample of oracle iterations into a time
to 1%.  Calls only the oracle and the seeded instance generator.

Procedure: (1) a long oracle run with the default options (max-min through
alpha-continuation, gamma = 1e-3) of --ref-iters iterations gives the
reference totals OPT_d (exact max-min is out of reach by LP at this size);
(2) a second run from the initial state projects every --every iterations
(Algorithm 2) and records the first iteration whose projected allocation
has optimality >= 0.99 against OPT.

    python oracle/iters_to_1pct.py --workload large --threads 6
"""
import argparse
import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2605_01748_b300 import instances  # noqa: E402


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ref-iters", type=int, default=3000)
    ap.add_argument("--every", type=int, default=25)
    ap.add_argument("--target", type=float, default=0.99)
    a = ap.parse_args()
    inst = instances.make(a.workload, threads=a.threads)
    theta = 1e-6 * float(inst.capacity.max())
    t0 = time.time()
    ref = O.OracleSolver(inst, threads=a.threads)
    ref.run(a.ref_iters)
    opt_S = O.demand_totals(inst, O.project(inst, ref.allocation(), ref.alpha))
    t_ref = time.time() - t0
    trace = []
    s = O.OracleSolver(inst, threads=a.threads)
    K = None
    t1 = time.time()
    while s.iters < a.ref_iters:
        s.run(a.every)
        xp = O.project(inst, s.allocation(), s.alpha)
        q = O.optimality(O.demand_totals(inst, xp), opt_S, theta)
        trace.append([s.iters, s.alpha, q])
        print(json.dumps({"iters": s.iters, "alpha": s.alpha, "optimality": q}), flush=True)
        if q >= a.target:
            K = s.iters
            break
    out = {"workload": a.workload, "digest": inst.digest(), "iters_to_target": K, "target": a.target,
           "snapshot_every": a.every, "reference_iters": ref.iters, "reference_alpha": ref.alpha,
           "threads": a.threads, "seconds_reference": round(t_ref, 1), "seconds_probe": round(time.time() - t1, 1),
           "trace": trace}
    path = os.path.join(_ROOT, "oracle", f"iters_to_1pct_{a.workload}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
