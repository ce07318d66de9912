"""Writes fd_medium_alpha1_K200.json: FP64 central differences of the
differentiated objective on the 200-node workload (the differentiated
alpha = 1 configuration), computed by the FP64 oracle only.

J(C, D) = sum_c log S_c after K = 200 iterations of the fixed schedule
(alpha = 1, beta0 = 1 / (mean path length * mean initial rate) in caller
units, no residual balancing, no continuation) from the initial state of
Algorithm 1.  50 coordinates are drawn with a seeded generator among the
1,180 capacities and 39,800 demands (half each); for each, the central
difference (J(theta + h) - J(theta - h)) / (2 h) with h = 1e-3 |theta|.

Run from the repository root:  python tests/golden/make_fd_medium.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2605_01748_b300 import instances  # noqa: E402
from paper_2605_01748_b300.instances import Instance  # noqa: E402

ALPHA, K, REL_STEP, N_COORD, SEED = 1.0, 200, 1e-3, 50, 2026
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fd_medium_alpha1_K200.json")


def beta0_of(inst):
    return inst.n_paths ** 2 / (inst.nnz * inst.demand.sum())


def objective(inst, C, D, beta0, threads):
    I = Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst, C, inst.demand_src, inst.demand_dst, D,
                 inst.demand_path_off, inst.path_edge_off, inst.path_edges, {})
    s = O.OracleSolver(I, alpha_target=ALPHA, alpha_start=ALPHA, beta0=beta0, adapt_beta=False,
                       continuation=False, gamma=-1.0, scale_mode=2, threads=threads)
    s.run(K)
    S = O.demand_totals(I, s.allocation())
    return float(np.sum(np.log(S)))


def main():
    inst = instances.make_medium(seed=0, threads=os.cpu_count() or 0)
    b0 = beta0_of(inst)
    rng = np.random.Generator(np.random.PCG64(SEED))
    ce = rng.choice(inst.n_edges, N_COORD // 2, replace=False)
    cd = rng.choice(inst.n_demands, N_COORD - N_COORD // 2, replace=False)
    rows = []
    threads = os.cpu_count() or 0
    J0 = objective(inst, inst.capacity, inst.demand, b0, threads)
    for kind, idx in [("C", int(e)) for e in ce] + [("D", int(c)) for c in cd]:
        base = inst.capacity if kind == "C" else inst.demand
        theta = float(base[idx])
        h = REL_STEP * abs(theta)
        vals = []
        for sgn in (+1, -1):
            v = base.copy()
            v[idx] = theta + sgn * h
            C, D = (v, inst.demand) if kind == "C" else (inst.capacity, v)
            vals.append(objective(inst, C, D, b0, threads))
        rows.append({"kind": kind, "index": idx, "theta": theta, "h": h, "J_plus": vals[0], "J_minus": vals[1],
                     "fd": (vals[0] - vals[1]) / (2 * h)})
        print(kind, idx, rows[-1]["fd"], flush=True)
    json.dump({"workload": "200-node synthetic WAN, seed 0 (instances.make_medium)", "alpha": ALPHA, "K": K,
               "beta0": b0, "rel_step": REL_STEP, "seed": SEED, "J": J0, "coords": rows}, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
