"""Pins of the oracle's gradient of the fairness objective through K
fixed-schedule iterations (reverse mode, checkpointed): FP64 central finite
differences of J on the 12-node instance, J against a separate forward run,
independence of the checkpoint spacing, and the closed form at K = 0
(J = sum_c U(D_c), dJ/dD_c = U'(D_c), dJ/dC = 0)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_01748_b300.instances import Instance

K, BETA0 = 30, 0.05


def _with(inst, C=None, D=None):
    return Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst, inst.capacity if C is None else C,
                    inst.demand_src, inst.demand_dst, inst.demand if D is None else D, inst.demand_path_off,
                    inst.path_edge_off, inst.path_edges, {})


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
def test_gradient_matches_central_differences(tiny, alpha):
    J, gC, gD = O.gradient(tiny, alpha, BETA0, K)
    scale = max(np.abs(gC).max(), np.abs(gD).max())
    rng = np.random.default_rng(0)
    for e in rng.choice(tiny.n_edges, 6, replace=False):
        h = 1e-6 * tiny.capacity[e]
        C1, C2 = tiny.capacity.copy(), tiny.capacity.copy()
        C1[e] += h
        C2[e] -= h
        fd = (O.gradient(_with(tiny, C=C1), alpha, BETA0, K)[0] - O.gradient(_with(tiny, C=C2), alpha, BETA0, K)[0]) / (2 * h)
        assert abs(fd - gC[e]) <= 1e-6 * scale, (e, fd, gC[e])
    for c in rng.choice(tiny.n_demands, 6, replace=False):
        h = 1e-6 * tiny.demand[c]
        D1, D2 = tiny.demand.copy(), tiny.demand.copy()
        D1[c] += h
        D2[c] -= h
        fd = (O.gradient(_with(tiny, D=D1), alpha, BETA0, K)[0] - O.gradient(_with(tiny, D=D2), alpha, BETA0, K)[0]) / (2 * h)
        assert abs(fd - gD[c]) <= 1e-6 * scale, (c, fd, gD[c])


def test_objective_matches_a_separate_forward_run(tiny):
    J, _, _ = O.gradient(tiny, 1.0, BETA0, K)
    s = O.OracleSolver(tiny, alpha_target=1.0, alpha_start=1.0, beta0=BETA0, adapt_beta=False,
                       continuation=False, gamma=-1.0, scale_mode=2)
    s.run(K)
    S = O.demand_totals(tiny, s.allocation())
    assert abs(J - float(np.sum(np.log(S)))) <= 1e-12 * abs(J)


def test_checkpoint_spacing_does_not_change_the_result(tiny):
    a = O.gradient(tiny, 1.0, BETA0, K, checkpoint=20)
    b = O.gradient(tiny, 1.0, BETA0, K, checkpoint=7)
    c = O.gradient(tiny, 1.0, BETA0, K, checkpoint=1)
    assert a[0] == b[0] == c[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[1], c[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[2], c[2])


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_zero_iterations_closed_form(tiny, alpha):
    J, gC, gD = O.gradient(tiny, alpha, BETA0, 0)
    assert abs(J - float(np.sum(O.utility(tiny.demand, alpha)))) <= 1e-12 * abs(J)
    assert np.abs(gC).max() == 0.0
    assert np.allclose(gD, tiny.demand ** (-alpha), rtol=1e-14, atol=0)


def _fd_golden():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fd_medium_alpha1_K200.json")
    return json.load(open(path))


def test_oracle_adjoint_matches_central_differences_medium():
    """The differentiated configuration (200-node workload, alpha = 1, K = 200,
    checkpoints every 20): the oracle's reverse pass against FP64 central
    differences at relative step 1e-3 on 50 seeded coordinates
    (tests/golden/fd_medium_alpha1_K200.json, written by
    tests/golden/make_fd_medium.py from the oracle's forward runs).  The map
    after K iterations is piecewise smooth (active paths, binding caps and
    positive prices switch), so a step of 1e-3 can cross a kink: every
    coordinate agrees within 2e-3 of the largest derivative, and the typical
    one (the median) to the differences' truncation error."""
    from paper_2605_01748_b300 import instances
    d = _fd_golden()
    inst = instances.make_medium(seed=0)
    J, gC, gD = O.gradient(inst, d["alpha"], d["beta0"], d["K"], checkpoint=20)
    assert abs(J - d["J"]) <= 1e-9 * abs(d["J"])
    fd = np.array([c["fd"] for c in d["coords"]])
    g = np.array([gC[c["index"]] if c["kind"] == "C" else gD[c["index"]] for c in d["coords"]])
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g - fd)) <= 2e-3 * scale
    rel = np.abs(g - fd) / np.maximum(np.abs(fd), 1e-3 * scale)
    assert np.median(rel) <= 1e-5
