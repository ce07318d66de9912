"""The hand-written reverse pass on the GPU (te_gradient) against the FP64
oracle's reverse pass and against FP64 central differences of the oracle's
objective, and through torch.autograd."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_01748_b300.instances import Instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def _beta0(inst):
    """1 / (mean path length * mean initial rate), caller units."""
    return inst.n_paths ** 2 / (inst.nnz * inst.demand.sum())


def _with(inst, C=None, D=None):
    return Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst, inst.capacity if C is None else C,
                    inst.demand_src, inst.demand_dst, inst.demand if D is None else D, inst.demand_path_off,
                    inst.path_edge_off, inst.path_edges, {})


def _fixed(te, inst, alpha, beta0):
    return te.TE(inst, alpha_target=alpha, alpha_start=alpha, beta0=beta0, adapt_beta=0, continuation=0,
                 gamma=-1.0, scale_mode=2)


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_gradient_matches_oracle_tiny(te, tiny, alpha):
    K, b0 = 40, _beta0(tiny)
    t = _fixed(te, tiny, alpha, b0)
    J, gC, gD = t.gradient(K, 7)
    Jo, gCo, gDo = O.gradient(tiny, alpha, b0, K)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    g, go = np.concatenate([gC, gD]), np.concatenate([gCo, gDo])
    assert np.max(np.abs(g - go)) <= 1e-3 * np.max(np.abs(go))
    # central differences of the FP64 objective on a few coordinates
    rng = np.random.default_rng(5)
    for e in rng.choice(tiny.n_edges, 4, replace=False):
        h = 1e-6 * tiny.capacity[e]
        C1, C2 = tiny.capacity.copy(), tiny.capacity.copy()
        C1[e] += h
        C2[e] -= h
        fd = (O.gradient(_with(tiny, C=C1), alpha, b0, K)[0] - O.gradient(_with(tiny, C=C2), alpha, b0, K)[0]) / (2 * h)
        assert abs(fd - gC[e]) <= 1e-3 * np.max(np.abs(go))
    t.close()


@pytest.mark.parametrize("alpha,K", [(1.0, 200), (2.0, 100)])
def test_gradient_matches_oracle_medium(te, medium, alpha, K):
    """Differentiated form on the 200-node instance, checkpoints every 20.
    The forward pass runs in FP32 and the oracle's in FP64, so the two
    trajectories part at the level of FP32 rounding; the adjoint takes every
    branch (active path, binding cap, positive price) from the forward pass's
    own FP32 state.  Measured: rel2 about 1e-6, largest element error about
    3e-5 of the largest gradient entry."""
    b0 = _beta0(medium)
    t = _fixed(te, medium, alpha, b0)
    J, gC, gD = t.gradient(K, 20)
    Jo, gCo, gDo = O.gradient(medium, alpha, b0, K)
    assert abs(J - Jo) <= 1e-6 * abs(Jo)
    g, go = np.concatenate([gC, gD]), np.concatenate([gCo, gDo])
    rel2 = np.linalg.norm(g - go) / np.linalg.norm(go)
    assert rel2 <= 1e-4, rel2
    assert np.max(np.abs(g - go)) <= 1e-3 * np.max(np.abs(go))
    t.close()


def test_gradient_is_bit_identical_across_calls(te, medium):
    """J is summed in a fixed order and the weight adjoints as fixed-point
    integers, so two te_gradient calls on one handle return the same bits."""
    b0 = _beta0(medium)
    t = _fixed(te, medium, 1.0, b0)
    J1, gC1, gD1 = t.gradient(60, 20)
    J2, gC2, gD2 = t.gradient(60, 20)
    t.close()
    assert J1 == J2
    assert np.array_equal(np.asarray(gC1).view(np.uint64), np.asarray(gC2).view(np.uint64))
    assert np.array_equal(np.asarray(gD1).view(np.uint64), np.asarray(gD2).view(np.uint64))
    assert np.abs(gC1).max() > 0


def test_autograd_function(te, tiny):
    import torch
    K, b0 = 30, _beta0(tiny)
    f = te.make_objective(tiny, 1.0, b0, K, checkpoint=10)
    C = torch.tensor(tiny.capacity, dtype=torch.float64, requires_grad=True)
    D = torch.tensor(tiny.demand, dtype=torch.float64, requires_grad=True)
    J = f(C, D)
    J.backward()
    Jo, gCo, gDo = O.gradient(tiny, 1.0, b0, K)
    assert abs(J.item() - Jo) <= 1e-5 * abs(Jo)
    g = np.concatenate([C.grad.numpy(), D.grad.numpy()])
    go = np.concatenate([gCo, gDo])
    assert np.max(np.abs(g - go)) <= 1e-3 * np.max(np.abs(go))


def test_gradient_rejects_adaptive_schedule(te, tiny):
    t = te.TE(tiny)
    with pytest.raises(te.TEError):
        t.gradient(10)
    t.close()


def test_gradient_matches_central_differences_config5(te, medium):
    """The differentiated configuration: alpha = 1 on the 200-node workload,
    K = 200 unrolled iterations, checkpoints every 20; te_gradient against
    FP64 central differences of the oracle's objective at relative step 1e-3
    on 50 seeded coordinates of capacities and demands (tests/golden/
    fd_medium_alpha1_K200.json, from tests/golden/make_fd_medium.py).  Same
    bounds as the oracle's own reverse pass against these differences: every
    coordinate within 2e-3 of the largest derivative (a step can cross a
    kink of the piecewise-smooth map), the median to truncation error."""
    import json
    import os
    d = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "fd_medium_alpha1_K200.json")))
    t = _fixed(te, medium, d["alpha"], d["beta0"])
    J, gC, gD = t.gradient(d["K"], 20)
    t.close()
    assert abs(J - d["J"]) <= 1e-6 * abs(d["J"])
    fd = np.array([c["fd"] for c in d["coords"]])
    g = np.array([gC[c["index"]] if c["kind"] == "C" else gD[c["index"]] for c in d["coords"]])
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(g - fd)) <= 2e-3 * scale
    rel = np.abs(g - fd) / np.maximum(np.abs(fd), 1e-3 * scale)
    assert np.median(rel) <= 1e-4
