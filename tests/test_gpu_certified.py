"""The alpha-fair objective (Eq. 4, fixed alpha) against its exact optimum on
the GPU, through the C-ABI.

The duality gap of Section 3.1's problem (weak duality of Eqs. 1-4, tight by
Slater's condition, Appendix C) brackets the exact optimum between the
objective of the feasible, proportionally scaled allocation and the
Lagrangian dual at the solver's prices, so bench.certified_eps bounds the
distance to the optimum without a reference solve; its CPU pins in
test_bench_host.py check it against closed-form and LP optima.  Here the
GPU path must reach a certificate of 1e-3 on the 200-node workload, the
certificate it computes must equal the oracle's FP64 evaluation of the same
allocation and prices, and at alpha = 0 the 12-node solve must land within
1e-3 of the exact LP optimum.
"""
import numpy as np
import pytest

import bench
import refsolvers as R
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_certificate_within_1e3_medium(te, medium, alpha):
    t = te.TE(medium, alpha_target=alpha, alpha_start=alpha, continuation=0, gamma=-1.0)
    eps, n = np.inf, 0
    while n < 12000:
        n = t.solve(500)["total_iters"]
        g, pr, du = t.gap(project=te.PROJECT_SCALE)
        eps = bench.certified_eps(g, pr, du, alpha, medium.n_demands)
        if eps <= 1e-3:
            break
    assert eps <= 1e-3, (n, eps)
    # the certificate is the oracle's FP64 gap of the same allocation and
    # prices; the allocation comes back in FP32 caller units, whose rounding
    # (2^-24 of each rate) moves a utility term by about U'(S) S 2^-24
    xs = t.allocation(project=te.PROJECT_SCALE).astype(np.float64)
    go, pro, duo = O.gap(medium, xs, t.prices(), alpha)
    S = O.demand_totals(medium, xs)
    fp32_rates = 2.0 ** -21 * float(np.sum(S ** (1.0 - alpha)))
    assert abs(pr - pro) <= fp32_rates, (pr, pro, fp32_rates)
    assert abs(du - duo) <= 1e-7 * abs(duo), (du, duo)
    assert bench.certified_eps(go, pro, duo, alpha, medium.n_demands) <= 1.1e-3
    loads = O.edge_loads(medium, xs)
    assert (xs >= 0).all() and (loads <= medium.capacity * (1 + 1e-5)).all()
    t.close()


def test_alpha0_objective_within_1e3_of_lp_tiny(te, tiny):
    lp, _ = R.lp_max_flow(tiny)
    t = te.TE(tiny, alpha_target=0.0, alpha_start=0.0, continuation=0, gamma=-1.0)
    t.solve(2000)
    xs = t.allocation(project=te.PROJECT_SCALE).astype(np.float64)
    thr = float(xs.sum())
    assert thr <= lp * (1 + 1e-6)
    assert (lp - thr) / lp <= 1e-3, (lp, thr)
    g, pr, du = t.gap(project=te.PROJECT_SCALE)
    assert (lp - thr) / lp <= bench.certified_eps(g, pr, du, 0.0, tiny.n_demands) + 1e-6
    t.close()
