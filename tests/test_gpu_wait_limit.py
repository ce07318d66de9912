"""Bounded waits of the persistent iteration kernel, exercised without a GPU
fault: one CTA withholds its arrival at the grid barrier (the test hook of
te_options.test_withhold_cta), so every other CTA's wait runs out after
wait_timeout_ms.  The kernel must return, te_solve must report TE_ETIMEOUT,
and the context must stay usable: the handle still answers te_allocation
and a second handle solves normally and matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    from paper_2605_01748_b300 import build
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def test_withheld_barrier_arrival_times_out(te, tiny):
    bad = te.TE(tiny, gamma=-1.0, wait_timeout_ms=200, test_withhold_cta=1)  # CTA 0
    with pytest.raises(te.TEError) as err:
        bad.solve(10)
    assert err.value.status == te.TE_ETIMEOUT
    # state of the last completed iteration (here: the initial state) is kept
    npaths = np.diff(tiny.demand_path_off)
    x0 = bad.allocation(project=te.PROJECT_NONE)
    np.testing.assert_allclose(x0, np.repeat(tiny.demand / npaths, npaths), rtol=1e-6)
    bad.close()
    good = te.TE(tiny, gamma=-1.0)
    good.solve(50)
    xg = good.allocation(project=te.PROJECT_NONE)
    s = O.OracleSolver(tiny, gamma=-1.0)
    s.run(50)
    xo = s.allocation()
    assert np.max(np.abs(xg - xo)) <= 1e-4 * np.max(np.abs(xo))
    good.close()
