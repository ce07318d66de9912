"""The C-ABI library on a host without a GPU: it loads, exports every entry
point that include/te.h declares, fills the paper's default options, and
rejects invalid instances in te_create before touching a device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2605_01748_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def te():
    build.build_te()
    from paper_2605_01748_b300 import te as te_mod
    return te_mod


def _declared():
    src = open(os.path.join(ROOT, "include", "te.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(te_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(te):
    names = _declared()
    assert "te_create" in names and "te_solve" in names and "te_gap" in names
    lib = ctypes.CDLL(te.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(te.EXPORTED)


def test_default_options_match_paper(te):
    o = te.te_default_options()
    assert math.isinf(o.alpha_target) and o.alpha_start == 0.0 and o.alpha_step == 1.0
    assert o.gamma == 1e-3 and o.A == 10.0 and o.C == 2.0
    assert o.adapt_beta == 1 and o.continuation == 1 and o.test_withhold_cta == 0
    assert o.scale_mode == 1 and o.beta0 == 0.0


def _broken(tiny, **changes):
    import dataclasses
    return dataclasses.replace(tiny, **changes)


@pytest.mark.parametrize("case", ["zero_demand", "nan_capacity", "edge_out_of_range", "empty_path",
                                  "bad_offsets", "zero_cap_on_path", "not_a_walk", "too_many_paths"])
def test_create_rejects_invalid_instances(te, tiny, case):
    if case == "zero_demand":
        d = tiny.demand.copy(); d[5] = 0.0
        inst = _broken(tiny, demand=d)
    elif case == "nan_capacity":
        c = tiny.capacity.copy(); c[3] = np.nan
        inst = _broken(tiny, capacity=c)
    elif case == "edge_out_of_range":
        pe = tiny.path_edges.copy(); pe[10] = tiny.n_edges
        inst = _broken(tiny, path_edges=pe)
    elif case == "empty_path":
        peo = tiny.path_edge_off.copy(); peo[2] = peo[1]
        inst = _broken(tiny, path_edge_off=peo)
    elif case == "bad_offsets":
        dpo = tiny.demand_path_off.copy(); dpo[-1] += 1
        inst = _broken(tiny, demand_path_off=dpo)
    elif case == "zero_cap_on_path":
        c = tiny.capacity.copy(); c[tiny.path_edges[0]] = 0.0
        inst = _broken(tiny, capacity=c)
    elif case == "not_a_walk":
        pe = tiny.path_edges.copy()
        r = int(np.argmax(np.diff(tiny.path_edge_off) >= 2))
        i0 = tiny.path_edge_off[r]
        pe[i0], pe[i0 + 1] = pe[i0 + 1], pe[i0]
        inst = _broken(tiny, path_edges=pe)
    else:
        from paper_2605_01748_b300.instances import Instance
        n = 40
        inst = Instance("wide", 2, np.array([0], np.int32), np.array([1], np.int32), np.array([1.0]),
                        np.array([0], np.int32), np.array([1], np.int32), np.array([1.0]),
                        np.array([0, n], np.int64), np.arange(n + 1, dtype=np.int64),
                        np.zeros(n, np.int32), {})
    with pytest.raises(te.TEError) as ei:
        te.te_create(inst)
    assert ei.value.status in (te.TE_EINVAL, te.TE_EUNSUPPORTED)
    assert str(ei.value)


def test_options_struct_matches_header(te, tmp_path):
    """The ctypes mirror of te_options, te_solve_result and te_layout_info has
    the C header's size and field offsets (compiled here with gcc)."""
    fields = {"te_options": [f for f, _ in te.te_options._fields_],
              "te_solve_result": [f for f, _ in te.te_solve_result._fields_],
              "te_layout_info": [f for f, _ in te.te_layout_info._fields_],
              "te_batch_info_t": [f for f, _ in te.te_batch_info_t._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "te.h"', 'int main(void) {']
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for st, fs in fields.items():
        cls = getattr(te, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_default_options_deterministic_fp32(te):
    o = te.te_default_options()
    assert o.deterministic == 1 and o.precision == te.PRECISION_FP32


def test_create_rejects_unsupported_precision(te, tiny):
    # options are checked on the host before any device work
    with pytest.raises(te.TEError) as ei:
        te.te_create(tiny, te.te_default_options(precision=1))
    assert ei.value.status == te.TE_EUNSUPPORTED
    with pytest.raises(te.TEError) as ei:
        te.te_create(tiny, te.te_default_options(deterministic=2))
    assert ei.value.status == te.TE_EINVAL


def test_edge_mode_default_and_checked(te, tiny):
    o = te.te_default_options()
    assert o.edge_mode == te.EDGES_AUTO
    with pytest.raises(te.TEError) as ei:
        te.te_create(tiny, te.te_default_options(edge_mode=2))
    assert ei.value.status == te.TE_EINVAL


def test_literal_run_checks_arguments_on_the_host(te, tiny):
    # argument and instance checks come before any device work
    for alpha, beta, iters in ((-1.0, 1.0, 10), (1.0, 0.0, 10), (1.0, 1.0, -1)):
        with pytest.raises(te.TEError) as ei:
            te.te_literal_run(tiny, alpha, beta, iters)
        assert ei.value.status == te.TE_EINVAL
    import dataclasses
    bad = dataclasses.replace(tiny, demand=-tiny.demand)
    with pytest.raises(te.TEError) as ei:
        te.te_literal_run(bad, 1.0, 1.0, 10)
    assert ei.value.status == te.TE_EINVAL and "demand" in str(ei.value)


def test_solve_rejects_null_handle(te):
    res = te.te_solve_result()
    assert te.lib().te_solve(None, 10, -1.0, ctypes.byref(res)) == te.TE_EINVAL
