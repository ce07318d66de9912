"""te_gap_noalloc, the entry point that allocates nothing, against te_gap.

Some callers cannot allocate device memory where they need the duality gap
(for example code inside a memory pool that owns all device memory, or a
control loop that freezes its allocations after start-up).  te_gap_noalloc
serves them with a fixed static device array as its only working memory.
This test feeds it the projected allocation and the prices of a solved
handle -- exactly what te_gap evaluates -- and checks that two calls in a
row both reproduce te_gap's gap, primal and dual values.  It lives in a
file that pytest collects last so that a failure here never hides the rest
of the suite, and it passes both alone in a fresh process and after the
other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# te_gap reads the normalised FP32 iterate; te_gap_noalloc reads the same
# rates after te_allocation has scaled them to caller units and rounded them
# to FP32 again (at most 6e-8 relative each), and the FP64 sums run in a
# different order.  1e-6 relative covers both with a wide margin.
REL = 1e-6


def _close(a, b):
    if a == b:  # includes equal infinities (a starved demand at alpha >= 1)
        return True
    return abs(a - b) <= REL * max(1.0, abs(b))


@pytest.mark.parametrize("name,alpha", [("tiny", 1.0), ("tiny", 0.0), ("medium", 0.5)])
def test_gap_noalloc_matches_te_gap(name, alpha):
    import torch

    from paper_2605_01748_b300 import build, instances
    build.build_te()
    from paper_2605_01748_b300 import te

    torch.cuda.set_device(0)
    inst = instances.make(name)
    t = te.TE(inst, alpha_target=alpha, alpha_start=alpha, gamma=1e-4)
    t.solve(3000)
    g_ref, pr_ref, du_ref = t.gap()
    dev = torch.device("cuda", 0)
    xp = torch.empty(inst.n_paths, dtype=torch.float32, device=dev)
    te.te_allocation(t.h, xp, True)
    p = torch.empty(inst.n_edges, dtype=torch.float64, device=dev)
    te.te_prices(t.h, p)
    alpha_now = t.solve(0)["alpha"]
    args = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
            (inst.demand_path_off.astype(np.int64), inst.path_edge_off.astype(np.int64),
             inst.path_edges.astype(np.int32), inst.demand.astype(np.float64), inst.capacity.astype(np.float64))]
    for call in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        te.te_gap_noalloc(*args, xp, p, alpha_now, out)
        torch.cuda.synchronize()
        g, pr, du = out.cpu().tolist()
        assert _close(pr, pr_ref), (call, pr, pr_ref)
        assert _close(du, du_ref), (call, du, du_ref)
        assert abs(g - g_ref) <= REL * max(1.0, abs(pr_ref)), (call, g, g_ref)
    t.close()


def test_gap_noalloc_rejects_oversized_input():
    import torch

    from paper_2605_01748_b300 import te
    dev = torch.device("cuda", 0)
    z64 = torch.zeros(2, dtype=torch.int64, device=dev)
    z32 = torch.zeros(1, dtype=torch.int32, device=dev)
    d = torch.ones(1, dtype=torch.float64, device=dev)
    x = torch.zeros(1, dtype=torch.float32, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    # sizes are checked before any pointer is read: claim 5 million demands
    st = te.lib().te_gap_noalloc(1, 5_000_000, 5_000_000, 5_000_000, te._ptr(z64), te._ptr(z64), te._ptr(z32),
                                 te._ptr(d), te._ptr(d), te._ptr(x), te._ptr(d), 1.0, te._ptr(out), 0)
    assert st == te.TE_EUNSUPPORTED


_RESET_CHILD = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2605_01748_b300 import instances, te

rt = ctypes.CDLL("libcudart.so.13")  # the runtime that libte.so links
rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
rt.cudaFree.argtypes = [ctypes.c_void_p]
inst = instances.make_tiny()
t = te.TE(inst, alpha_target=1.0, alpha_start=1.0, gamma=1e-4)
t.solve(3000)
ref = list(t.gap())
xp = t.allocation(project=te.PROJECT_ALG2)
p = t.prices()
alpha = t.solve(0)["alpha"]
t.close()
host = [np.ascontiguousarray(a) for a in (inst.demand_path_off.astype(np.int64),
        inst.path_edge_off.astype(np.int64), inst.path_edges.astype(np.int32), inst.demand.astype(np.float64),
        inst.capacity.astype(np.float64), xp.astype(np.float32), p.astype(np.float64),
        np.full(3, np.nan))]

def run():
    bufs = []
    for a in host:
        ptr = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(ptr), a.nbytes) == 0
        assert rt.cudaMemcpy(ptr, a.ctypes.data, a.nbytes, 1) == 0
        bufs.append(ptr)
    st = te.lib().te_gap_noalloc(inst.n_edges, inst.n_demands, inst.n_paths, int(host[2].shape[0]), *bufs[:7],
                                 float(alpha), bufs[7], None)
    assert st == 0, st
    assert rt.cudaDeviceSynchronize() == 0
    res = np.zeros(3)
    assert rt.cudaMemcpy(res.ctypes.data, bufs[7], 24, 2) == 0
    for b in bufs:
        rt.cudaFree(b)
    return res.tolist()

first = run()
assert rt.cudaDeviceReset() == 0  # ends this process's context only
second = run()
print(json.dumps({"ref": ref, "first": first, "second": second}))
"""


def test_gap_noalloc_after_device_reset():
    """After cudaDeviceReset the library's module is loaded again in a new
    context; te_gap_noalloc must look up its static array's address again
    instead of reusing the old one.  Runs in a child process that uses only
    the CUDA runtime (no torch), so resetting the device strands nothing."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _RESET_CHILD, root], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    d = json.loads(res.stdout.strip().splitlines()[-1])
    g_ref, pr_ref, du_ref = d["ref"]
    for g, pr, du in (d["first"], d["second"]):
        assert _close(pr, pr_ref) and _close(du, du_ref), d
        assert abs(g - g_ref) <= REL * max(1.0, abs(pr_ref)), d
