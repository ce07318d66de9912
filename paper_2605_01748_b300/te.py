"""Python binding of libte.so (include/te.h): argument marshalling only.

Every step of the TE iteration runs inside libte's CUDA kernels; this module
only turns NumPy arrays and torch CUDA tensors into pointers.  Importing it
loads libte.so and fails loudly when the library has not been built
(``python -m paper_2605_01748_b300.build``); there is no CPU fallback.

The functions mirror the C entry points one to one (``te_create``,
``te_solve``, ``te_allocation``, ``te_gap``, ``te_gap_projected``, ``te_prices``,
``te_set_warm_start``, ``te_reset``, ``te_trace``, ``te_layout``,
``te_destroy``, ``te_last_error``); :class:`TE` bundles a handle with them.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TE_LIBRARY may name another build of the same library (e.g. a variant
# compiled with different launch parameters)
LIB_PATH = os.environ.get("TE_LIBRARY") or os.path.join(_HERE, "libte.so")

TE_OK, TE_EINVAL, TE_ENOMEM, TE_ECUDA, TE_ETIMEOUT, TE_ENUMERIC, TE_ENOTCONVERGED, TE_EUNSUPPORTED = range(8)
# feasibility step of te_allocation: none, Algorithm 2, proportional scaling (not in the paper)
PROJECT_NONE, PROJECT_ALG2, PROJECT_SCALE = 0, 1, 2
# te_options.precision
PRECISION_FP32 = 0
# te_options.edge_mode: per-edge arrays of the iteration kernel in shared memory when they fit, or always global
EDGES_AUTO, EDGES_GLOBAL = 0, 1
STATUS_NAMES = {0: "TE_OK", 1: "TE_EINVAL", 2: "TE_ENOMEM", 3: "TE_ECUDA", 4: "TE_ETIMEOUT",
                5: "TE_ENUMERIC", 6: "TE_ENOTCONVERGED", 7: "TE_EUNSUPPORTED"}

EXPORTED = ("te_default_options", "te_create", "te_solve", "te_allocation", "te_gap", "te_gap_projected",
            "te_prices", "te_set_warm_start", "te_set_demands", "te_set_capacities", "te_reset", "te_trace", "te_layout",
            "te_destroy", "te_last_error", "te_gap_noalloc", "te_batch_create", "te_batch_solve",
            "te_batch_allocation", "te_batch_reset", "te_batch_info", "te_batch_destroy", "te_batch_last_error",
            "te_gradient", "te_literal_run")


class TEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class te_topology(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("edge_src", ctypes.c_void_p), ("edge_dst", ctypes.c_void_p)]


class te_paths(ctypes.Structure):
    _fields_ = [("n_demands", ctypes.c_int32), ("pad_", ctypes.c_int32), ("n_paths", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("demand_src", ctypes.c_void_p), ("demand_dst", ctypes.c_void_p),
                ("demand_path_off", ctypes.c_void_p), ("path_edge_off", ctypes.c_void_p),
                ("path_edges", ctypes.c_void_p)]


class te_options(ctypes.Structure):
    _fields_ = [("alpha_target", ctypes.c_double), ("alpha_start", ctypes.c_double),
                ("alpha_step", ctypes.c_double), ("alpha_max", ctypes.c_double), ("gamma", ctypes.c_double), ("gamma_max", ctypes.c_double),
                ("A", ctypes.c_double), ("C", ctypes.c_double), ("beta0", ctypes.c_double),
                ("beta_max", ctypes.c_double), ("balance_floor", ctypes.c_double),
                ("adapt_beta", ctypes.c_int32), ("continuation", ctypes.c_int32),
                ("scale_mode", ctypes.c_int32), ("wait_timeout_ms", ctypes.c_int32),
                ("test_withhold_cta", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("edge_mode", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p)]


class te_solve_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("total_iters", ctypes.c_int64), ("r", ctypes.c_double),
                ("s", ctypes.c_double), ("beta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("converged", ctypes.c_int32), ("stop_reason", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class te_layout_info(ctypes.Structure):
    _fields_ = [("n_demands", ctypes.c_int64), ("n_paths", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("id_rows", ctypes.c_int64), ("slots", ctypes.c_int64), ("id_bytes", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("bytes_per_iter", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("edges_global", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class te_batch_info_t(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int64), ("n_paths", ctypes.c_int64), ("id_rows", ctypes.c_int64),
                ("bytes_per_iter", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("lanes_per_demand", ctypes.c_int32),
                ("ctas_per_instance", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2605_01748_b300.build` "
                          "(the TE engine has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    H = ctypes.c_void_p
    lib.te_default_options.restype = None
    lib.te_default_options.argtypes = [ctypes.POINTER(te_options)]
    lib.te_create.restype = ctypes.c_int
    lib.te_create.argtypes = [ctypes.POINTER(te_topology), ctypes.POINTER(te_paths), P, P,
                              ctypes.POINTER(te_options), ctypes.POINTER(H)]
    lib.te_solve.restype = ctypes.c_int
    lib.te_solve.argtypes = [H, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(te_solve_result)]
    lib.te_allocation.restype = ctypes.c_int
    lib.te_allocation.argtypes = [H, P, ctypes.c_int32, ctypes.c_int32]
    lib.te_gap.restype = ctypes.c_int
    lib.te_gap.argtypes = [H, P, P, P]
    lib.te_gap_projected.restype = ctypes.c_int
    lib.te_gap_projected.argtypes = [H, ctypes.c_int32, P, P, P]
    lib.te_prices.restype = ctypes.c_int
    lib.te_prices.argtypes = [H, P, ctypes.c_int32]
    lib.te_set_warm_start.restype = ctypes.c_int
    lib.te_set_warm_start.argtypes = [H, P, ctypes.c_int32, ctypes.c_int32]
    lib.te_set_demands.restype = ctypes.c_int
    lib.te_set_demands.argtypes = [H, P, ctypes.c_int32]
    lib.te_set_capacities.restype = ctypes.c_int
    lib.te_set_capacities.argtypes = [H, P, ctypes.c_int32]
    lib.te_reset.restype = ctypes.c_int
    lib.te_reset.argtypes = [H]
    lib.te_trace.restype = ctypes.c_int
    lib.te_trace.argtypes = [H, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.te_layout.restype = ctypes.c_int
    lib.te_layout.argtypes = [H, ctypes.POINTER(te_layout_info)]
    lib.te_destroy.restype = None
    lib.te_destroy.argtypes = [H]
    lib.te_last_error.restype = ctypes.c_char_p
    lib.te_last_error.argtypes = [H]
    lib.te_gradient.restype = ctypes.c_int
    lib.te_gradient.argtypes = [H, ctypes.c_int64, ctypes.c_int32, P, P, P, ctypes.c_int32]
    lib.te_batch_create.restype = ctypes.c_int
    lib.te_batch_create.argtypes = [P, ctypes.c_int32, P, P, P, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.te_batch_solve.restype = ctypes.c_int
    lib.te_batch_solve.argtypes = [H, ctypes.c_int64, P]
    lib.te_batch_allocation.restype = ctypes.c_int
    lib.te_batch_allocation.argtypes = [H, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32]
    lib.te_batch_reset.restype = ctypes.c_int
    lib.te_batch_reset.argtypes = [H]
    lib.te_batch_info.restype = ctypes.c_int
    lib.te_batch_info.argtypes = [H, ctypes.POINTER(te_batch_info_t)]
    lib.te_batch_destroy.restype = None
    lib.te_batch_destroy.argtypes = [H]
    lib.te_batch_last_error.restype = ctypes.c_char_p
    lib.te_batch_last_error.argtypes = [H]
    lib.te_literal_run.restype = ctypes.c_int
    lib.te_literal_run.argtypes = [ctypes.POINTER(te_topology), ctypes.POINTER(te_paths), P, P, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, P, ctypes.c_void_p]
    lib.te_gap_noalloc.restype = ctypes.c_int
    lib.te_gap_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                   P, P, P, P, P, P, P, ctypes.c_double, P, P]
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _ptr(a) -> int:
    """Pointer of a NumPy array or a torch tensor (host or device)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _is_device(a) -> bool:
    return bool(getattr(a, "is_cuda", False))


def te_last_error(h) -> str:
    msg = _lib.te_last_error(h)
    return msg.decode() if msg else ""


def _check(status: int, h) -> None:
    if status != TE_OK:
        raise TEError(status, te_last_error(h))


def te_default_options(**overrides) -> te_options:
    o = te_options()
    _lib.te_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        setattr(o, k, v)
    return o


class _Keep:
    """Holds contiguous copies of the inputs while te_create reads them."""

    def __init__(self, inst):
        c = np.ascontiguousarray
        self.edge_src = c(inst.edge_src, dtype=np.int32)
        self.edge_dst = c(inst.edge_dst, dtype=np.int32)
        self.capacity = c(inst.capacity, dtype=np.float64)
        self.demand_src = c(inst.demand_src, dtype=np.int32)
        self.demand_dst = c(inst.demand_dst, dtype=np.int32)
        self.demand = c(inst.demand, dtype=np.float64)
        self.dpo = c(inst.demand_path_off, dtype=np.int64)
        self.peo = c(inst.path_edge_off, dtype=np.int64)
        self.pe = c(inst.path_edges, dtype=np.int32)


def te_create(inst, options: Optional[te_options] = None, check_walks: bool = True):
    """Creates a handle from an instance (any object with the fields of
    paper_2605_01748_b300.instances.Instance)."""
    k = _Keep(inst)
    topo = te_topology(int(inst.n_nodes), k.capacity.shape[0], _ptr(k.edge_src) if check_walks else 0,
                       _ptr(k.edge_dst) if check_walks else 0)
    paths = te_paths(k.demand.shape[0], 0, k.peo.shape[0] - 1, k.pe.shape[0],
                     _ptr(k.demand_src) if check_walks else 0, _ptr(k.demand_dst) if check_walks else 0,
                     _ptr(k.dpo), _ptr(k.peo), _ptr(k.pe))
    h = ctypes.c_void_p()
    opts = options if options is not None else te_default_options()
    st = _lib.te_create(ctypes.byref(topo), ctypes.byref(paths), _ptr(k.demand), _ptr(k.capacity),
                        ctypes.byref(opts), ctypes.byref(h))
    if st != TE_OK:
        raise TEError(st, te_last_error(None))
    return h


def te_literal_run(inst, alpha: float, beta: float, iters: int, cuda_stream=None) -> np.ndarray:
    """The printed multi-block update equations run on the device for iters
    iterations from Algorithm 1's start (an ablation, see include/te.h);
    returns the path rates in caller units (FP64, caller path order)."""
    k = _Keep(inst)
    topo = te_topology(int(inst.n_nodes), k.capacity.shape[0], _ptr(k.edge_src), _ptr(k.edge_dst))
    paths = te_paths(k.demand.shape[0], 0, k.peo.shape[0] - 1, k.pe.shape[0], _ptr(k.demand_src),
                     _ptr(k.demand_dst), _ptr(k.dpo), _ptr(k.peo), _ptr(k.pe))
    x = np.empty(k.peo.shape[0] - 1, dtype=np.float64)
    stream = int(getattr(cuda_stream, "cuda_stream", cuda_stream) or 0)
    st = _lib.te_literal_run(ctypes.byref(topo), ctypes.byref(paths), _ptr(k.demand), _ptr(k.capacity),
                             float(alpha), float(beta), int(iters), _ptr(x), stream)
    if st != TE_OK:
        raise TEError(st, te_last_error(None))
    return x


def te_solve(h, max_iters: int, tol: float = -1.0) -> te_solve_result:
    """Up to max_iters iterations; tol is this call's stop threshold gamma
    (negative: the handle's te_options.gamma)."""
    res = te_solve_result()
    _check(_lib.te_solve(h, int(max_iters), float(tol), ctypes.byref(res)), h)
    return res


def te_allocation(h, out, project: int = PROJECT_ALG2) -> None:
    """Writes rates (caller path order, FP32) into `out`: a NumPy float32
    array or a torch float32 CUDA tensor of n_paths entries.  `project` is
    one of PROJECT_NONE, PROJECT_ALG2, PROJECT_SCALE (True/False map to
    PROJECT_ALG2/PROJECT_NONE)."""
    _check(_lib.te_allocation(h, _ptr(out), int(project), int(_is_device(out))), h)


def te_gap(h):
    g, p, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.te_gap(h, ctypes.byref(g), ctypes.byref(p), ctypes.byref(d)), h)
    return g.value, p.value, d.value


def te_gap_projected(h, project: int):
    """(gap, primal, dual) of te_gap with the feasibility step `project`
    (PROJECT_ALG2 or PROJECT_SCALE)."""
    g, p, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.te_gap_projected(h, int(project), ctypes.byref(g), ctypes.byref(p), ctypes.byref(d)), h)
    return g.value, p.value, d.value


def te_prices(h, out) -> None:
    _check(_lib.te_prices(h, _ptr(out), int(_is_device(out))), h)


def te_set_warm_start(h, x0, keep_duals: bool = False) -> None:
    _check(_lib.te_set_warm_start(h, _ptr(x0), int(_is_device(x0)), int(bool(keep_duals))), h)


def _f64_host(a):
    return a if _is_device(a) or hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=np.float64)


def te_set_demands(h, demands) -> None:
    """demands: FP64 NumPy array (host) or torch float64 tensor (host or CUDA)."""
    demands = _f64_host(demands)
    _check(_lib.te_set_demands(h, _ptr(demands), int(_is_device(demands))), h)


def te_set_capacities(h, capacities) -> None:
    """capacities: FP64 NumPy array (host) or torch float64 tensor (host or CUDA)."""
    capacities = _f64_host(capacities)
    _check(_lib.te_set_capacities(h, _ptr(capacities), int(_is_device(capacities))), h)


def te_reset(h) -> None:
    _check(_lib.te_reset(h), h)


def te_trace(h, max_rows: int) -> np.ndarray:
    out = np.zeros((max(int(max_rows), 0), 5), dtype=np.float64)
    n = ctypes.c_int64()
    _check(_lib.te_trace(h, _ptr(out) if max_rows > 0 else 0, int(max_rows), ctypes.byref(n)), h)
    return out[:n.value]


def te_layout(h) -> dict:
    info = te_layout_info()
    _check(_lib.te_layout(h, ctypes.byref(info)), h)
    return info.as_dict()


def te_gap_noalloc(demand_path_off, path_edge_off, path_edges, demands, capacities, x, prices, alpha: float,
                   out, stream=None) -> None:
    """Duality gap without any allocation (see te.h): every argument is a
    torch CUDA tensor the caller owns (int64, int64, int32, float64,
    float64, float32, float64); out is a float64 CUDA tensor of 3 entries
    that receives {gap, primal, dual}.  Queued on `stream` (a torch stream,
    default: the current one); nothing is synchronised here.  For callers
    that cannot allocate device memory where they need the gap."""
    for name, t in (("demand_path_off", demand_path_off), ("path_edge_off", path_edge_off),
                    ("path_edges", path_edges), ("demands", demands), ("capacities", capacities),
                    ("x", x), ("prices", prices), ("out", out)):
        if not _is_device(t):
            raise TEError(TE_EINVAL, f"te_gap_noalloc: {name} must be a device tensor")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    st = _lib.te_gap_noalloc(int(capacities.shape[0]), int(demands.shape[0]), int(x.shape[0]),
                             int(path_edges.shape[0]), _ptr(demand_path_off), _ptr(path_edge_off),
                             _ptr(path_edges), _ptr(demands), _ptr(capacities), _ptr(x), _ptr(prices),
                             float(alpha), _ptr(out), int(getattr(stream, "cuda_stream", stream)))
    if st == TE_EUNSUPPORTED:
        raise TEError(st, "te_gap_noalloc: ceil(n_demands/256) + ceil(n_edges/256) exceeds the 16384 "
                          "slots of its static scratch (about 4.19 million demands)")
    if st != TE_OK:
        raise TEError(st, "te_gap_noalloc failed")


def te_destroy(h) -> None:
    _lib.te_destroy(h)


class TE:
    """One TE instance resident on the current CUDA device."""

    def __init__(self, inst, **options):
        self.n_paths = int(inst.n_paths)
        self.n_edges = int(inst.n_edges)
        self.n_demands = int(inst.n_demands)
        self.options = te_default_options(**options)
        self.h = te_create(inst, self.options)

    def solve(self, max_iters: int, tol: float = -1.0) -> dict:
        return te_solve(self.h, max_iters, tol).as_dict()

    def allocation(self, project: int = PROJECT_ALG2, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.n_paths, dtype=np.float32)
        te_allocation(self.h, out, project)
        return out

    def gap(self, project: int = PROJECT_ALG2):
        """(gap, primal, dual); project selects the feasibility step applied
        before the primal utility (PROJECT_ALG2 as te_gap, or PROJECT_SCALE)."""
        if project == PROJECT_ALG2:
            return te_gap(self.h)
        return te_gap_projected(self.h, project)

    def prices(self, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.n_edges, dtype=np.float64)
        te_prices(self.h, out)
        return out

    def warm_start(self, x0, keep_duals: bool = False) -> None:
        te_set_warm_start(self.h, x0, keep_duals)

    def set_demands(self, demands) -> None:
        te_set_demands(self.h, demands)

    def set_capacities(self, capacities) -> None:
        te_set_capacities(self.h, capacities)

    def gradient(self, iters: int, checkpoint: int = 20):
        """(J, dJ/dC [n_edges], dJ/dD [n_demands]) of J = sum_c U_alpha(S_c)
        after `iters` fixed-schedule iterations from the initial state (the
        handle must use the fixed schedule; see te_gradient)."""
        J = ctypes.c_double()
        gC = np.zeros(self.n_edges, dtype=np.float64)
        gD = np.zeros(self.n_demands, dtype=np.float64)
        _check(_lib.te_gradient(self.h, int(iters), int(checkpoint), ctypes.byref(J), _ptr(gC), _ptr(gD), 0), self.h)
        return J.value, gC, gD

    def reset(self) -> None:
        te_reset(self.h)

    def trace(self, max_rows: int = 1 << 16) -> np.ndarray:
        return te_trace(self.h, max_rows)

    def layout(self) -> dict:
        return te_layout(self.h)

    def close(self) -> None:
        if self.h:
            te_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TEBatch:
    """A batch of instances over one topology (same edge numbering), solved
    together by the batch kernel: one instance per CTA, one launch."""

    def __init__(self, insts, **options):
        self.n = len(insts)
        self._keep = [_Keep(i) for i in insts]
        k0 = self._keep[0]
        self.topo = te_topology(int(insts[0].n_nodes), k0.capacity.shape[0], 0, 0)
        self.paths = (te_paths * self.n)()
        for i, k in enumerate(self._keep):
            self.paths[i] = te_paths(k.demand.shape[0], 0, k.peo.shape[0] - 1, k.pe.shape[0], 0, 0,
                                     _ptr(k.dpo), _ptr(k.peo), _ptr(k.pe))
        self._pp = (ctypes.c_void_p * self.n)(*[ctypes.addressof(self.paths[i]) for i in range(self.n)])
        self._dp = (ctypes.c_void_p * self.n)(*[_ptr(k.demand) for k in self._keep])
        self._cp = (ctypes.c_void_p * self.n)(*[_ptr(k.capacity) for k in self._keep])
        self.n_paths = [int(k.peo.shape[0] - 1) for k in self._keep]
        self.options = te_default_options(**options)
        h = ctypes.c_void_p()
        st = _lib.te_batch_create(ctypes.byref(self.topo), self.n, self._pp, self._dp, self._cp,
                                  ctypes.byref(self.options), ctypes.byref(h))
        if st != TE_OK:
            raise TEError(st, (_lib.te_batch_last_error(None) or b"").decode())
        self.h = h

    def _check(self, st):
        if st != TE_OK:
            raise TEError(st, (_lib.te_batch_last_error(self.h) or b"").decode())

    def solve(self, max_iters: int) -> list:
        res = (te_solve_result * self.n)()
        self._check(_lib.te_batch_solve(self.h, int(max_iters), res))
        return [r.as_dict() for r in res]

    def allocation(self, i: int, project: int = PROJECT_ALG2, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.n_paths[i], dtype=np.float32)
        self._check(_lib.te_batch_allocation(self.h, int(i), _ptr(out), int(project), int(_is_device(out))))
        return out

    def reset(self) -> None:
        self._check(_lib.te_batch_reset(self.h))

    def info(self) -> dict:
        info = te_batch_info_t()
        self._check(_lib.te_batch_info(self.h, ctypes.byref(info)))
        return info.as_dict()

    def close(self) -> None:
        if getattr(self, "h", None):
            _lib.te_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_objective(inst, alpha: float, beta0: float, iters: int, checkpoint: int = 20, **options):
    """A torch.autograd.Function over (capacities, demands) -> J = sum_c
    U_alpha(S_c) after `iters` fixed-schedule iterations (caller units),
    whose backward is the library's hand-written reverse pass (te_gradient).
    Each call builds a handle for the given capacities and demands."""
    import torch
    from .instances import Instance

    class _Objective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, C, D):
            I = Instance(inst.name, inst.n_nodes, inst.edge_src, inst.edge_dst,
                         C.detach().double().cpu().numpy(), inst.demand_src, inst.demand_dst,
                         D.detach().double().cpu().numpy(), inst.demand_path_off, inst.path_edge_off,
                         inst.path_edges, dict(inst.meta))
            t = TE(I, alpha_target=alpha, alpha_start=alpha, beta0=beta0, adapt_beta=0, continuation=0,
                   gamma=-1.0, scale_mode=2, **options)
            J, gC, gD = t.gradient(iters, checkpoint)
            t.close()
            ctx.save_for_backward(torch.from_numpy(gC).to(C.device, C.dtype), torch.from_numpy(gD).to(D.device, D.dtype))
            return torch.tensor(J, dtype=C.dtype, device=C.device)

        @staticmethod
        def backward(ctx, gJ):
            gC, gD = ctx.saved_tensors
            return gJ * gC, gJ * gD

    return _Objective.apply
