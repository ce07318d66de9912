"""ctypes wrapper of the FP64 CPU oracle (te_oracle.c) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  It shares nothing with the CUDA library: the two
only see the same generated instance arrays.

Functions (all FP64; paper references are to GATE, Section 3 and Appendix B):

* :func:`solve` / :class:`OracleSolver` -- the ADMM iteration of Algorithm 1
  with residual balancing (Eq. 17), the stop rule (Eq. 18) and
  alpha-continuation (Section 3.4).
* :func:`demand_solve` -- one per-demand x-block subproblem (Appendix B.2).
* :func:`run_expanded` -- the same iteration with every consensus copy
  y_{e,r} and dual u_{e,r} kept per incidence (Eqs. 5-7, 10, 13).
* :func:`project` -- the feasibility projection (Algorithm 2).
* :func:`project_scale` -- a proportional feasibility scaling (not in the
  paper; scales where Algorithm 2 trims whole paths).
* :func:`gap` -- the Lagrangian duality gap of a feasible allocation.
* :func:`maxmin_single_path` -- exact max-min fair rates of single-path
  demands (progressive filling), the exact optimum of the k = 1 variants.
* :func:`gradient` -- the fairness objective after K fixed-schedule
  iterations and its gradient in capacities and demands (reverse mode,
  checkpointed; not in the paper).
* :func:`optimality` -- the optimality metric of Section 4.1.
* :func:`literal_run` -- the update equations of Section 3.3 as printed, run
  as a multi-block iteration (an ablation; numpy).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "te_oracle.c")
_LIB = os.path.join(_HERE, "libteoracle.so")

TRACE_WIDTH = 5  # r, s, beta, alpha, event bits (1 beta change, 2 alpha step, 4/8/16 stop)


def build(force: bool = False) -> str:
    """Compile te_oracle.c with gcc (FP64, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + res.stderr)
    return _LIB


class _Inst(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int32), ("n_demands", ctypes.c_int32),
                ("n_paths", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("cap", ctypes.c_void_p), ("demand", ctypes.c_void_p),
                ("dpo", ctypes.c_void_p), ("peo", ctypes.c_void_p), ("pe", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("alpha_target", ctypes.c_double), ("alpha_start", ctypes.c_double),
                ("alpha_step", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("gamma", ctypes.c_double), ("gamma_max", ctypes.c_double), ("A", ctypes.c_double),
                ("C", ctypes.c_double),
                ("beta0", ctypes.c_double), ("beta_max", ctypes.c_double), ("balance_floor", ctypes.c_double),
                ("adapt_beta", ctypes.c_int32),
                ("continuation", ctypes.c_int32), ("threads", ctypes.c_int32), ("scale_mode", ctypes.c_int32)]


class _Scalars(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("alpha", ctypes.c_double), ("scale", ctypes.c_double),
                ("beta0", ctypes.c_double), ("iter", ctypes.c_int64), ("iter_alpha", ctypes.c_int64),
                ("converged", ctypes.c_int32), ("pad", ctypes.c_int32)]


_lib: Optional[ctypes.CDLL] = None


def _L() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.or_init.restype = ctypes.c_int
        lib.or_init.argtypes = [P, P, P, P, P, P, P]
        lib.or_run.restype = ctypes.c_int64
        lib.or_run.argtypes = [P, P, P, P, P, P, ctypes.c_int64, P]
        lib.or_demand_solve.restype = ctypes.c_double
        lib.or_demand_solve.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double, P]
        lib.or_run_expanded.restype = None
        lib.or_run_expanded.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P,
                                        ctypes.c_int64]
        lib.or_project.restype = None
        lib.or_project.argtypes = [P, P, ctypes.c_double]
        lib.or_maxmin_single_path.restype = ctypes.c_int
        lib.or_maxmin_single_path.argtypes = [P, P]
        lib.or_gradient.restype = ctypes.c_int
        lib.or_gradient.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P]
        lib.or_project_scale.restype = None
        lib.or_project_scale.argtypes = [P, P]
        lib.or_gap.restype = ctypes.c_double
        lib.or_gap.argtypes = [P, P, P, ctypes.c_double, P, P]
        lib.or_utility.restype = ctypes.c_double
        lib.or_utility.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


class _InstanceView:
    """Keeps contiguous copies of the arrays alive while C holds pointers."""

    def __init__(self, inst):
        self.cap = _c(inst.capacity, np.float64)
        self.demand = _c(inst.demand, np.float64)
        self.dpo = _c(inst.demand_path_off, np.int64)
        self.peo = _c(inst.path_edge_off, np.int64)
        self.pe = _c(inst.path_edges, np.int32)
        self.s = _Inst(self.cap.shape[0], self.demand.shape[0], self.peo.shape[0] - 1, self.pe.shape[0],
                       self.cap.ctypes.data, self.demand.ctypes.data, self.dpo.ctypes.data,
                       self.peo.ctypes.data, self.pe.ctypes.data)


def utility(S, alpha: float):
    """alpha-fair utility U_alpha (Eq. 4), elementwise."""
    S = np.asarray(S, dtype=np.float64)
    return np.vectorize(lambda v: _L().or_utility(float(v), float(alpha)))(S)


class OracleSolver:
    """Stateful FP64 solver: ``run(n)`` advances up to n iterations."""

    def __init__(self, inst, alpha_target: float = math.inf, gamma: float = 1e-3, A: float = 10.0,
                 C: float = 2.0, beta0: float = 0.0, adapt_beta: bool = True, continuation: bool = True,
                 alpha_start: float = 0.0, alpha_step: float = 1.0, alpha_max: float = 32.0,
                 threads: int = 0, x0: Optional[np.ndarray] = None, scale_mode: int = 1,
                 balance_floor: float = 1e-6, gamma_max: float = 0.0, beta_max: float = 0.0):
        """Defaults: the paper's A = 10, C = 2, gamma = 1e-3 (Section 3.7),
        alpha from 0 in steps of 1 (Algorithm 1); the unit of the normalised
        problem is the geometric mean of the demands (scale_mode = 1) and
        beta0 <= 0 picks 1 / (mean path length * mean initial path rate);
        residual balancing pauses while both residuals are at or below
        balance_floor."""
        self.inst = inst
        self.view = _InstanceView(inst)
        self.opts = _Opts(alpha_target, alpha_start, alpha_step, alpha_max, gamma, gamma_max, A, C, beta0,
                          float(beta_max), float(balance_floor), int(adapt_beta), int(continuation), int(threads),
                          int(scale_mode))
        self.x = np.zeros(inst.n_paths, dtype=np.float64)
        self.u = np.zeros(inst.n_edges, dtype=np.float64)
        self.d = np.zeros(inst.n_edges, dtype=np.float64)
        self.sc = _Scalars()
        x0c = None if x0 is None else _c(x0, np.float64)
        rc = _L().or_init(ctypes.byref(self.view.s), ctypes.byref(self.opts),
                          None if x0c is None else x0c.ctypes.data, self.x.ctypes.data,
                          self.u.ctypes.data, self.d.ctypes.data, ctypes.byref(self.sc))
        if rc != 0:
            raise ValueError("oracle init failed (no positive capacity)")
        self.trace = np.zeros((0, TRACE_WIDTH))

    def run(self, max_iters: int) -> int:
        tr = np.zeros((max(int(max_iters), 1), TRACE_WIDTH), dtype=np.float64)
        n = _L().or_run(ctypes.byref(self.view.s), ctypes.byref(self.opts), self.x.ctypes.data,
                        self.u.ctypes.data, self.d.ctypes.data, ctypes.byref(self.sc), int(max_iters),
                        tr.ctypes.data)
        self.trace = np.concatenate([self.trace, tr[:n]])
        return int(n)

    # state accessors (caller units unless stated)
    @property
    def scale(self) -> float:
        return self.sc.scale

    @property
    def beta(self) -> float:
        return self.sc.beta

    @property
    def alpha(self) -> float:
        return self.sc.alpha

    @property
    def iters(self) -> int:
        return int(self.sc.iter)

    @property
    def converged(self) -> bool:
        return bool(self.sc.converged)

    def allocation(self) -> np.ndarray:
        return self.x * self.scale

    def prices(self) -> np.ndarray:
        """Capacity prices p_e = beta u_e in caller units (U' scales as scale^-alpha)."""
        return self.sc.beta * self.u * self.scale ** (-self.sc.alpha)


def solve(inst, max_iters: int = 10000, **kw) -> OracleSolver:
    s = OracleSolver(inst, **kw)
    s.run(max_iters)
    return s


def demand_solve(m: np.ndarray, w: np.ndarray, D: float, alpha: float):
    """Per-demand x-block: returns (lambda, x)."""
    m = _c(m, np.float64)
    w = _c(w, np.float64)
    x = np.zeros_like(m)
    lam = _L().or_demand_solve(int(m.shape[0]), m.ctypes.data, w.ctypes.data, float(D), float(alpha),
                               x.ctypes.data)
    return lam, x


def run_expanded(inst, beta: float, alpha: float, iters: int, scale: Optional[float] = None):
    """Per-incidence ADMM from the default start: returns (x, y, u) normalised
    by `scale` (default max_e C_e)."""
    v = _InstanceView(inst)
    scale = float(np.max(inst.capacity)) if scale is None else float(scale)
    npaths = np.diff(inst.demand_path_off)
    x = np.repeat(inst.demand / scale / npaths, npaths).astype(np.float64)
    plen = np.diff(inst.path_edge_off)
    y = np.repeat(x, plen).astype(np.float64)
    u = np.zeros(inst.nnz, dtype=np.float64)
    _L().or_run_expanded(ctypes.byref(v.s), float(beta), float(alpha), scale, x.ctypes.data, y.ctypes.data,
                         u.ctypes.data, int(iters))
    return x, y, u


def project(inst, x: np.ndarray, alpha: float) -> np.ndarray:
    """Algorithm 2 on a copy of x (caller units)."""
    v = _InstanceView(inst)
    out = np.array(x, dtype=np.float64, copy=True)
    _L().or_project(ctypes.byref(v.s), out.ctypes.data, float(alpha))
    return out


def project_scale(inst, x: np.ndarray) -> np.ndarray:
    """Proportional feasibility scaling (not in the paper) on a copy of x
    (caller units): clamp at 0, scale each over-served demand down to D_c,
    then scale each path by min over its edges of min(1, C_e / L_e)."""
    v = _InstanceView(inst)
    out = np.array(x, dtype=np.float64, copy=True)
    _L().or_project_scale(ctypes.byref(v.s), out.ctypes.data)
    return out


def maxmin_single_path(inst) -> np.ndarray:
    """Exact max-min fair demand rates when every demand has one path
    (progressive filling), caller units."""
    view = _InstanceView(inst)
    rate = np.zeros(inst.n_demands, dtype=np.float64)
    if _L().or_maxmin_single_path(ctypes.byref(view.s), rate.ctypes.data) != 0:
        raise ValueError("maxmin_single_path needs exactly one path per demand")
    return rate


def gradient(inst, alpha: float, beta0: float, iters: int, checkpoint: int = 20, scale_mode: int = 2,
             threads: int = 0):
    """(J, dJ/dC, dJ/dD) of J = sum_c U_alpha(S_c) after `iters` iterations
    of the fixed schedule (beta0, alpha fixed) from the initial state, the
    normalisation unit held fixed (scale_mode 2: caller units)."""
    view = _InstanceView(inst)
    opts = _Opts(alpha, alpha, 1.0, alpha, -1.0, 0.0, 10.0, 2.0, beta0, 0.0, 1e-6, 0, 0, int(threads), int(scale_mode))
    J = ctypes.c_double()
    gC = np.zeros(inst.n_edges, dtype=np.float64)
    gD = np.zeros(inst.n_demands, dtype=np.float64)
    rc = _L().or_gradient(ctypes.byref(view.s), ctypes.byref(opts), int(iters), int(checkpoint), ctypes.byref(J),
                          gC.ctypes.data, gD.ctypes.data)
    if rc != 0:
        raise ValueError("or_gradient: bad options")
    return J.value, gC, gD


def gap(inst, x: np.ndarray, prices: np.ndarray, alpha: float):
    """(gap, primal, dual) of a feasible x under edge prices p >= 0 (caller units)."""
    v = _InstanceView(inst)
    xc = _c(x, np.float64)
    pc = _c(prices, np.float64)
    pr = ctypes.c_double()
    du = ctypes.c_double()
    g = _L().or_gap(ctypes.byref(v.s), xc.ctypes.data, pc.ctypes.data, float(alpha), ctypes.byref(pr),
                    ctypes.byref(du))
    return float(g), float(pr.value), float(du.value)


def demand_totals(inst, x: np.ndarray) -> np.ndarray:
    """S_c = sum of x over each demand's paths."""
    return np.add.reduceat(np.asarray(x, dtype=np.float64), inst.demand_path_off[:-1]) \
        if inst.n_demands else np.zeros(0)


def edge_loads(inst, x: np.ndarray) -> np.ndarray:
    """L_e = sum of x over the paths through e."""
    plen = np.diff(inst.path_edge_off)
    return np.bincount(inst.path_edges, weights=np.repeat(np.asarray(x, dtype=np.float64), plen),
                       minlength=inst.n_edges)


def optimality(S: np.ndarray, opt: np.ndarray, theta: float) -> float:
    """Section 4.1: mean over demands of min(S_d / max(OPT_d, theta), 1)."""
    S = np.asarray(S, dtype=np.float64)
    opt = np.asarray(opt, dtype=np.float64)
    return float(np.mean(np.minimum(S / np.maximum(opt, theta), 1.0)))


def literal_run(inst, alpha: float, beta: float, iters: int) -> np.ndarray:
    """The update equations of Section 3.3 as printed, run as a multi-block
    iteration in Algorithm 1's order from its start (x = D_c/|P_c|, y = x on
    every incidence, all duals zero), normalised by the geometric mean of the
    demands; returns the path rates in caller units.  Per iteration, from the
    previous x, y and duals: dual-updates-dem/cap/con/neg, the per-incidence
    cost of penalty-b and the rate suggestion y = [(mean_e cost - cost) /
    beta]_+, and eq. rate-computation x_r = (Q_r + U'(S)/beta - (S - D +
    dual_dem) + dual_neg_r) / (1 + n_r) with Q_r = sum_{e in r} (y - dual_con)
    and S the demand's total solved from the sum of that formula (closed form
    at alpha = 0, bisection otherwise).  An ablation: as printed the capacity
    cancels in the rate suggestion.  numpy, FP64; sums in index order."""
    scale = float(np.exp(np.mean(np.log(inst.demand))))
    C = inst.capacity / scale
    D = inst.demand / scale
    P, K = inst.n_paths, inst.n_demands
    plen = np.diff(inst.path_edge_off)
    inc_path = np.repeat(np.arange(P), plen)          # path of each incidence
    inc_edge = inst.path_edges.astype(np.int64)       # edge of each incidence
    path_dem = np.repeat(np.arange(K), np.diff(inst.demand_path_off))
    n_e = np.bincount(inc_edge, minlength=inst.n_edges).astype(np.float64)
    x = np.repeat(D / np.diff(inst.demand_path_off), np.diff(inst.demand_path_off))
    y = x[inc_path].copy()
    d_dem = np.zeros(K)
    d_cap = np.zeros(inst.n_edges)
    d_con = np.zeros(inc_edge.shape[0])
    d_neg = np.zeros(P)
    w = 1.0 / (1.0 + plen)
    for _ in range(iters):
        S = np.bincount(path_dem, weights=x, minlength=K)
        # dual updates from x^k, y^k
        d_dem_n = np.maximum(d_dem + (S - D), 0.0)
        d_cap_n = np.maximum(d_cap + (np.bincount(inc_edge, weights=y, minlength=inst.n_edges) - C), 0.0)
        d_con_n = np.maximum(d_con + (x[inc_path] - y), 0.0)
        d_neg_n = np.maximum(d_neg - x, 0.0)
        # rate suggestions
        cost = beta * (-C[inc_edge] - x[inc_path]) - d_cap_n[inc_edge] - d_con_n
        mean_e = np.bincount(inc_edge, weights=cost, minlength=inst.n_edges) / np.maximum(n_e, 1.0)
        y_n = np.maximum((mean_e[inc_edge] - cost) / beta, 0.0)
        # rate computation from the previous y and duals
        Q = np.bincount(inc_path, weights=y - d_con, minlength=P)
        a = np.bincount(path_dem, weights=w * (Q + d_neg), minlength=K)
        W = np.bincount(path_dem, weights=w, minlength=K)
        # S (1 + W) = a + W (D - d_dem) + W S^-alpha / beta, solved by bisection (the
        # right side falls as S grows for alpha > 0; alpha = 0 is linear)
        rhs0 = a + W * (D - d_dem)
        if alpha == 0.0:
            S_new = (rhs0 + W / beta) / (1.0 + W)
        else:
            lo = np.full(K, 1e-12)
            hi = np.maximum(1.0, np.abs(rhs0) + W / beta) * 10.0 + 1.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                f = mid * (1.0 + W) - rhs0 - W * mid ** (-alpha) / beta
                lo = np.where(f < 0, mid, lo)
                hi = np.where(f < 0, hi, mid)
            S_new = 0.5 * (lo + hi)
        Sp = S_new[path_dem]
        x = w * (Q + Sp ** (-alpha) / beta - (Sp - D[path_dem] + d_dem[path_dem]) + d_neg) if alpha > 0.0 else \
            w * (Q + 1.0 / beta - (Sp - D[path_dem] + d_dem[path_dem]) + d_neg)
        y, d_dem, d_cap, d_con, d_neg = y_n, d_dem_n, d_cap_n, d_con_n, d_neg_n
    return x * scale
