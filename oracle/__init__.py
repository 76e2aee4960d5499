"""CPU oracle for run-time loop-chain tiling (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library: the
interpreter is `oracle.c` (built here with gcc), the tiling plans are the
plain Python restatements in `oracle.plan`.

Layout used by the oracle: each dat is a dense float64 array of shape
(ez, ey, ex) over its allocated box, halos included, x fastest; grid point
(0, 0, 0) sits at index (d_m[2], d_m[1], d_m[0]).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            L.ora_fsum.restype = C.c_double
            L.ora_fsum.argtypes = [P(C.c_double), C.c_int64]
            L.ora_run_loops.restype = C.c_int
            L.ora_cg64.restype = C.c_int
            L.ora_cg_refine.restype = C.c_int
            L.ora_relres.restype = C.c_double
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _fp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def fsum(x) -> float:
    """Exactly rounded sum of a float64 vector."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    return lib().ora_fsum(_dp(a), a.size)


# ---------------------------------------------------------------------------
# chain execution
# ---------------------------------------------------------------------------
class OracleError(RuntimeError):
    pass


def _rng6(lp, ndim: int) -> List[int]:
    out = []
    for d in range(3):
        if d < ndim:
            out += [int(lp.rng[d][0]), int(lp.rng[d][1])]
        else:
            out += [0, 1]
    return out


def run_loops(chain, dats: List[np.ndarray], loops: Sequence, red_vals: List[float],
              nthreads: int = 0) -> List[float]:
    """Run `loops` in program order on `dats` (modified in place); returns the
    reduction values after the loops, starting from `red_vals`."""
    L = lib()
    nd = len(dats)
    f32 = nd > 0 and dats[0].dtype == np.float32
    for a in dats:
        assert a.dtype == (np.float32 if f32 else np.float64) and a.flags.c_contiguous
    ptrs = (C.POINTER(C.c_double) * max(nd, 1))(*[C.cast(a.ctypes.data, C.POINTER(C.c_double)) for a in dats])
    ext = np.array([[a.shape[2], a.shape[1], a.shape[0]] for a in dats], dtype=np.int32).ravel()
    dm = np.array([list(chain.d_m) for _ in dats], dtype=np.int32).ravel()
    st_npts = np.array([len(s) for s in chain.stencils], dtype=np.int32)
    st_start = np.concatenate([[0], np.cumsum(st_npts)[:-1]]).astype(np.int32)
    st_off = np.array([list(p) for s in chain.stencils for p in s], dtype=np.int32).ravel()
    red_op = np.array(chain.reductions if chain.reductions else [0], dtype=np.int32)
    red_val = np.array(list(red_vals) if red_vals else [0.0], dtype=np.float64)
    nl = len(loops)
    rngs = np.array([_rng6(lp, chain.ndim) for lp in loops], dtype=np.int32).ravel()
    nargs = np.array([len(lp.args) for lp in loops], dtype=np.int32)
    arg0 = np.concatenate([[0], np.cumsum(nargs)[:-1]]).astype(np.int32)
    args = np.array([[a.kind, a.handle, a.stencil, a.access] for lp in loops for a in lp.args],
                    dtype=np.int32).ravel()
    nins = np.array([lp.code.shape[0] for lp in loops], dtype=np.int32)
    ins0 = np.concatenate([[0], np.cumsum(nins)[:-1]]).astype(np.int32)
    ins = np.ascontiguousarray(np.concatenate([lp.code for lp in loops]).astype(np.int32).ravel())
    consts = [getattr(lp, "_consts_now", lp.consts) for lp in loops]
    nk = np.array([len(k) for k in consts], dtype=np.int32)
    k0 = np.concatenate([[0], np.cumsum(nk)[:-1]]).astype(np.int32)
    K = np.ascontiguousarray(np.concatenate(consts).astype(np.float64))
    err = C.create_string_buffer(256)
    rc = L.ora_run_loops(C.c_int(nd), ptrs, _ip(ext), _ip(dm), _ip(st_npts), _ip(st_start), _ip(st_off),
                         C.c_int(len(chain.reductions)), _ip(red_op), _dp(red_val),
                         C.c_int(nl), _ip(rngs), _ip(nargs), _ip(arg0), _ip(args), _ip(nins), _ip(ins0),
                         _ip(ins), _ip(k0), _ip(nk), _dp(K), C.c_int(nthreads), C.c_int(1 if f32 else 0), err)
    if rc != 0:
        raise OracleError(err.value.decode())
    return [float(v) for v in red_val[:len(chain.reductions)]]


def red_identity(op: int) -> float:
    return 0.0 if op == 0 else (np.inf if op == 1 else -np.inf)


def run_chain(chain, steps: Optional[int] = None, nthreads: int = 0, fp32: bool = False):
    """Run the chain's steps untiled in program order.

    Returns (dats, history): the final dats (dense arrays) and, per step,
    the reduction values the host reads at the end of that step.  fp32: the
    dats start as the initial values rounded to float and every operation
    is an IEEE single one."""
    dats = [np.ascontiguousarray(d.init.astype(np.float32 if fp32 else np.float64)) for d in chain.dats]
    nsteps = chain.steps if steps is None else steps
    dt = 1.0
    hist = []
    for s in range(nsteps):
        loops = []
        for lp in chain.loops:
            lp2 = _with_consts(lp, lp.consts_for(dt))
            loops.append(lp2)
        vals = run_loops(chain, dats, loops, [red_identity(op) for op in chain.reductions], nthreads)
        hist.append(vals)
        if chain.dt_red >= 0:
            dt = vals[chain.dt_red]
    return dats, hist


def run_chain_tiled(chain, tile: Sequence[int], steps: Optional[int] = None, nthreads: int = 0,
                    fp32: bool = False):
    """The paper's CPU execution of the same steps: each step's loops get
    Algorithm 1's skewed ranges (oracle.plan.skewed_plan) for the tile sizes
    `tile`, then run as Algorithm 2 does, tile by tile in lexicographic
    order (x fastest) and loop by loop within a tile, with the rows of each
    (tile, loop) box spread over the host cores.  Every point is evaluated
    as in run_chain and reductions are exact, so the results are identical."""
    from . import plan as oplan
    import itertools
    dats = [np.ascontiguousarray(d.init.astype(np.float32 if fp32 else np.float64)) for d in chain.dats]
    nsteps = chain.steps if steps is None else steps
    nd = chain.ndim
    dt = 1.0
    hist = []
    for s in range(nsteps):
        loops = [_with_consts(lp, lp.consts_for(dt)) for lp in chain.loops]
        ntiles, ranges, _ = oplan.skewed_plan(loops, chain.stencils, nd, list(tile)[:nd])
        phases = []
        for rev in itertools.product(*[range(ntiles[d]) for d in reversed(range(nd))]):
            t = tuple(reversed(rev))
            for l, lp in enumerate(loops):
                box = [ranges[d][t[d]][l] for d in range(nd)]
                if all(hi > lo for lo, hi in box):
                    phases.append(_BoxView(lp, box))
        vals = run_loops(chain, dats, phases, [red_identity(op) for op in chain.reductions], nthreads)
        hist.append(vals)
        if chain.dt_red >= 0:
            dt = vals[chain.dt_red]
    return dats, hist


def run_chain_wavefront(chain, tile: Sequence[int], steps: Optional[int] = None, seed: int = 0,
                        fp32: bool = False, drop=None):
    """The phases of each step's skewed plan (Algorithm 1 ranges for the tile
    sizes `tile`) executed in a random order that keeps every pair of
    conflicting phases (oracle.plan.phase_conflicts) in plan order: at each
    point one of the phases whose earlier conflicting phases are all done is
    drawn at random.  This is the freedom a wavefront schedule of the tiles
    uses (Sec. 4.B leaves such schedules to future work); the results are
    those of program order.  drop(q, deps) -> deps, if given, edits the
    dependency list of phase q before the order is drawn (tests use it to
    show that the relation is needed)."""
    import random
    from . import plan as oplan
    rnd = random.Random(seed)
    dats = [np.ascontiguousarray(d.init.astype(np.float32 if fp32 else np.float64)) for d in chain.dats]
    nsteps = chain.steps if steps is None else steps
    nd = chain.ndim
    dt = 1.0
    hist = []
    for s in range(nsteps):
        loops = [_with_consts(lp, lp.consts_for(dt)) for lp in chain.loops]
        ntiles, ranges, _ = oplan.skewed_plan(loops, chain.stencils, nd, list(tile)[:nd])
        phases = oplan.phases_in_order(loops, ntiles, ranges, nd)
        deps = oplan.phase_conflicts(loops, chain.stencils, nd, phases)
        if drop is not None:
            deps = [drop(q, list(d)) for q, d in enumerate(deps)]
        waiting = [len(d) for d in deps]
        users = [[] for _ in phases]
        for q, d in enumerate(deps):
            for p in d:
                users[p].append(q)
        ready = [q for q in range(len(phases)) if waiting[q] == 0]
        order = []
        while ready:
            q = ready.pop(rnd.randrange(len(ready)))
            order.append(q)
            for u in users[q]:
                waiting[u] -= 1
                if waiting[u] == 0:
                    ready.append(u)
        assert len(order) == len(phases)
        views = [_BoxView(loops[phases[q][0]], phases[q][1]) for q in order]
        vals = run_loops(chain, dats, views, [red_identity(op) for op in chain.reductions])
        hist.append(vals)
        if chain.dt_red >= 0:
            dt = vals[chain.dt_red]
    return dats, hist


class _BoxView:
    """A loop restricted to one (tile, loop) box."""

    def __init__(self, lp, box):
        self._lp = lp
        self.rng = tuple(box)

    def __getattr__(self, k):
        return getattr(self._lp, k)


class _LoopView:
    def __init__(self, lp, consts):
        self._lp = lp
        self._consts_now = consts

    def __getattr__(self, k):
        return getattr(self._lp, k)


def _with_consts(lp, consts):
    return _LoopView(lp, consts)


# ---------------------------------------------------------------------------
# heat-conduction CG (configs 4 and 5)
# ---------------------------------------------------------------------------
def faces(kappa: np.ndarray):
    n = kappa.shape[0]
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    kx = np.zeros((n, n + 1))
    ky = np.zeros((n + 1, n))
    dg = np.zeros((n, n))
    lib().ora_faces(C.c_int(n), _dp(k), _dp(kx), _dp(ky), _dp(dg))
    return kx, ky, dg


def matvec(kappa: np.ndarray, u: np.ndarray) -> np.ndarray:
    n = kappa.shape[0]
    kx, ky, dg = faces(kappa)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros((n, n))
    lib().ora_matvec(C.c_int(n), _dp(kx), _dp(ky), _dp(dg), _dp(uu), _dp(w))
    return w


def matvec32(kappa: np.ndarray, u: np.ndarray) -> np.ndarray:
    """The FP32 operator: FP64 faces rounded to float, u rounded to float,
    the same term order with single-rounding float fma; result widened."""
    n = kappa.shape[0]
    kx, ky, dg = faces(kappa)
    kxf = np.ascontiguousarray(kx, dtype=np.float32)
    kyf = np.ascontiguousarray(ky, dtype=np.float32)
    dgf = np.ascontiguousarray(dg, dtype=np.float32)
    uf = np.ascontiguousarray(u, dtype=np.float32)
    w = np.zeros((n, n), dtype=np.float32)
    lib().ora_matvec32(C.c_int(n), _fp(kxf), _fp(kyf), _fp(dgf), _fp(uf), _fp(w))
    return w.astype(np.float64)


def cg64(kappa: np.ndarray, b: np.ndarray, tol: float, maxit: int = 100000):
    n = kappa.shape[0]
    x = np.zeros((n, n))
    rr = C.c_double()
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    it = lib().ora_cg64(C.c_int(n), _dp(k), _dp(bb), C.c_double(tol), C.c_int(maxit), _dp(x), C.byref(rr))
    return x, it, rr.value


def cg_refine(kappa: np.ndarray, b: np.ndarray, tol: float, inner_tol: float = 1e-4,
              maxit: int = 1000000, maxouter: int = 100):
    n = kappa.shape[0]
    x = np.zeros((n, n))
    rr = C.c_double()
    outer = C.c_int()
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    it = lib().ora_cg_refine(C.c_int(n), _dp(k), _dp(bb), C.c_double(tol), C.c_double(inner_tol),
                             C.c_int(maxit), C.c_int(maxouter), _dp(x), C.byref(rr), C.byref(outer))
    return x, it, rr.value, outer.value


def relres(kappa: np.ndarray, b: np.ndarray, x: np.ndarray) -> float:
    n = kappa.shape[0]
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    return lib().ora_relres(C.c_int(n), _dp(k), _dp(bb), _dp(xx))
