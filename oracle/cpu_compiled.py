"""The paper's CPU execution, compiled: loop bodies turned into C and run
untiled or tile by tile with OpenMP inside each tile (Algorithm 2 as the
paper runs it on CPUs, Sec. 4 and Sec. 6).

TEST INFRASTRUCTURE AND CPU CONTEXT ONLY (see the package docstring).  It
shares no code with the CUDA library: the C is generated here from the
chain's IR with this module's own reading of the opcodes, compiled with
gcc (-O3, -fopenmp, no FP contraction) and loaded with ctypes.  The tiles
come from oracle.plan.skewed_plan.

Every point evaluates its loop's IR in the fixed statement and term order,
with fma() where the IR has an fma, so the dats are bit-identical to the
oracle's (checked by the tests).  Reductions are accumulated per thread
(sums in plain FP64, min and max exactly) and folded in thread order, so
sums agree with the oracle's exactly rounded ones to rounding, not bit for
bit.  A schedule runs in one OpenMP parallel region: each (tile, loop)
phase is an `omp for` over the phase's rows, whose closing barrier is the
only synchronisation between phases.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build", "cpu_compiled")
_lock = threading.Lock()
_libs = {}

LD, CST, ADD, SUB, MUL, FMA, DIV, MIN, MAX, SGT, WSUM, WACC, POLY, ST, RED = range(1, 16)
K_DAT, K_SCALAR, K_RED = 0, 1, 2
A_READ, A_WRITE, A_RW, A_INC = 0, 1, 2, 3
R_SUM, R_MIN, R_MAX = 0, 1, 2


def _body(lp, stencils, l: int) -> List[str]:
    """C statements of loop l's IR at the point whose flat index is `c`."""
    out = ["double " + ", ".join(f"r{i} = 0.0" for i in range(8)) + ";"]

    def v(a, p):
        arg = lp.args[a]
        dx, dy, dz = stencils[arg.stencil][p]
        return f"d{arg.handle}[c + ({dx}) + ({dy}) * pitch + ({dz}) * plane]"

    for row in lp.code:
        op, d, a, b, cc, e = (int(x) for x in row)
        if op == LD:
            if lp.args[a].kind == K_SCALAR:
                out.append(f"r{d} = S[{lp.args[a].handle}];")
            else:
                out.append(f"r{d} = {v(a, b)};")
        elif op == CST:
            out.append(f"r{d} = K[{a}];")
        elif op == ADD:
            out.append(f"r{d} = r{a} + r{b};")
        elif op == SUB:
            out.append(f"r{d} = r{a} - r{b};")
        elif op == MUL:
            out.append(f"r{d} = r{a} * r{b};")
        elif op == DIV:
            out.append(f"r{d} = r{a} / r{b};")
        elif op == FMA:
            out.append(f"r{d} = fma(r{a}, r{b}, r{cc});")
        elif op == MIN:
            out.append(f"r{d} = (r{b} < r{a}) ? r{b} : r{a};")
        elif op == MAX:
            out.append(f"r{d} = (r{b} > r{a}) ? r{b} : r{a};")
        elif op == SGT:
            out.append(f"r{d} = (r{a} > r{b}) ? r{cc} : r{e};")
        elif op in (WSUM, WACC):
            n = len(stencils[lp.args[a].stencil])
            stmts = []
            q = 0
            if op == WSUM:
                stmts.append(f"double t = K[{b}] * {v(a, 0)};")
                q = 1
            else:
                stmts.append(f"double t = r{d};")
            for p in range(q, n):
                stmts.append(f"t = fma(K[{b + p}], {v(a, p)}, t);")
            stmts.append(f"r{d} = t;")
            out.append("{ " + " ".join(stmts) + " }")
        elif op == POLY:
            stmts = [f"double t = K[{b + cc}];"]
            for i in range(cc - 1, -1, -1):
                stmts.append(f"t = fma(t, r{a}, K[{b + i}]);")
            stmts.append(f"r{d} = t;")
            out.append("{ " + " ".join(stmts) + " }")
        elif op == ST:
            arg = lp.args[d]
            tgt = f"d{arg.handle}[c]"
            if arg.access == A_INC:
                out.append(f"{tgt} = {tgt} + r{a};")
            else:
                out.append(f"{tgt} = r{a};")
        elif op == RED:
            h = lp.args[d].handle
            out.append(f"red_{h}(acc, r{a});")
        else:
            raise ValueError(f"loop {l}: opcode {op}")
    return out


def generate(chain) -> str:
    """C source of one chain: a loop function per loop and a schedule runner."""
    src = ["#include <math.h>", "#include <omp.h>", "#include <stdlib.h>", "#include <string.h>", "",
           "typedef long long i64;", ""]
    ops = chain.reductions
    for h, op in enumerate(ops):
        if op == R_SUM:
            f = f"acc[{h}] = acc[{h}] + x;"
        elif op == R_MIN:
            f = f"acc[{h}] = (x < acc[{h}]) ? x : acc[{h}];"
        else:
            f = f"acc[{h}] = (x > acc[{h}]) ? x : acc[{h}];"
        src.append(f"static inline void red_{h}(double* acc, double x) {{ {f} }}")
    for l, lp in enumerate(chain.loops):
        src.append(f"static void loop_{l}(double* const* P, i64 pitch, i64 plane, const int* bx, const double* K,")
        src.append("                   const double* S, double* acc) {")
        # one restrict pointer per dat: distinct dats never overlap, and a
        # parallel loop reads no neighbour of a point it writes (Sec. 3)
        for h in sorted({a.handle for a in lp.args if a.kind == K_DAT}):
            src.append(f"  double* restrict d{h} = P[{h}];")
        src.append("  (void)S; (void)acc; (void)K;")
        src.append("  const i64 ny = bx[3] - bx[2], nz = bx[5] - bx[4];")
        src.append("#pragma omp for schedule(static) nowait")
        src.append("  for (i64 o = 0; o < ny * nz; ++o) {")
        src.append("    const i64 z = bx[4] + o / ny, y = bx[2] + o % ny;")
        src.append("    const i64 row = z * plane + y * pitch;")
        src.append("    for (i64 x = bx[0]; x < bx[1]; ++x) {")
        src.append("      const i64 c = row + x;")
        for st in _body(lp, chain.stencils, l):
            src.append("      " + st)
        src.append("    }")
        src.append("  }")
        src.append("}")
    nred = max(1, len(ops))
    src.append("")
    src.append("/* phases: (loop, x0, x1, y0, y1, z0, z1) each; K + koff[l]: loop l's constants;")
    src.append("   red: reduction values in, folded values out; every thread keeps its own partials */")
    src.append("int run_schedule(double* const* P, i64 pitch, i64 plane, const int* ph, int nph, const double* K,")
    src.append("                 const int* koff, const double* S, const int* red_op, double* red, int nthreads) {")
    src.append(f"  const int nred = {len(ops)};")
    src.append("  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();")
    src.append(f"  double* part = (double*)malloc(sizeof(double) * {nred} * (size_t)nt);")
    src.append("  for (int t = 0; t < nt; ++t)")
    src.append("    for (int h = 0; h < nred; ++h)")
    src.append(f"      part[t * {nred} + h] = red_op[h] == {R_SUM} ? 0.0 : (red_op[h] == {R_MIN} ? INFINITY : -INFINITY);")
    src.append("#pragma omp parallel num_threads(nt)")
    src.append("  {")
    src.append(f"    double* acc = part + (size_t)omp_get_thread_num() * {nred};")
    src.append("    for (int q = 0; q < nph; ++q) {")
    src.append("      const int* p = ph + 7 * q;")
    src.append("      switch (p[0]) {")
    for l in range(len(chain.loops)):
        src.append(f"        case {l}: loop_{l}(P, pitch, plane, p + 1, K + koff[{l}], S, acc); break;")
    src.append("        default: break;")
    src.append("      }")
    src.append("#pragma omp barrier")
    src.append("    }")
    src.append("  }")
    src.append("  for (int t = 0; t < nt; ++t)")
    src.append("    for (int h = 0; h < nred; ++h) {")
    src.append(f"      const double x = part[t * {nred} + h];")
    src.append(f"      if (red_op[h] == {R_SUM}) red[h] = red[h] + x;")
    src.append(f"      else if (red_op[h] == {R_MIN}) red[h] = (x < red[h]) ? x : red[h];")
    src.append("      else red[h] = (x > red[h]) ? x : red[h];")
    src.append("    }")
    src.append("  free(part);")
    src.append("  return nt;")
    src.append("}")
    return "\n".join(src) + "\n"


def _lib(chain):
    src = generate(chain)
    key = hashlib.sha256(src.encode()).hexdigest()[:16]
    with _lock:
        if key in _libs:
            return _libs[key]
        os.makedirs(_BUILD, exist_ok=True)
        so = os.path.join(_BUILD, f"chain_{key}.so")
        if not os.path.exists(so):
            c = os.path.join(_BUILD, f"chain_{key}.c")
            with open(c, "w") as f:
                f.write(src)
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                                   "-shared", "-fPIC", "-o", tmp, c, "-lm"])
            os.replace(tmp, so)
        L = C.CDLL(so)
        L.run_schedule.restype = C.c_int
        _libs[key] = L
        return L


class CompiledChain:
    """One chain compiled for the host; run() executes one step untiled (tile
    None) or tiled with Algorithm 1's ranges for the given tile sizes."""

    def __init__(self, chain, nthreads: int = 0):
        self.chain = chain
        self.lib = _lib(chain)
        self.nthreads = nthreads
        for lp in chain.loops:
            for a in lp.args:
                if a.kind == K_DAT:
                    assert a.access in (A_READ, A_WRITE, A_RW, A_INC)
        self.ops = np.array(chain.reductions if chain.reductions else [0], dtype=np.int32)
        self.threads_used = 0

    def _segments(self, loops):
        """Loop index ranges that need no flush inside: a loop reading a
        reduction that an earlier loop of the segment contributes to starts
        a new one (the value must be final when it is read)."""
        segs, start, reduced = [], 0, set()
        for i, lp in enumerate(loops):
            reads = {a.handle for a in lp.args if a.kind == K_SCALAR}
            if reads & reduced:
                segs.append((start, i))
                start, reduced = i, set()
            reduced |= {a.handle for a in lp.args if a.kind == K_RED}
        segs.append((start, len(loops)))
        return segs

    def run(self, dats: Sequence[np.ndarray], red_vals: List[float], dt: float = 1.0,
            tile: Optional[Sequence[int]] = None) -> List[float]:
        from . import plan as oplan
        ch = self.chain
        nd = ch.ndim
        for a in dats:
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == dats[0].shape
        ez, ey, ex = dats[0].shape
        pitch, plane = ex, ex * ey
        off = ch.d_m[0] + ch.d_m[1] * pitch + ch.d_m[2] * plane
        P = (C.c_void_p * len(dats))(*[a.ctypes.data + 8 * off for a in dats])
        loops = ch.loops
        consts = [lp.consts_for(dt) for lp in loops]
        koff = np.zeros(len(loops), dtype=np.int32)
        k = 0
        for i, kk in enumerate(consts):
            koff[i] = k
            k += len(kk)
        K = np.ascontiguousarray(np.concatenate(consts).astype(np.float64)) if k else np.zeros(1)
        red = np.array(list(red_vals) if red_vals else [0.0], dtype=np.float64)
        for s0, s1 in self._segments(loops):
            seg = loops[s0:s1]
            phases = []
            if tile is None:
                for j, lp in enumerate(seg):
                    b = [lp.rng[d] if d < nd else (0, 1) for d in range(3)]
                    phases.append([s0 + j] + [v for lo_hi in b for v in lo_hi])
            else:
                ntiles, ranges, _ = oplan.skewed_plan(seg, ch.stencils, nd, list(tile)[:nd])
                for l, box in oplan.phases_in_order(seg, ntiles, ranges, nd):
                    b = [box[d] if d < nd else (0, 1) for d in range(3)]
                    phases.append([s0 + l] + [v for lo_hi in b for v in lo_hi])
            ph = np.ascontiguousarray(np.array(phases, dtype=np.int32).reshape(-1))
            S = red.copy()  # scalars: the reduction values before the segment
            self.threads_used = self.lib.run_schedule(
                P, C.c_longlong(pitch), C.c_longlong(plane), ph.ctypes.data_as(C.POINTER(C.c_int)),
                C.c_int(len(phases)), K.ctypes.data_as(C.POINTER(C.c_double)),
                koff.ctypes.data_as(C.POINTER(C.c_int)), S.ctypes.data_as(C.POINTER(C.c_double)),
                self.ops.ctypes.data_as(C.POINTER(C.c_int)), red.ctypes.data_as(C.POINTER(C.c_double)),
                C.c_int(self.nthreads))
        return [float(v) for v in red[:len(ch.reductions)]]


def run_chain(chain, tile: Optional[Sequence[int]] = None, steps: Optional[int] = None, nthreads: int = 0):
    """All steps of a chain, untiled (tile None) or tiled; the dt reduction
    feeds the next step's constants as in oracle.run_chain."""
    from . import red_identity
    cc = CompiledChain(chain, nthreads)
    dats = [np.ascontiguousarray(d.init.astype(np.float64)) for d in chain.dats]
    dt = 1.0
    hist = []
    for _ in range(chain.steps if steps is None else steps):
        vals = cc.run(dats, [red_identity(op) for op in chain.reductions], dt, tile)
        hist.append(vals)
        if chain.dt_red >= 0:
            dt = vals[chain.dt_red]
    return dats, hist
