"""The loop-chain program format shared by the synthetic workloads.

A chain is what an OPS application enqueues between two flushes: a block,
its datasets (dats) with halos, stencils, reduction handles and a sequence of
parallel loops (Sec. 3, Sec. 4.A).  Each loop carries an iteration range, an
argument list (dat + stencil + access mode, or a reduction / scalar handle)
and a body written in a small register IR instead of a function pointer.

This module only *describes* programs (numbers and enums of the interchange
format); it evaluates nothing.  Both the CPU oracle and the CUDA library
decode this format with their own code.

IR encoding: a body is an int32 array of shape (n, 6), one instruction per
row `(op, d, a, b, c, e)`, plus a float64 constant pool.  Eight registers
r0..r7 per grid point start at +0.0.  `v(arg, p)` is the value of the dat of
argument `arg` at the current point shifted by point `p` of that argument's
stencil.

    LD   d a b      r[d] = v(a, b)            (a SCALAR arg: its value; b = 0)
    CST  d a        r[d] = K[a]
    ADD  d a b      r[d] = r[a] + r[b]
    SUB  d a b      r[d] = r[a] - r[b]
    MUL  d a b      r[d] = r[a] * r[b]
    FMA  d a b c    r[d] = fma(r[a], r[b], r[c])   (one rounding)
    DIV  d a b      r[d] = r[a] / r[b]
    MIN  d a b      r[d] = r[b] if r[b] < r[a] else r[a]
    MAX  d a b      r[d] = r[b] if r[b] > r[a] else r[a]
    SGT  d a b c e  r[d] = r[c] if r[a] > r[b] else r[e]
    WSUM d a b      r[d] = K[b]*v(a,0); then r[d] = fma(K[b+p], v(a,p), r[d]) for p = 1..np-1
    WACC d a b      r[d] = fma(K[b+p], v(a,p), r[d]) for p = 0..np-1
    POLY d a b c    t = K[b+c]; t = fma(t, r[a], K[b+i]) for i = c-1..0; r[d] = t
    ST   d a        arg d (WRITE or RW): dat = r[a];  arg d (INC): dat = dat + r[a]
    RED  d a        reduction arg d takes the contribution r[a]
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# opcodes
LD, CST, ADD, SUB, MUL, FMA, DIV, MIN, MAX, SGT, WSUM, WACC, POLY, ST, RED = range(1, 16)
OPNAMES = {1: "LD", 2: "CST", 3: "ADD", 4: "SUB", 5: "MUL", 6: "FMA", 7: "DIV", 8: "MIN",
           9: "MAX", 10: "SGT", 11: "WSUM", 12: "WACC", 13: "POLY", 14: "ST", 15: "RED"}
NREG = 8

# argument kinds and access modes
DAT, SCALAR, REDARG = 0, 1, 2
READ, WRITE, RW, INC = 0, 1, 2, 3
# reduction operators
RSUM, RMIN, RMAX = 0, 1, 2


@dataclass
class Arg:
    kind: int          # DAT, SCALAR or REDARG
    handle: int        # dat index, or reduction index (SCALAR reads a reduction's value)
    stencil: int = -1  # stencil index for DAT args
    access: int = READ


@dataclass
class Loop:
    name: str
    rng: Tuple[Tuple[int, int], ...]     # per dimension [lo, hi)
    args: List[Arg]
    code: np.ndarray                     # int32 (n, 6)
    consts: np.ndarray                   # float64
    dt_slot: int = -1                    # constant slot that the host fills each step
    dt_scale: float = 0.0                #   with dt_scale * (last value of the dt reduction)

    def consts_for(self, dt: float) -> np.ndarray:
        k = self.consts.copy()
        if self.dt_slot >= 0:
            k[self.dt_slot] = self.dt_scale * dt
        return k


@dataclass
class DatSpec:
    name: str
    init: np.ndarray   # dense float64, shape (ez, ey, ex) of the allocated box incl. halos


@dataclass
class Chain:
    """A block with its dats and one step's loop sequence, repeated `steps` times.

    After every step the host reads every reduction (a flush, Sec. 4.A); the
    value of reduction `dt_red` becomes the next step's dt (1.0 for step 0).
    """
    name: str
    ndim: int
    size: Tuple[int, int, int]
    d_m: Tuple[int, int, int]
    d_p: Tuple[int, int, int]
    dats: List[DatSpec]
    stencils: List[List[Tuple[int, int, int]]]
    reductions: List[int]
    loops: List[Loop]
    steps: int = 1
    dt_red: int = -1
    meta: dict = field(default_factory=dict)

    @property
    def ext(self) -> Tuple[int, int, int]:
        return tuple(self.size[d] + self.d_m[d] + self.d_p[d] for d in range(3))


class BodyBuilder:
    """Tiny assembler for the register IR."""

    def __init__(self):
        self.code: List[List[int]] = []
        self.consts: List[float] = []

    def k(self, *vals: float) -> int:
        base = len(self.consts)
        self.consts.extend(float(v) for v in vals)
        return base

    def emit(self, op: int, d: int = 0, a: int = 0, b: int = 0, c: int = 0, e: int = 0):
        self.code.append([op, d, a, b, c, e])
        return self

    def ld(self, d, arg, pt=0):
        return self.emit(LD, d, arg, pt)

    def cst(self, d, value):
        return self.emit(CST, d, self.k(value))

    def wsum(self, d, arg, weights: Sequence[float]):
        return self.emit(WSUM, d, arg, self.k(*weights))

    def wacc(self, d, arg, weights: Sequence[float]):
        return self.emit(WACC, d, arg, self.k(*weights))

    def poly(self, d, a, coefs: Sequence[float]):
        return self.emit(POLY, d, a, self.k(*coefs), len(coefs) - 1)

    def st(self, arg, r):
        return self.emit(ST, arg, r)

    def red(self, arg, r):
        return self.emit(RED, arg, r)

    def build(self) -> Tuple[np.ndarray, np.ndarray]:
        code = np.asarray(self.code, dtype=np.int32).reshape(-1, 6)
        consts = np.asarray(self.consts if self.consts else [0.0], dtype=np.float64)
        return code, consts


def stencil_extent(points: Sequence[Tuple[int, int, int]], d: int) -> Tuple[int, int]:
    """(most negative offset or 0, most positive offset or 0) along dimension d."""
    lo = min(0, min(p[d] for p in points))
    hi = max(0, max(p[d] for p in points))
    return lo, hi


def untiled_bytes(chain: Chain, loops: Optional[Sequence[Loop]] = None) -> int:
    """Bytes moved per step by the paper's accounting (Sec. 6.A): every dat
    argument of a loop costs 8 B per point of its range, RW counts twice,
    stencil re-use within a loop is ignored."""
    total = 0
    for lp in (chain.loops if loops is None else loops):
        pts = 1
        for lo, hi in lp.rng:
            pts *= max(0, hi - lo)
        nacc = 0
        for a in lp.args:
            if a.kind != DAT:
                continue
            nacc += 2 if a.access in (RW, INC) else 1
        total += pts * nacc * 8
    return total


def body_flops(lp: Loop, chain: Chain) -> int:
    """Floating-point operations per grid point of one loop body: an fma
    counts 2, add/sub/mul/div/min/max/compare count 1, an INC store adds 1."""
    f = 0
    for op, d, a, b, c, e in lp.code.tolist():
        if op in (ADD, SUB, MUL, DIV, MIN, MAX, SGT):
            f += 1
        elif op == FMA:
            f += 2
        elif op in (WSUM, WACC):
            npts = len(chain.stencils[lp.args[a].stencil])
            f += 2 * npts - (1 if op == WSUM else 0)
        elif op == POLY:
            f += 2 * c
        elif op == ST and lp.args[d].access == INC:
            f += 1
        elif op == RED:
            f += 1
    return f


def loop_points(lp: Loop) -> int:
    n = 1
    for lo, hi in lp.rng:
        n *= max(0, hi - lo)
    return n
