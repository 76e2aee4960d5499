"""Seeded synthetic loop chains shaped after the paper's workloads.

None of the applications, input decks or comparison systems of the paper is
available, so every workload here is a stand-in with the shapes of the
paper's benchmarks (Sec. 5, Sec. 6): the two-loop 1D example of Sec. 4.B, the
2D heat-equation Jacobi iteration, a small 2D chain, a CloverLeaf-2D-shaped
83-loop step and an OpenSBLI-shaped 3D Runge-Kutta step.  Structure choices
come from `random.Random(seed)`, field values from the counter-based
generator in `synth.rng`.  Nothing here evaluates a loop body.
"""
from __future__ import annotations

import math
import random
from typing import List, Sequence, Tuple

import numpy as np

from . import rng as R
from .program import (DAT, REDARG, SCALAR, READ, WRITE, RW, INC, RSUM, RMIN, RMAX,
                      ADD, SUB, MUL, MIN, MAX, SGT, FMA, Arg, BodyBuilder, Chain, DatSpec, Loop)

P0 = [(0, 0, 0)]
S5 = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
S9 = [(dx, dy, 0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
S4P = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)]
S4M = [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (-1, -1, 0)]


def _alloc_shape(size, d_m, d_p):
    return tuple(size[d] + d_m[d] + d_p[d] for d in (2, 1, 0))


def _zero_halo(a: np.ndarray, size, d_m) -> np.ndarray:
    out = np.zeros_like(a)
    sl = tuple(slice(d_m[d], d_m[d] + size[d]) for d in (2, 1, 0))
    out[sl] = a[sl]
    return out


# --------------------------------------------------------------------------
# Sec. 4.B worked example
# --------------------------------------------------------------------------
def worked_example_1d() -> Chain:
    """Two 1D loops on [0, 8): loop 1 reads dat 1 and writes dat 2; loop 2
    reads dat 2 with a 3-point stencil and writes dat 1 (Sec. 4.B, Fig. 2)."""
    size, d_m, d_p = (8, 1, 1), (1, 0, 0), (1, 0, 0)
    shp = _alloc_shape(size, d_m, d_p)
    dats = [DatSpec("dat1", R.uniform(R.subseed(R.BASE_SEED, "ex1d", 1), shp)),
            DatSpec("dat2", R.uniform(R.subseed(R.BASE_SEED, "ex1d", 2), shp))]
    st = [[(0, 0, 0)], [(-1, 0, 0), (0, 0, 0), (1, 0, 0)]]
    b1 = BodyBuilder().wsum(0, 0, [0.5]).st(1, 0)
    c1, k1 = b1.build()
    b2 = BodyBuilder().wsum(0, 0, [0.25, 0.5, 0.25]).st(1, 0)
    c2, k2 = b2.build()
    loops = [Loop("loop1", ((0, 8),), [Arg(DAT, 0, 0, READ), Arg(DAT, 1, 0, WRITE)], c1, k1),
             Loop("loop2", ((0, 8),), [Arg(DAT, 1, 1, READ), Arg(DAT, 0, 0, WRITE)], c2, k2)]
    return Chain("worked_example_1d", 1, size, d_m, d_p, dats, st, [], loops)


# --------------------------------------------------------------------------
# Sec. 5 / Sec. 6.B heat equation (Jacobi), copy variant
# --------------------------------------------------------------------------
def jacobi2d(n: int, iters: int, nu: float = 0.125, p: int = 1, q: int = 1,
             init: str = "eigen") -> Chain:
    """2D heat equation, one Dirichlet halo layer: b = a + nu * L5(a), then a = b.

    With init="eigen" the field is the Dirichlet Laplacian eigenmode
    sin(pi p (i+1)/(n+1)) sin(pi q (j+1)/(n+1)), evaluated with the host libm.
    """
    size, d_m, d_p = (n, n, 1), (1, 1, 0), (1, 1, 0)
    shp = _alloc_shape(size, d_m, d_p)
    a = np.zeros(shp)
    if init == "eigen":
        i = np.arange(n)
        sx = np.array([math.sin(math.pi * p * (k + 1) / (n + 1)) for k in i])
        sy = np.array([math.sin(math.pi * q * (k + 1) / (n + 1)) for k in i])
        a[0, 1:n + 1, 1:n + 1] = np.outer(sy, sx)
    else:
        a = _zero_halo(R.uniform(R.subseed(R.BASE_SEED, "jacobi", n), shp), size, d_m)
    dats = [DatSpec("a", a), DatSpec("b", np.zeros(shp))]
    st = [P0, S5]
    bb = BodyBuilder().wsum(0, 0, [1.0 - 4.0 * nu, nu, nu, nu, nu]).st(1, 0)
    c1, k1 = bb.build()
    bc = BodyBuilder().ld(0, 0, 0).st(1, 0)
    c2, k2 = bc.build()
    rng2 = ((0, n), (0, n))
    loops = []
    for it in range(iters):
        loops.append(Loop(f"stencil{it}", rng2, [Arg(DAT, 0, 1, READ), Arg(DAT, 1, 0, WRITE)], c1, k1))
        loops.append(Loop(f"copy{it}", rng2, [Arg(DAT, 1, 0, READ), Arg(DAT, 0, 0, WRITE)], c2, k2))
    return Chain(f"jacobi2d_{n}", 2, size, d_m, d_p, dats, st, [], loops,
                 meta=dict(nu=nu, p=p, q=q, iters=iters))


# --------------------------------------------------------------------------
# Config 1: 2D 8-loop chain, 6 dats, radius-1 stencils, zero Dirichlet halo
# --------------------------------------------------------------------------
def _dyadic_weights(rnd: random.Random, n: int, total: int = 1024) -> List[float]:
    """n positive weights k_i / 1024 with sum exactly 1."""
    cuts = sorted(rnd.sample(range(1, total), n - 1))
    parts = [b - a for a, b in zip([0] + cuts, cuts + [total])]
    return [p / total for p in parts]


def small2d(n: int = 256, reps: int = 10, seed: int = None, constant: float = None,
            nloops: int = 8, ndats: int = 6) -> Chain:
    """8 loops, each reading 1-3 of 6 dats through a 5- or 9-point radius-1
    stencil and writing one other dat as a weighted sum with total |w| <= 1.

    constant=c fills every dat and halo with c and uses positive dyadic
    weights summing to exactly 1 (a constant-preservation case)."""
    seed = R.subseed(R.BASE_SEED, "small2d") if seed is None else seed
    rnd = random.Random(seed)
    h = 2
    size, d_m, d_p = (n, n, 1), (h, h, 0), (h, h, 0)
    shp = _alloc_shape(size, d_m, d_p)
    dats = []
    for k in range(ndats):
        if constant is None:
            a = _zero_halo(R.uniform(R.subseed(seed, "dat", k), shp), size, d_m)
        else:
            a = np.full(shp, float(constant))
        dats.append(DatSpec(f"d{k}", a))
    st = [P0, S5, S9]
    loops = []
    for l in range(nloops):
        nread = rnd.randint(1, 3)
        out = rnd.randrange(ndats)
        reads = rnd.sample([k for k in range(ndats) if k != out], nread)
        args, bb = [], BodyBuilder()
        npts_total = 0
        sts = []
        for r in reads:
            s = rnd.choice([1, 2])
            sts.append(s)
            npts_total += len(st[s])
        if constant is None:
            ws = [rnd.uniform(-1.0, 1.0) for _ in range(npts_total)]
            scale = rnd.uniform(0.6, 1.0) / sum(abs(w) for w in ws)
            ws = [w * scale for w in ws]
        else:
            ws = _dyadic_weights(rnd, npts_total)
        pos = 0
        for ai, (r, s) in enumerate(zip(reads, sts)):
            args.append(Arg(DAT, r, s, READ))
            w = ws[pos:pos + len(st[s])]
            pos += len(st[s])
            if ai == 0:
                bb.wsum(0, ai, w)
            else:
                bb.wacc(0, ai, w)
        args.append(Arg(DAT, out, 0, WRITE))
        bb.st(len(args) - 1, 0)
        code, consts = bb.build()
        loops.append(Loop(f"l{l}", ((0, n), (0, n)), args, code, consts))
    return Chain(f"small2d_{n}", 2, size, d_m, d_p, dats, st, [], loops, steps=reps)


def linear2d(n: int, a0: float, bx: float, by: float) -> Chain:
    """Linear field f = a0 + bx*x + by*y on every point incl. halos, then
    (1) a symmetric 9-point average with weights summing to 1, (2) the
    5-point Laplacian, (3) a one-sided 4-point average (weights 1/8, 1/4,
    3/8, 1/4 at (0,0), (1,0), (0,1), (1,1))."""
    h = 2
    size, d_m, d_p = (n, n, 1), (h, h, 0), (h, h, 0)
    shp = _alloc_shape(size, d_m, d_p)
    y = np.arange(-h, n + h, dtype=np.float64)[:, None]
    x = np.arange(-h, n + h, dtype=np.float64)[None, :]
    f = (a0 + bx * x + by * y)[None, :, :]
    dats = [DatSpec("f", f.copy()), DatSpec("avg9", np.zeros(shp)), DatSpec("lap", np.zeros(shp)),
            DatSpec("avg4", np.zeros(shp))]
    st = [P0, S5, S9, S4P]
    w9 = [1 / 16, 1 / 8, 1 / 16, 1 / 8, 1 / 4, 1 / 8, 1 / 16, 1 / 8, 1 / 16]
    c1, k1 = BodyBuilder().wsum(0, 0, w9).st(1, 0).build()
    c2, k2 = BodyBuilder().wsum(0, 0, [-4.0, 1.0, 1.0, 1.0, 1.0]).st(1, 0).build()
    c3, k3 = BodyBuilder().wsum(0, 0, [1 / 8, 1 / 4, 3 / 8, 1 / 4]).st(1, 0).build()
    rr = ((0, n), (0, n))
    loops = [Loop("avg9", rr, [Arg(DAT, 0, 2, READ), Arg(DAT, 1, 0, WRITE)], c1, k1),
             Loop("lap5", rr, [Arg(DAT, 0, 1, READ), Arg(DAT, 2, 0, WRITE)], c2, k2),
             Loop("avg4", rr, [Arg(DAT, 0, 3, READ), Arg(DAT, 3, 0, WRITE)], c3, k3)]
    return Chain(f"linear2d_{n}", 2, size, d_m, d_p, dats, st, [], loops,
                 meta=dict(a0=a0, bx=bx, by=by))


# --------------------------------------------------------------------------
# Config 2: CloverLeaf-2D-shaped synthetic step
# --------------------------------------------------------------------------
def cloverleaf2d(n: int = 3840, steps: int = 20, seed: int = None, nloops: int = 83,
                 ndats: int = 25, nstatic: int = 4) -> Chain:
    """A CloverLeaf-2D-shaped step: 25 dats U(0.5, 1.5) (halos included),
    83 loops mixing point, 5-point, 9-point and the one-sided 4-point
    stencils {(0,0),(1,0),(0,1),(1,1)} (and its mirror), each loop reading
    2-5 dats and writing 1-2.  Bodies are seeded weighted sums, polynomials,
    min/max and upwind-style selects; most loops cover the cells, some the
    nodes ([0, n+1)^2) and a few are thin halo strips, as in the paper's
    hydro code.  One loop in the middle takes a sum reduction (a field
    summary) and the last one a min reduction whose value, read by the host
    after the step, scales two loops of the next step (the time step).
    """
    seed = R.subseed(R.BASE_SEED, "cloverleaf2d") if seed is None else seed
    return _hydro_chain(2, n, steps, seed, nloops, ndats, nstatic, {3, 45})


S7 = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
S27 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
S8P = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
S8M = [(-x, -y, -z) for x, y, z in S8P]


def cloverleaf3d(n: int = 330, steps: int = 10, seed: int = None, nloops: int = 141,
                 ndats: int = 30, nstatic: int = 5) -> Chain:
    """A CloverLeaf-3D-shaped step (the paper's 3D hydro code has 141
    distinct loops): 30 dats U(0.5, 1.5), 141 loops built like the 2D step
    with the 3D stencils (point, 7-point, 27-point, the one-sided 8-point
    node stencil {0,1}^3 and its mirror), cell, node ([0, n+1)^3) and
    halo-plane ranges, a sum reduction mid-step and a min reduction (the
    time step) at the end."""
    seed = R.subseed(R.BASE_SEED, "cloverleaf3d") if seed is None else seed
    return _hydro_chain(3, n, steps, seed, nloops, ndats, nstatic, {3, 45, 90})


def _hydro_chain(ndim, n, steps, seed, nloops, ndats, nstatic, dt_users) -> Chain:
    rnd = random.Random(seed)
    h = 2
    if ndim == 2:
        size, d_m, d_p = (n, n, 1), (h, h, 0), (h, h, 0)
        st = [P0, S5, S9, S4P, S4M]
        stname = {0: "P", 1: "S5", 2: "S9", 3: "S4P", 4: "S4M"}
        cell = ((0, n), (0, n))
        node = ((0, n + 1), (0, n + 1))
        strips = [((0, n), (-2, 0)), ((0, n), (n, n + 2)), ((-2, 0), (0, n)), ((n, n + 2), (0, n))]
    else:
        size, d_m, d_p = (n, n, n), (h, h, h), (h, h, h)
        st = [P0, S7, S27, S8P, S8M]
        stname = {0: "P", 1: "S7", 2: "S27", 3: "S8P", 4: "S8M"}
        cell = ((0, n), (0, n), (0, n))
        node = ((0, n + 1), (0, n + 1), (0, n + 1))
        strips = []
        for d in range(3):
            for lo, hi in ((-2, 0), (n, n + 2)):
                strips.append(tuple((lo, hi) if e == d else (0, n) for e in range(3)))
    shp = _alloc_shape(size, d_m, d_p)
    dats = [DatSpec(f"d{k:02d}", R.uniform(R.subseed(seed, "dat", k), shp, 0.5, 1.5))
            for k in range(ndats)]
    evolving = list(range(nstatic, ndats))
    recent: List[int] = []
    loops: List[Loop] = []
    sum_at = nloops // 2

    def pick_reads(count, exclude):
        pool = [k for k in range(ndats) if k not in exclude]
        out = []
        fresh = [k for k in recent[-6:] if k not in exclude]
        if fresh:
            out.append(rnd.choice(fresh))
        while len(out) < count:
            k = rnd.choice(pool)
            if k not in out:
                out.append(k)
        return out

    def weights(npts, budget):
        ws = [rnd.uniform(-1.0, 1.0) for _ in range(npts)]
        s = sum(abs(w) for w in ws)
        return [w * budget / s for w in ws]

    for l in range(nloops):
        kind = rnd.choices(["copy", "point", "stencil", "minmax", "select"],
                           weights=[14, 30, 34, 10, 12])[0]
        if l == sum_at or l == nloops - 1:
            kind = "reduce"
        elif l in dt_users:
            kind = "point"
        thin = kind in ("copy", "point") and rnd.random() < 0.12
        rng2 = rnd.choice(strips) if thin else (node if rnd.random() < 0.15 else cell)
        nwrite = 2 if (kind in ("copy", "point", "stencil") and rnd.random() < 0.25) else 1
        writes = [] if kind == "reduce" else rnd.sample(evolving, nwrite)
        nread = rnd.randint(2, 5)
        reads = pick_reads(nread, set(writes))
        # stencils: thin strips and copies use points; one stencil arg elsewhere
        sts = [0] * len(reads)
        if not thin and kind in ("stencil", "minmax", "reduce"):
            sts[0] = rnd.choice([1, 2, 3, 4])
            if kind == "stencil" and len(reads) >= 3 and rnd.random() < 0.4:
                sts[1] = rnd.choice([1, 3, 4])
        if not thin and kind == "select":
            sts[1] = rnd.choice([3, 4])
        args = [Arg(DAT, r, s, READ) for r, s in zip(reads, sts)]
        # a written dat is sometimes updated in place (RW) instead of overwritten
        wargs = []
        for w in writes:
            acc = RW if rnd.random() < 0.2 else WRITE
            wargs.append(len(args))
            args.append(Arg(DAT, w, 0, acc))
        bb = BodyBuilder()
        dt_slot, dt_scale = -1, 0.0
        npts = [len(st[s]) for s in sts]
        if kind == "copy":
            bb.ld(0, 0, 0)
            if len(wargs) > 1:
                bb.ld(1, 1, 0)
            for i, wa in enumerate(wargs):
                bb.st(wa, i if i < 2 else 0)
        elif kind in ("point", "stencil", "reduce"):
            tot = sum(npts)
            has_rw = any(args[wa].access == RW for wa in wargs)
            ws = weights(tot, 0.3 if has_rw else rnd.uniform(0.3, 0.5))
            pos = 0
            for ai in range(len(reads)):
                w = ws[pos:pos + npts[ai]]
                pos += npts[ai]
                (bb.wsum if ai == 0 else bb.wacc)(0, ai, w)
            for wa in wargs:
                if args[wa].access == RW:
                    bb.ld(1, wa, 0)
                    bb.cst(2, 0.5)
                    bb.emit(FMA, 0, 1, 2, 0)   # r0 = old * 0.5 + r0
            if l in dt_users:
                bb.ld(3, len(reads) - 1, 0)
                dt_slot = bb.k(0.0)
                dt_scale = 0.05
                bb.emit(2, 4, dt_slot)           # CST r4 = dt * scale
                bb.emit(FMA, 0, 3, 4, 0)         # r0 = x * (0.05 dt) + r0
            bb.cst(2, 0.5)
            bb.emit(ADD, 0, 0, 2)
            if kind == "reduce":
                rid = 0 if l == sum_at else 1
                args.append(Arg(REDARG, rid, -1, READ))
                bb.red(len(args) - 1, 0)
            else:
                bb.st(wargs[0], 0)
                if len(wargs) > 1:
                    bb.poly(5, 0, [0.3, 0.4, -0.2])
                    bb.st(wargs[1], 5)
        elif kind == "minmax":
            tot0 = npts[0]
            bb.wsum(0, 0, weights(tot0, 0.5))
            rest = sum(npts[1:])
            ws = weights(rest, 0.5)
            pos = 0
            for ai in range(1, len(reads)):
                w = ws[pos:pos + npts[ai]]
                pos += npts[ai]
                (bb.wsum if ai == 1 else bb.wacc)(1, ai, w)
            bb.emit(MIN if rnd.random() < 0.5 else MAX, 0, 0, 1)
            bb.cst(2, 0.6)
            bb.emit(ADD, 0, 0, 2)
            for wa in wargs:
                if args[wa].access == RW:
                    bb.ld(1, wa, 0)
                    bb.emit(MIN, 0, 0, 1)
            bb.st(wargs[0], 0)
        elif kind == "select":
            # upwind: choose between the two neighbours of arg 1 on the sign of (arg0 - 1)
            bb.ld(0, 0, 0)
            bb.cst(1, 1.0)
            bb.ld(2, 1, 0)
            bb.ld(3, 1, 1 if len(st[sts[1]]) > 1 else 0)
            bb.emit(SGT, 4, 0, 1, 2, 3)
            c = rnd.uniform(0.3, 0.6)
            bb.cst(5, c)
            bb.cst(6, 0.5 * (1 - c))
            bb.emit(FMA, 4, 4, 5, 6)
            for ai in range(2, len(reads)):
                bb.wacc(4, ai, weights(npts[ai], 0.2))
            for wa in wargs:
                if args[wa].access == RW:
                    bb.ld(1, wa, 0)
                    bb.emit(MAX, 4, 4, 1)
                    bb.cst(1, 0.5)
                    bb.emit(MUL, 4, 4, 1)
                    bb.cst(1, 0.3)
                    bb.emit(ADD, 4, 4, 1)
            bb.st(wargs[0], 4)
        code, consts = bb.build()
        name = f"{kind}{l}" + ("_strip" if thin else "")
        lp = Loop(name, rng2, args, code, consts, dt_slot, dt_scale)
        lp.stencil_names = [stname.get(a.stencil, "-") for a in args]
        loops.append(lp)
        recent.extend(writes)
    return Chain(f"cloverleaf{ndim}d_{n}", ndim, size, d_m, d_p, dats, st, [RSUM, RMIN], loops,
                 steps=steps, dt_red=1)


# --------------------------------------------------------------------------
# Config 3: OpenSBLI-shaped 3D Runge-Kutta step with radius-2 derivatives
# --------------------------------------------------------------------------
def opensbli3d(n: int = 320, steps: int = 10, seed: int = None) -> Chain:
    """5 conserved variables q0..q4 and 10 work dats on an n^3 grid with halo 2,
    smooth seeded sinusoids (host libm).  Each of 3 Runge-Kutta stages has:
    3 flux loops (a pointwise polynomial of two conserved variables per
    direction, over the range the derivative reads), 3 derivative loops
    (4th-order central first derivative, weights (1, -8, 0, 8, -1)/12 at
    offsets -2..2 along one axis), 1 loop summing the derivatives into a
    residual, and 5 update loops q_k <- a q_k + b q0_k + c R_k (one per
    conserved variable, with its own residual weighting), with a saved copy
    of q at the start of the step: 3 * 13 + 1 = 40 loops per step."""
    seed = R.subseed(R.BASE_SEED, "opensbli3d") if seed is None else seed
    rnd = random.Random(seed)
    h = 2
    size, d_m, d_p = (n, n, n), (h, h, h), (h, h, h)
    shp = _alloc_shape(size, d_m, d_p)
    coords = [np.arange(-h, n + h, dtype=np.float64) * (2 * math.pi / n) for _ in range(3)]
    dats = []
    for k in range(5):
        ph = [rnd.uniform(0, 2 * math.pi) for _ in range(3)]
        amp = rnd.uniform(0.05, 0.2)
        fx = np.array([math.sin(v + ph[0]) for v in coords[0]])
        fy = np.array([math.cos(v + ph[1]) for v in coords[1]])
        fz = np.array([math.sin(v + ph[2]) for v in coords[2]])
        f = 1.0 + amp * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        dats.append(DatSpec(f"q{k}", f))
    names = ["q0s", "q1s", "q2s", "q3s", "q4s", "F", "Dx", "Dy", "Dz", "Res"]
    for nm in names:
        dats.append(DatSpec(nm, np.zeros(shp)))
    Q = list(range(5))
    QS = list(range(5, 10))
    F, DX, DY, DZ, RES = 10, 11, 12, 13, 14
    st = [P0,
          [(o, 0, 0) for o in (-2, -1, 0, 1, 2)],
          [(0, o, 0) for o in (-2, -1, 0, 1, 2)],
          [(0, 0, o) for o in (-2, -1, 0, 1, 2)]]
    inv12 = 1.0 / 12.0
    dw = [inv12, -8 * inv12, 0.0, 8 * inv12, -inv12]
    cells = ((0, n), (0, n), (0, n))
    loops: List[Loop] = []
    # save q at step start
    for k in range(5):
        c, kk = BodyBuilder().ld(0, 0, 0).st(1, 0).build()
        loops.append(Loop(f"save{k}", cells, [Arg(DAT, Q[k], 0, READ), Arg(DAT, QS[k], 0, WRITE)], c, kk))
    rk = [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1 / 3, 2 / 3, 2 / 3)]
    for s, (a_old, a_cur, c_res) in enumerate(rk):
        for d, DD in enumerate((DX, DY, DZ)):
            # flux over the cells widened by 2 along the derivative axis
            rr = [list(x) for x in cells]
            rr[d] = [-2, n + 2]
            rr = tuple(tuple(x) for x in rr)
            qa, qb = rnd.sample(Q, 2)
            bb = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0)
            bb.emit(MUL, 2, 0, 1)                   # qa*qb
            bb.poly(3, 0, [0.1, rnd.uniform(0.2, 0.4), rnd.uniform(-0.1, 0.1)])
            bb.emit(ADD, 2, 2, 3).st(2, 2)
            c, kk = bb.build()
            loops.append(Loop(f"flux{s}{'xyz'[d]}", rr, [Arg(DAT, qa, 0, READ), Arg(DAT, qb, 0, READ),
                                                        Arg(DAT, F, 0, WRITE)], c, kk))
            c, kk = BodyBuilder().wsum(0, 0, dw).st(1, 0).build()
            loops.append(Loop(f"deriv{s}{'xyz'[d]}", cells, [Arg(DAT, F, 1 + d, READ), Arg(DAT, DD, 0, WRITE)],
                              c, kk))
        c, kk = (BodyBuilder().wsum(0, 0, [-1.0]).wacc(0, 1, [-1.0]).wacc(0, 2, [-1.0]).st(3, 0).build())
        loops.append(Loop(f"resid{s}", cells, [Arg(DAT, DX, 0, READ), Arg(DAT, DY, 0, READ),
                                               Arg(DAT, DZ, 0, READ), Arg(DAT, RES, 0, WRITE)], c, kk))
        for k in range(5):
            dtk = 0.02 * rnd.uniform(0.5, 1.0)
            bb = BodyBuilder()
            bb.wsum(0, 0, [a_cur]).wacc(0, 1, [a_old]).wacc(0, 2, [c_res * dtk]).st(0, 0)
            c, kk = bb.build()
            loops.append(Loop(f"rk{s}q{k}", cells, [Arg(DAT, Q[k], 0, RW), Arg(DAT, QS[k], 0, READ),
                                                    Arg(DAT, RES, 0, READ)], c, kk))
    return Chain(f"opensbli3d_{n}", 3, size, d_m, d_p, dats, st, [], loops, steps=steps)


# --------------------------------------------------------------------------
# TeaLeaf-PPCG-shaped chain: the polynomial preconditioner's inner loops
# --------------------------------------------------------------------------
def ppcg2d(n: int = 4000, inner: int = 10, steps: int = 1, seed: int = None, kappa_const: float = None,
           r_mode: Tuple[int, int] = None) -> Chain:
    """A TeaLeaf-PPCG-shaped chain (Sec. 6.D): one application of a Chebyshev
    polynomial preconditioner to a residual r on the 5-point heat operator.
    Setup loops build the negated face coefficients and the diagonal from a
    conductivity log-uniform in [0.1, 10] (harmonic means inside, the cell's
    own at the boundary; d = 1 + sum of the faces); then sd = r / theta,
    rt = r, z = sd, and `inner` iterations of
        w = A sd;   rt = rt - w;   sd = alpha_k sd + beta_k rt, z = z + sd
    with the Chebyshev coefficients for the spectrum bound [1, 81]; a last
    loop reduces z.r for the outer CG.  No loop before it reduces, so the
    whole application is one segment.  kappa_const and r_mode = (p, q) (the
    Dirichlet eigenmode sin(pi p (i+1)/(n+1)) sin(pi q (j+1)/(n+1))) give a
    case with a closed form."""
    seed = R.subseed(R.BASE_SEED, "ppcg2d", n) if seed is None else seed
    h = 1
    size, d_m, d_p = (n, n, 1), (h, h, 0), (h, h, 0)
    shp = _alloc_shape(size, d_m, d_p)
    if kappa_const is None:
        u = R.uniform(R.subseed(seed, "kappa"), shp, 0.0, 1.0)
        kappa = _zero_halo(np.exp(np.log(0.1) + (np.log(10.0) - np.log(0.1)) * u), size, d_m)
    else:
        kappa = _zero_halo(np.full(shp, float(kappa_const)), size, d_m)
    if r_mode is None:
        r = _zero_halo(R.uniform(R.subseed(seed, "r"), shp, 0.0, 1.0), size, d_m)
    else:
        p, q = r_mode
        i = np.arange(n)
        sx = np.array([math.sin(math.pi * p * (k + 1) / (n + 1)) for k in i])
        sy = np.array([math.sin(math.pi * q * (k + 1) / (n + 1)) for k in i])
        r = np.zeros(shp)
        r[0, h:n + h, h:n + h] = np.outer(sy, sx)
    names = ["kappa", "r", "rt", "sd", "w", "z", "nkx", "nky", "dg"]
    init = {"kappa": kappa, "r": r}
    dats = [DatSpec(nm, init.get(nm, np.zeros(shp))) for nm in names]
    K, Rr, RT, SD, Wd, Z, NKX, NKY, DG = range(len(names))
    st = [P0, S5, [(0, 0, 0), (1, 0, 0)], [(0, 0, 0), (0, 1, 0)], [(0, 0, 0), (-1, 0, 0)], [(0, 0, 0), (0, -1, 0)]]
    SP, SS5, SEX, SEY, SWX, SSY = range(len(st))
    cells = ((0, n), (0, n))
    loops: List[Loop] = []

    def face_loops(dat, sten, interior, west, east):
        bb = BodyBuilder().ld(0, 0, 1).ld(1, 0, 0).cst(2, 2.0).emit(MUL, 3, 2, 0).emit(MUL, 3, 3, 1)
        bb.emit(ADD, 4, 0, 1).emit(7, 5, 3, 4).cst(6, 0.0).emit(SUB, 7, 6, 5).st(1, 7)
        c, k = bb.build()
        args = [Arg(DAT, K, sten, READ), Arg(DAT, dat, SP, WRITE)]
        loops.append(Loop(f"face_in{dat}", interior, args, c, k))
        c, k = BodyBuilder().ld(0, 0, 0).cst(6, 0.0).emit(SUB, 7, 6, 0).st(1, 7).build()
        loops.append(Loop(f"face_lo{dat}", west, args, c, k))
        c, k = BodyBuilder().ld(0, 0, 1).cst(6, 0.0).emit(SUB, 7, 6, 0).st(1, 7).build()
        loops.append(Loop(f"face_hi{dat}", east, args, c, k))

    face_loops(NKX, SWX, ((1, n), (0, n)), ((0, 1), (0, n)), ((n, n + 1), (0, n)))
    face_loops(NKY, SSY, ((0, n), (1, n)), ((0, n), (0, 1)), ((0, n), (n, n + 1)))
    bb = BodyBuilder().cst(0, 1.0)
    for a, pt in ((0, 0), (0, 1), (1, 0), (1, 1)):
        bb.ld(1, a, pt).emit(SUB, 0, 0, 1)
    c, k = bb.st(2, 0).build()
    loops.append(Loop("diag", cells, [Arg(DAT, NKX, SEX, READ), Arg(DAT, NKY, SEY, READ), Arg(DAT, DG, SP, WRITE)],
                      c, k))
    lmin, lmax = 1.0, 81.0
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    c, k = BodyBuilder().ld(0, 0, 0).cst(1, 1.0 / theta).emit(MUL, 2, 0, 1).st(1, 2).st(2, 0).st(3, 2).build()
    loops.append(Loop("init", cells, [Arg(DAT, Rr, SP, READ), Arg(DAT, SD, SP, WRITE), Arg(DAT, RT, SP, WRITE),
                                      Arg(DAT, Z, SP, WRITE)], c, k))
    sigma = theta / delta
    rho_old = 1.0 / sigma
    for it in range(inner):
        # w = A sd, the engine's term order
        bb = BodyBuilder().ld(0, 1, 0).ld(1, 0, 0).emit(MUL, 2, 0, 1)
        for a, pa, pp in ((2, 0, 1), (2, 1, 2), (3, 0, 3), (3, 1, 4)):
            bb.ld(0, a, pa).ld(1, 0, pp).emit(FMA, 2, 0, 1, 2)
        c, k = bb.st(4, 2).build()
        loops.append(Loop(f"matvec{it}", cells, [Arg(DAT, SD, SS5, READ), Arg(DAT, DG, SP, READ),
                                                   Arg(DAT, NKX, SEX, READ), Arg(DAT, NKY, SEY, READ),
                                                   Arg(DAT, Wd, SP, WRITE)], c, k))
        c, k = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).emit(SUB, 2, 0, 1).st(0, 2).build()
        loops.append(Loop(f"resid{it}", cells, [Arg(DAT, RT, SP, RW), Arg(DAT, Wd, SP, READ)], c, k))
        rho = 1.0 / (2.0 * sigma - rho_old)
        alpha, beta = rho * rho_old, 2.0 * rho / delta
        rho_old = rho
        bb = BodyBuilder().cst(0, alpha).ld(1, 0, 0).emit(MUL, 2, 0, 1).cst(3, beta).ld(4, 1, 0)
        bb.emit(FMA, 2, 3, 4, 2).st(0, 2).ld(5, 2, 0).emit(ADD, 5, 5, 2).st(2, 5)
        c, k = bb.build()
        loops.append(Loop(f"cheby{it}", cells, [Arg(DAT, SD, SP, RW), Arg(DAT, RT, SP, READ), Arg(DAT, Z, SP, RW)],
                          c, k))
    c, k = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).emit(MUL, 2, 0, 1).red(2, 2).build()
    loops.append(Loop("zr", cells, [Arg(DAT, Z, SP, READ), Arg(DAT, Rr, SP, READ), Arg(REDARG, 0, -1, READ)], c, k))
    return Chain(f"ppcg2d_{n}", 2, size, d_m, d_p, dats, st, [RSUM], loops, steps=steps,
                 meta=dict(inner=inner, theta=theta, delta=delta))


# --------------------------------------------------------------------------
# Configs 4 and 5: heat-conduction CG problems
# --------------------------------------------------------------------------
def cg_problem(n: int, klo: float, khi: float, seed: int = None):
    """Cell conductivity log-uniform in [klo, khi] and a U(0,1) right-hand side
    on an n x n grid (row-major, x fastest)."""
    seed = R.subseed(R.BASE_SEED, "cg", n) if seed is None else seed
    # numpy's PCG64 (same stream on every platform) is used here for speed:
    # the serving workload draws hundreds of grids of up to 2048^2 cells
    g = np.random.Generator(np.random.PCG64(seed & ((1 << 63) - 1)))
    u = g.random((n, n))
    kappa = np.exp(np.log(klo) + (np.log(khi) - np.log(klo)) * u)
    rhs = g.random((n, n))
    return kappa, rhs


def serving_stream(nreq: int = 512, seed: int = None, sizes: Sequence[int] = None,
                   rate: float = 1.0):
    """Requests (arrival time, n, request seed) with Poisson arrivals at `rate`
    per second and n uniform over `sizes` (default: multiples of 64 in
    [64, 2048])."""
    seed = R.subseed(R.BASE_SEED, "serve") if seed is None else seed
    sizes = list(range(64, 2049, 64)) if sizes is None else list(sizes)
    gaps = R.exponential(R.subseed(seed, "gaps"), nreq, rate)
    t = np.cumsum(gaps) - gaps[0]
    pick = R.splitmix64(R.subseed(seed, "size"), np.arange(nreq)) % np.uint64(len(sizes))
    return [(float(t[i]), int(sizes[int(pick[i])]), R.subseed(seed, "req", i)) for i in range(nreq)]


def instances(chain: Chain, count: int, seed: int = None) -> List[Chain]:
    """count copies of chain with the same loops, stencils and reductions and
    fresh field values (the grids of a batch): each dat is drawn U(lo, hi)
    over the range of the original's non-zero values, keeping the original's
    zeros (the halos some workloads zero) and keeping a dat that is constant.
    Instance 0 is chain itself."""
    import copy
    seed = R.subseed(R.BASE_SEED, "instances", chain.name) if seed is None else seed
    out = [chain]
    for k in range(1, count):
        c = copy.copy(chain)
        dats = []
        for j, d in enumerate(chain.dats):
            a = d.init
            nz = a != 0.0
            if not nz.any() or a[nz].min() == a[nz].max():
                dats.append(DatSpec(d.name, a.copy()))
                continue
            lo, hi = float(a[nz].min()), float(a[nz].max())
            u = R.uniform(R.subseed(seed, "inst", k, j), a.shape)
            dats.append(DatSpec(d.name, np.where(nz, lo + (hi - lo) * u, 0.0)))
        c.dats = dats
        c.meta = dict(chain.meta, instance=k)
        out.append(c)
    return out
