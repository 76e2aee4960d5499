"""Brute-force dependence checks for tiling plans on tiny grids.

The reference semantics is the untiled program order (Sec. 3: a parallel
loop must not depend on the order of its points).  Instead of values we
track *versions*: every dat cell remembers which loop wrote it last (-1 for
the initial value).  A tiled schedule is valid iff every read of every
(loop, point) sees the same version as in program order and every cell ends
with the same version.  This catches any violated RAW, WAR or WAW ordering
without trusting the planner's own reasoning.
"""
from __future__ import annotations

import itertools
import random
from typing import Dict, List, Sequence, Tuple

from synth.program import DAT, READ, WRITE, RW, INC, Arg, Loop

import numpy as np


def _points(box):
    return itertools.product(*[range(lo, hi) for lo, hi in reversed(box)])


def _pt(rev):
    return tuple(reversed(rev))


def _reads(a):
    return a.kind == DAT and a.access in (READ, RW, INC)


def _writes(a):
    return a.kind == DAT and a.access in (WRITE, RW, INC)


def _shift(P, off, ndim):
    return tuple(P[d] + off[d] for d in range(ndim))


def run_point(lp, l, P, stencils, ndim, ver, seen):
    for ai, a in enumerate(lp.args):
        if _reads(a):
            for pi, off in enumerate(stencils[a.stencil]):
                X = _shift(P, off, ndim)
                seen[(l, P, ai, pi)] = ver.get((a.handle, X), -1)
    for a in lp.args:
        if _writes(a):
            ver[(a.handle, P)] = l


def untiled(loops, stencils, ndim):
    ver, seen = {}, {}
    for l, lp in enumerate(loops):
        box = lp.rng[:ndim]
        for rev in _points(box):
            run_point(lp, l, _pt(rev), stencils, ndim, ver, seen)
    return ver, seen


def check_skewed(loops, stencils, ndim, ntiles, ranges):
    """ranges[d][t][l] = (start, end).  Tiles run lexicographically, x fastest."""
    ref_ver, ref_seen = untiled(loops, stencils, ndim)
    ver, seen = {}, {}
    done = set()
    order = itertools.product(*[range(ntiles[d]) for d in reversed(range(ndim))])
    for rev_t in order:
        t = tuple(reversed(rev_t))
        for l, lp in enumerate(loops):
            box = tuple(ranges[d][t[d]][l] for d in range(ndim))
            for rev in _points(box):
                P = _pt(rev)
                assert (l, P) not in done, f"loop {l} point {P} executed twice"
                done.add((l, P))
                run_point(lp, l, P, stencils, ndim, ver, seen)
    for l, lp in enumerate(loops):
        for rev in _points(lp.rng[:ndim]):
            assert (l, _pt(rev)) in done, f"loop {l} point {_pt(rev)} never executed"
    for k, v in ref_seen.items():
        assert seen[k] == v, f"read {k}: tiled sees version {seen[k]}, program order {v}"
    assert ver == ref_ver, "final versions differ"


def check_phase_order(loops, stencils, ndim, phases, order):
    """phases: [(loop, box)]; order: the sequence of phase indices actually
    executed.  Every (loop, point) of every loop's range must run exactly
    once, every read must see its program-order version and every cell must
    end with its program-order version."""
    ref_ver, ref_seen = untiled(loops, stencils, ndim)
    ver, seen = {}, {}
    done = set()
    for q in order:
        l, box = phases[q]
        for rev in _points(box):
            P = _pt(rev)
            assert (l, P) not in done, f"loop {l} point {P} executed twice"
            done.add((l, P))
            run_point(loops[l], l, P, stencils, ndim, ver, seen)
    for l, lp in enumerate(loops):
        for rev in _points(lp.rng[:ndim]):
            assert (l, _pt(rev)) in done, f"loop {l} point {_pt(rev)} never executed"
    for k, v in ref_seen.items():
        assert seen[k] == v, f"read {k}: sees version {seen[k]}, program order {v}"
    assert ver == ref_ver, "final versions differ"


def random_topological(deps, rnd: random.Random):
    """A random order of range(len(deps)) that puts every p in deps[q] before q."""
    waiting = [len(d) for d in deps]
    users = [[] for _ in deps]
    for q, d in enumerate(deps):
        for p in d:
            users[p].append(q)
    ready = [q for q in range(len(deps)) if waiting[q] == 0]
    order = []
    while ready:
        q = ready.pop(rnd.randrange(len(ready)))
        order.append(q)
        for u in users[q]:
            waiting[u] -= 1
            if waiting[u] == 0:
                ready.append(u)
    assert len(order) == len(deps), "dependency cycle"
    return order


def check_overlapped(loops, stencils, ndim, tiles: Sequence, plan_fn):
    """Every tile runs on a private copy of the pre-segment state; every point
    it computes must see program-order inputs, every live-in read must lie in
    the tile's footprint, and the owned cells of written dats must end with
    the program-order version."""
    ref_ver, ref_seen = untiled(loops, stencils, ndim)
    for owned in tiles:
        boxes, foot = plan_fn(loops, stencils, ndim, owned)
        ver, seen = {}, {}
        for l, lp in enumerate(loops):
            box = boxes[l]
            own = tuple((max(lp.rng[d][0], owned[d][0]), min(lp.rng[d][1], owned[d][1])) for d in range(ndim))
            if all(lo < hi for lo, hi in own):
                for d in range(ndim):
                    assert box[d][0] <= own[d][0] and own[d][1] <= box[d][1], \
                        f"loop {l}: tile box {box} misses owned part {own}"
            for rev in _points(box):
                P = _pt(rev)
                assert all(lp.rng[d][0] <= P[d] < lp.rng[d][1] for d in range(ndim)), \
                    f"loop {l} computes {P} outside its range"
                run_point(lp, l, P, stencils, ndim, ver, seen)
                for ai, a in enumerate(lp.args):
                    if _reads(a):
                        for pi, off in enumerate(stencils[a.stencil]):
                            k = (l, P, ai, pi)
                            assert seen[k] == ref_seen[k], \
                                f"tile {owned}: read {k} sees {seen[k]}, program order {ref_seen[k]}"
                            if seen[k] == -1:
                                X = _shift(P, off, ndim)
                                fb = foot[a.handle]
                                assert all(fb[d][0] <= X[d] < fb[d][1] for d in range(ndim)), \
                                    f"live-in {a.handle}@{X} outside footprint {fb}"
        for (dat, X), v in ref_ver.items():
            if all(owned[d][0] <= X[d] < owned[d][1] for d in range(ndim)):
                assert ver.get((dat, X), -1) == v, f"tile {owned}: dat {dat} cell {X} ends at {ver.get((dat, X), -1)}, want {v}"


# ---------------------------------------------------------------------------
# random tiny chains
# ---------------------------------------------------------------------------
def random_chain(rnd: random.Random, ndim: int, n: Sequence[int], ndats: int, nloops: int,
                 halo: int = 2, maxr: int = 2):
    """Loops with random sub-ranges of [-1, n+1), random stencils with
    offsets in [-maxr, maxr] kept inside the halo, 1-3 read and 1-2 written
    dats (each dat at most once per loop, written args on point stencils)."""
    stencils = [[(0, 0, 0)]]
    loops = []
    for l in range(nloops):
        rng = []
        for d in range(3):
            if d < ndim:
                lo = rnd.randint(-1, max(-1, n[d] // 3))
                hi = rnd.randint(min(n[d] + 1, lo + 1), n[d] + 1)
                rng.append((lo, hi))
            else:
                rng.append((0, 1))
        dats = rnd.sample(range(ndats), min(ndats, rnd.randint(2, 4)))
        nw = rnd.randint(1, min(2, len(dats) - 1))
        writes, reads = dats[:nw], dats[nw:]
        args = []
        for r in reads:
            npts = rnd.randint(1, 4)
            pts = set()
            for _ in range(npts):
                off = [0, 0, 0]
                for d in range(ndim):
                    lo = max(-maxr, -halo - rng[d][0])
                    hi = min(maxr, n[d] + halo - rng[d][1])
                    off[d] = rnd.randint(lo, hi)
                pts.add(tuple(off))
            stencils.append(sorted(pts))
            args.append(Arg(DAT, r, len(stencils) - 1, READ))
        for w in writes:
            acc = rnd.choice([WRITE, WRITE, RW, INC])
            args.append(Arg(DAT, w, 0, acc))
        lp = Loop(f"l{l}", tuple(rng), args, np.zeros((0, 6), np.int32), np.zeros(1))
        loops.append(lp)
    return loops, stencils
