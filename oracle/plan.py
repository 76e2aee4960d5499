"""Tiling plans restated from the paper, for checking the library's planner.

TEST INFRASTRUCTURE ONLY (see the package docstring).

`skewed_plan` is Algorithm 1 (Sec. 4.B): the union of the loops' iteration
ranges is cut into tiles of a given size per dimension; walking the loops
backwards, every tile of every loop gets its own range so that executing all
loops of tile 0, then all loops of tile 1, ... (Algorithm 2) respects every
read-after-write, write-after-read and write-after-write dependency.  The
readings taken where the printed algorithm is ambiguous:

  * ranges are half-open [start, end);
  * a tile starts where the same loop's previous tile ends (the prose of
    Sec. 4.B step 3), so per (loop, dimension) the tiles are computed in
    increasing order, each one completely (start, RAW end, WAR/WAW end,
    default end) before the next;
  * the default end of 0-based tile t is min(loop end, start_d + (t+1) * tilesize);
  * every end is clamped to at least the tile's start, and the last tile
    takes the loop's end, so a loop's tiles partition its range (later tiles
    may be empty);
  * "largest negative stencil point" m is min(0, most negative offset),
    "largest positive" p is max(0, most positive offset);
  * WAR/WAW looks at all arguments of the loop (read and written); a written
    argument has a point stencil, so m = 0 gives the WAW case;
  * empty ranges leave the dependency records unchanged; read records are
    never reset when a later loop overwrites a dat (conservative);
  * write_dep_a.tile_l in the printed update is tile t;
  * dimensions are tiled separably and tiles run in lexicographic order,
    x fastest.

`overlapped_plan` is the overlapped tiling of Sec. 4.D used per tile instead
of per MPI rank: each tile owns a box, and walking the loops backwards with
read dependencies only, each loop's range inside the tile is grown to cover
what later loops of the same tile read; tiles are then independent.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

NEG = -(1 << 40)
POS = 1 << 40

DAT, READ, WRITE, RW, INC = 0, 0, 1, 2, 3


def _reads(arg) -> bool:
    return arg.kind == DAT and arg.access in (READ, RW, INC)


def _writes(arg) -> bool:
    return arg.kind == DAT and arg.access in (WRITE, RW, INC)


def _ext(stencil, d) -> Tuple[int, int]:
    lo = min(0, min(p[d] for p in stencil))
    hi = max(0, max(p[d] for p in stencil))
    return lo, hi


def skewed_plan(loops: Sequence, stencils: Sequence, ndim: int, tilesize: Sequence[int]):
    """Algorithm 1.  Returns (ntiles, ranges, union) where ntiles[d] is the
    tile count in dimension d and ranges[d][t][l] = (start, end) of loop l in
    tile index t along dimension d."""
    L = len(loops)
    union = []
    ntiles = []
    for d in range(ndim):
        s = min(lp.rng[d][0] for lp in loops)
        e = max(lp.rng[d][1] for lp in loops)
        union.append((s, e))
        ntiles.append((e - s - 1) // tilesize[d] + 1 if e > s else 1)
    ranges = [[[None] * L for _ in range(ntiles[d])] for d in range(ndim)]
    # dependency records per dimension, per tile, per dat: [start, end)
    read_dep: List[List[Dict[int, List[int]]]] = [[{} for _ in range(ntiles[d])] for d in range(ndim)]
    write_dep: List[List[Dict[int, List[int]]]] = [[{} for _ in range(ntiles[d])] for d in range(ndim)]

    for l in range(L - 1, -1, -1):
        lp = loops[l]
        for d in range(ndim):
            ls, le = lp.rng[d]
            T = ntiles[d]
            for t in range(T):
                start = ls if t == 0 else ranges[d][t - 1][l][1]
                end = NEG
                if t == T - 1:
                    end = le
                else:
                    # read-after-write: cover what later loops of this tile read
                    for a in lp.args:
                        if _writes(a):
                            rd = read_dep[d][t].get(a.handle)
                            if rd is not None:
                                end = min(le, max(end, rd[1]))
                    # write-after-read / write-after-write against later writers
                    for a in lp.args:
                        if a.kind != DAT:
                            continue
                        wd = write_dep[d][t].get(a.handle)
                        if wd is not None:
                            m = _ext(stencils[a.stencil], d)[0]
                            end = min(le, max(end, wd[1] - m))
                if end == NEG:
                    end = min(le, union[d][0] + (t + 1) * tilesize[d])
                end = max(end, start)
                ranges[d][t][l] = (start, end)
                if end <= start:
                    continue
                for a in lp.args:
                    if _reads(a):
                        m, p = _ext(stencils[a.stencil], d)
                        rd = read_dep[d][t].setdefault(a.handle, [POS, NEG])
                        rd[1] = max(rd[1], end + p)
                        rd[0] = min(rd[0], start + m)
                for a in lp.args:
                    if _writes(a):
                        wd = write_dep[d][t].setdefault(a.handle, [POS, NEG])
                        wd[1] = max(wd[1], end)
                        wd[0] = min(wd[0], start)
    return ntiles, ranges, union


def tile_boxes(ntiles, ranges, ndim: int, l: int):
    """Yield (tile multi-index, box) for loop l in execution order (x fastest)."""
    import itertools
    order = list(itertools.product(*[range(ntiles[d]) for d in reversed(range(ndim))]))
    for rev in order:
        t = tuple(reversed(rev))
        box = tuple(ranges[d][t[d]][l] for d in range(ndim))
        yield t, box


def overlapped_plan(loops: Sequence, stencils: Sequence, ndim: int, owned: Sequence[Tuple[int, int]]):
    """Per-tile ranges for overlapped tiling.  `owned` is the tile's box.

    Returns (boxes, footprint): boxes[l] = per-dimension (lo, hi) of loop l
    inside this tile (empty where lo >= hi), footprint[dat] = the box of dat
    values the tile reads that it did not compute itself."""
    L = len(loops)
    boxes = [None] * L
    readbox: Dict[int, List[List[int]]] = {}

    def hull(a, b):
        return [min(a[0], b[0]), max(a[1], b[1])]

    for l in range(L - 1, -1, -1):
        lp = loops[l]
        box = []
        for d in range(ndim):
            ls, le = lp.rng[d]
            lo, hi = max(ls, owned[d][0]), min(le, owned[d][1])
            if hi <= lo:
                lo, hi = POS, NEG
            for a in lp.args:
                if _writes(a) and a.handle in readbox:
                    rb = readbox[a.handle][d]
                    lo, hi = min(lo, max(ls, rb[0])), max(hi, min(le, rb[1]))
            box.append((lo, hi))
        if any(hi <= lo for lo, hi in box):
            box = [(0, 0)] * ndim
            boxes[l] = tuple(box)
            continue
        boxes[l] = tuple(box)
        for a in lp.args:
            if _reads(a):
                rb = readbox.setdefault(a.handle, [[POS, NEG] for _ in range(ndim)])
                for d in range(ndim):
                    m, p = _ext(stencils[a.stencil], d)
                    rb[d] = hull(rb[d], [box[d][0] + m, box[d][1] + p])
    # live-in footprint: values read before being produced inside the tile
    footprint: Dict[int, Tuple[Tuple[int, int], ...]] = {}
    for dat, rb in readbox.items():
        footprint[dat] = tuple((rb[d][0], rb[d][1]) for d in range(ndim))
    return boxes, footprint


def phases_in_order(loops: Sequence, ntiles, ranges, ndim: int):
    """Algorithm 2's execution order of a skewed plan: tiles in lexicographic
    order (x fastest), the loops in program order inside a tile; phases with
    an empty box are dropped.  Returns [(loop index, box)], box a tuple of
    per-dimension (lo, hi)."""
    import itertools
    out = []
    for rev in itertools.product(*[range(ntiles[d]) for d in reversed(range(ndim))]):
        t = tuple(reversed(rev))
        for l in range(len(loops)):
            box = tuple(ranges[d][t[d]][l] for d in range(ndim))
            if all(hi > lo for lo, hi in box):
                out.append((l, box))
    return out


def phase_conflicts(loops: Sequence, stencils: Sequence, ndim: int, phases):
    """For every phase q (in the given order) the sorted list of earlier
    phases p that must stay before it: p and q touch a common point of some
    dat and at least one of them writes that point.  A phase reads, for each
    reading argument, the points of its box shifted by each point of the
    argument's stencil, and writes the points of its box for each writing
    argument (the exact point sets, not bounding boxes).  Any execution that
    keeps every such pair in order computes what the given order computes
    (program order, for the phases of a skewed plan).  Brute force over
    boolean masks: small problems only."""
    import numpy as np
    n = len(phases)
    lo, hi = [0] * ndim, [1] * ndim
    for l, box in phases:
        for a in loops[l].args:
            if a.kind != DAT:
                continue
            for d in range(ndim):
                m, p = _ext(stencils[a.stencil], d)
                lo[d] = min(lo[d], box[d][0] + m)
                hi[d] = max(hi[d], box[d][1] + p)
    shape = tuple(hi[d] - lo[d] for d in reversed(range(ndim)))  # z, y, x
    dats = sorted({a.handle for lp in loops for a in lp.args if a.kind == DAT})
    conf = np.zeros((n, n), dtype=bool)
    for k in dats:
        idx = [i for i, (l, _) in enumerate(phases) if any(a.kind == DAT and a.handle == k for a in loops[l].args)]
        R = np.zeros((len(idx), int(np.prod(shape))), dtype=np.float32)
        Wm = np.zeros_like(R)
        for j, i in enumerate(idx):
            l, box = phases[i]
            for a in loops[l].args:
                if a.kind != DAT or a.handle != k:
                    continue
                pts = stencils[a.stencil] if _reads(a) else []
                for p in pts:
                    m = np.zeros(shape, dtype=bool)
                    sl = tuple(slice(box[d][0] + p[d] - lo[d], box[d][1] + p[d] - lo[d]) for d in reversed(range(ndim)))
                    m[sl] = True
                    R[j] = np.maximum(R[j], m.reshape(-1))
                if _writes(a):
                    m = np.zeros(shape, dtype=bool)
                    sl = tuple(slice(box[d][0] - lo[d], box[d][1] - lo[d]) for d in reversed(range(ndim)))
                    m[sl] = True
                    Wm[j] = np.maximum(Wm[j], m.reshape(-1))
        T = np.maximum(R, Wm)
        c = (Wm @ T.T > 0) | (T @ Wm.T > 0)
        ix = np.array(idx, dtype=np.int64)
        conf[np.ix_(ix, ix)] |= c
    return [sorted(int(p) for p in np.nonzero(conf[q, :q])[0]) for q in range(n)]
