"""Host checks of the tile-wavefront plan (OPS_MODE_TILEWAVE): no GPU.

The library's plan says, per tile class, predecessor direction and loop,
how many loops of the predecessor tile must be complete before the tile
runs that loop.  These tests hold it against the oracle's restatement of
Algorithm 1 and its exact phase-conflict relation, and against brute force:
random interleavings of the tiles that obey the plan must give every read
and every cell its program-order version.
"""
import itertools
import json
import os
import random

import numpy as np
import pytest

import paper_1704_00693_gb300 as ops
from paper_1704_00693_gb300 import _build
from oracle import plan as oplan
from synth import workloads as W
from synth.program import DAT, READ, BodyBuilder

from bruteforce import check_phase_order, random_chain

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ops.load()


def _plan(loops, stencils, ndim, tile):
    """The library's tile-wavefront plan of `loops` through the ABI (host-only
    context), or None when it reports the tiles too small."""
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    ctx = ops.ops_init(cfg)
    try:
        b = ops.ops_decl_block(ctx, ndim)
        ndats = 1 + max(a.handle for lp in loops for a in lp.args if a.kind == DAT)
        size = [1, 1, 1]
        for d in range(ndim):
            size[d] = max(lp.rng[d][1] for lp in loops) + 2
        dats = [ops.ops_decl_dat(ctx, b, size, [4 if d < ndim else 0 for d in range(3)],
                                 [4 if d < ndim else 0 for d in range(3)]) for _ in range(ndats)]
        st = [ops.ops_decl_stencil(ctx, ndim, s) for s in stencils]
        nreds = 1 + max([a.handle for lp in loops for a in lp.args if a.kind != DAT] + [-1])
        reds = [ops.ops_decl_reduction(ctx, ops.OPS_RED_SUM) for _ in range(nreds)]
        for lp in loops:
            args = [(a.kind, dats[a.handle], st[a.stencil], a.access) if a.kind == DAT else
                    (a.kind, reds[a.handle], -1, a.access) for a in lp.args]
            bb = BodyBuilder()
            for i, a in enumerate(lp.args):
                if a.kind == DAT and a.access != READ:
                    bb.st(i, 0)
            code, K = bb.build()
            ops.ops_par_loop(ctx, b, ndim, lp.rng[:ndim], args, code, K, lp.name)
        try:
            return ops.ops_plan_tilewave(ctx, list(tile))
        except ops.OpsError as e:
            assert e.code == ops.OPS_ERR_INVALID_ARG and "tiles" in str(e), str(e)
            return None
        finally:
            ops.ops_queue_clear(ctx)
    finally:
        ops.ops_finalize(ctx)


def _tile_phases(loops, ndim, nt, rg):
    """Non-empty (tile, loop, box) in Algorithm 2 order, tile as a tuple."""
    out = []
    for rev in itertools.product(*[range(nt[d]) for d in reversed(range(ndim))]):
        t = tuple(reversed(rev))
        for l in range(len(loops)):
            box = tuple(rg[d][t[d]][l] for d in range(ndim))
            if all(hi > lo for lo, hi in box):
                out.append((t, l, box))
    return out


def _lin(t, nt):
    k = 0
    for d in reversed(range(len(t))):
        k = k * nt[d] + t[d]
    return k


def _dir_index(delta):
    """Direction k steps back in dimension d when bit d of k + 1 is set."""
    m = sum(1 << d for d, v in enumerate(delta) if v)
    return m - 1


def _check(loops, st, ndim, tile, rnd, schedules=3):
    got = _plan(loops, st, ndim, tile)
    if got is None:
        return False
    need, cls, order, steps = got
    nt, rg, _ = oplan.skewed_plan(loops, st, ndim, tile)
    ntiles = int(np.prod(nt))
    assert len(cls) == ntiles and sorted(order.tolist()) == list(range(ntiles))
    assert need.shape[1] == (1 << ndim) - 1 and need.shape[2] == len(loops)
    tiles = list(itertools.product(*[range(nt[d]) for d in range(ndim)]))
    ticket = {int(order[k]): k for k in range(ntiles)}
    # every predecessor one step back has a smaller ticket
    for t in tiles:
        for m in range(1, 1 << ndim):
            p = tuple(t[d] - ((m >> d) & 1) for d in range(ndim))
            if min(p) >= 0:
                assert ticket[_lin(p, nt)] < ticket[_lin(t, nt)]
    # every exact conflict between phases of different tiles: a predecessor
    # one step back, an earlier loop, and covered by the need table
    ph = _tile_phases(loops, ndim, nt, rg)
    exact = oplan.phase_conflicts(loops, st, ndim, [(l, box) for _, l, box in ph])
    for q, (t, l, _) in enumerate(ph):
        for p in exact[q]:
            tp, lp_, _ = ph[p]
            if tp == t:
                continue
            delta = tuple(t[d] - tp[d] for d in range(ndim))
            assert all(v in (0, 1) for v in delta), f"phase {(t, l)} conflicts with {(tp, lp_)}"
            assert lp_ < l
            assert need[cls[_lin(t, nt)], _dir_index(delta), l] >= lp_ + 1, \
                f"tile {t} loop {l} does not wait for loop {lp_} of tile {tp}"
    # steps: consecutive loops that share no dat with a write among them
    steps = [int(v) for v in steps]
    assert steps[0] == 0 and steps[-1] == len(loops) and all(a < b for a, b in zip(steps, steps[1:]))
    for a, b in zip(steps, steps[1:]):
        for l in range(a, b):
            for m in range(a, l):
                for x in loops[l].args:
                    for y in loops[m].args:
                        assert not (x.kind == DAT and y.kind == DAT and x.handle == y.handle and
                                    (x.access != READ or y.access != READ)), f"loops {m} and {l} share a step"
    # random interleavings that obey the plan give the program-order versions:
    # a tile runs its steps in order, the loops of a step in any order,
    # once every predecessor has completed what the step's loops need
    idx = {(t, l): q for q, (t, l, _) in enumerate(ph)}
    for _ in range(schedules):
        prog = {t: 0 for t in tiles}     # loops completed (a step's end once it ran)
        seq = []
        while True:
            ready = []
            for t in tiles:
                l0 = prog[t]
                if l0 == len(loops):
                    continue
                l1 = steps[steps.index(l0) + 1]
                ok = True
                for m in range(1, 1 << ndim):
                    p = tuple(t[d] - ((m >> d) & 1) for d in range(ndim))
                    if min(p) >= 0 and prog[p] < max(need[cls[_lin(t, nt)], m - 1, l0:l1]):
                        ok = False
                        break
                if ok:
                    ready.append(t)
            if not ready:
                break
            t = rnd.choice(ready)
            l0 = prog[t]
            l1 = steps[steps.index(l0) + 1]
            members = list(range(l0, l1))
            rnd.shuffle(members)
            seq.extend(idx[(t, l)] for l in members if (t, l) in idx)
            prog[t] = l1
        assert all(v == len(loops) for v in prog.values()), "the plan's waits deadlock"
        check_phase_order(loops, st, ndim, [(l, box) for _, l, box in ph], seq)
    return True


def test_worked_example_tilewave(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_example_1d_tilewave.json")))
    c = W.worked_example_1d()
    need, cls, order, steps = _plan(c.loops, c.stencils, 1, g["tile"])
    assert len(cls) == g["tiles"]
    assert need[cls[1], 0].tolist() == g["need_tile1"]
    assert need[cls[0], 0].tolist() == g["need_tile0"]  # no predecessor: nothing to wait for
    assert _check(c.loops, c.stencils, 1, g["tile"], random.Random(1))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_tilewave_plan_bruteforce(lib, ndim):
    rnd = random.Random(7000 + ndim)
    sizes = {1: (30,), 2: (14, 12), 3: (8, 7, 6)}[ndim]
    valid = 0
    for trial in range({1: 50, 2: 30, 3: 12}[ndim]):
        n = [rnd.randint(max(3, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 7))
        ts = [rnd.randint(2, n[d] + 2) for d in range(ndim)]
        valid += _check(loops, st, ndim, ts, rnd, schedules=2 if ndim < 3 else 1)
    assert valid >= 3, "too few random plans were valid to test anything"


def test_tilewave_plan_cloverleaf_shape(lib):
    """The bench chain's shape at 64^2 with 32x32 tiles: the plan is valid,
    covers every exact conflict and its interleavings stay in program order."""
    c = W.cloverleaf2d(n=64, steps=1)
    assert _plan(c.loops, c.stencils, 2, [16, 16]) is None  # the step's skew exceeds 16 rows
    assert _check(c.loops, c.stencils, 2, [32, 32], random.Random(3), schedules=1)


def test_tilewave_rejects_tiles_below_the_skew(lib):
    """A chain of radius-1 stencils whose skew exceeds the tile: the plan
    reports the tiles too small instead of waiting on the wrong tiles."""
    c = W.jacobi2d(16, 6)
    assert _plan(c.loops, c.stencils, 2, [2, 2]) is None
    assert _check(c.loops, c.stencils, 2, [16, 8], random.Random(4), schedules=1)


def test_tilewave_check_catches_a_weakened_plan(lib):
    """The checks above are not vacuous: with every wait of the library's
    plan shortened by one loop (planted on the CPU, in the test's copy of the
    table), the exact-conflict coverage fails on the CloverLeaf shape."""
    c = W.cloverleaf2d(n=64, steps=1)
    need, cls, order, steps = _plan(c.loops, c.stencils, 2, [32, 32])
    nt, rg, _ = oplan.skewed_plan(c.loops, c.stencils, 2, [32, 32])
    ph = _tile_phases(c.loops, 2, nt, rg)
    exact = oplan.phase_conflicts(c.loops, c.stencils, 2, [(l, box) for _, l, box in ph])
    weak = np.maximum(need - 1, 0)
    missed = 0
    for q, (t, l, _) in enumerate(ph):
        for p in exact[q]:
            tp, lp_, _ = ph[p]
            if tp == t:
                continue
            delta = tuple(t[d] - tp[d] for d in range(2))
            if weak[cls[_lin(t, nt)], _dir_index(delta), l] < lp_ + 1:
                missed += 1
    assert missed > 0
