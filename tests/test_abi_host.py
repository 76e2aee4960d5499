"""Host-side checks of the C ABI: no GPU needed (host-only contexts)."""
import ctypes as C
import json
import os
import random
import re

import numpy as np
import pytest

import paper_1704_00693_gb300 as ops
from paper_1704_00693_gb300 import _build
from oracle import plan as oplan
from synth import workloads as W
from synth.program import DAT, READ, WRITE, RW, INC, BodyBuilder

from bruteforce import check_phase_order, check_skewed, random_chain, random_topological

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ops.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "opstile.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ops_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/opstile.h but not exported"


def host_ctx():
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    return ops.ops_init(cfg)


def declare(ctx, chain):
    b = ops.ops_decl_block(ctx, chain.ndim)
    dats = [ops.ops_decl_dat(ctx, b, chain.size, chain.d_m, chain.d_p) for _ in chain.dats]
    st = [ops.ops_decl_stencil(ctx, chain.ndim, s) for s in chain.stencils]
    reds = [ops.ops_decl_reduction(ctx, op) for op in chain.reductions]
    return b, dats, st, reds


def enqueue(ctx, chain, b, dats, st, reds, loops=None):
    for lp in (chain.loops if loops is None else loops):
        args = [(a.kind, dats[a.handle] if a.kind == DAT else reds[a.handle], st[a.stencil] if a.kind == DAT else -1,
                 a.access) for a in lp.args]
        code = lp.code if lp.code.size else np.array([[ops.OPS_ARG_DAT, 0, 0, 0, 0, 0]], np.int32)[:0]
        ops.ops_par_loop(ctx, b, chain.ndim, lp.rng, args, code, lp.consts, lp.name)


def test_host_context_rejects_execution(lib):
    ctx = host_ctx()
    c = W.small2d(n=16, reps=1)
    b, dats, st, reds = declare(ctx, c)
    enqueue(ctx, c, b, dats, st, reds)
    with pytest.raises(ops.OpsError) as e:
        ops.ops_execute(ctx)
    assert e.value.code == ops.OPS_ERR_NO_DEVICE
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


def test_validation_errors(lib):
    ctx = host_ctx()
    b = ops.ops_decl_block(ctx, 2)
    d0 = ops.ops_decl_dat(ctx, b, (8, 8, 1), (1, 1, 0), (1, 1, 0))
    d1 = ops.ops_decl_dat(ctx, b, (8, 8, 1), (1, 1, 0), (1, 1, 0))
    p0 = ops.ops_decl_stencil(ctx, 2, [(0, 0, 0)])
    s5 = ops.ops_decl_stencil(ctx, 2, W.S5)
    far = ops.ops_decl_stencil(ctx, 2, [(2, 0, 0)])
    code, K = BodyBuilder().wsum(0, 0, [0.2] * 5).st(1, 0).build()
    rng = ((0, 8), (0, 8))
    ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, p0, WRITE)], code, K)  # fine
    # reads outside the halo
    with pytest.raises(ops.OpsError) as e:
        c2, K2 = BodyBuilder().wsum(0, 0, [1.0]).st(1, 0).build()
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, far, READ), (0, d1, p0, WRITE)], c2, K2)
    assert e.value.code == ops.OPS_ERR_BOUNDS
    # a written dat with a non-point stencil
    with pytest.raises(ops.OpsError) as e:
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, s5, WRITE)], code, K)
    assert e.value.code == ops.OPS_ERR_INVALID_ARG
    # the same dat twice
    with pytest.raises(ops.OpsError):
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d0, p0, WRITE)], code, K)
    # malformed IR: register out of range, constant pool too short, LD of a WRITE arg
    bad = code.copy()
    bad[0, 1] = 9
    with pytest.raises(ops.OpsError):
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, p0, WRITE)], bad, K)
    with pytest.raises(ops.OpsError):
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, p0, WRITE)], code, K[:3])
    c3, K3 = BodyBuilder().ld(0, 1, 0).st(1, 0).build()
    with pytest.raises(ops.OpsError):
        ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, p0, WRITE)], c3, K3)
    # INC store is allowed, reading an INC arg is not
    c4, K4 = BodyBuilder().wsum(0, 0, [0.2] * 5).st(1, 0).build()
    ops.ops_par_loop(ctx, b, 2, rng, [(0, d0, s5, READ), (0, d1, p0, INC)], c4, K4)
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


def _abi_plan(chain_like, loops, stencils, ndim, tile, overlapped_owned=None, wavefront=False):
    ctx = host_ctx()
    b = ops.ops_decl_block(ctx, ndim)
    ndats = 1 + max(a.handle for lp in loops for a in lp.args if a.kind == DAT)
    nreds = 1 + max([a.handle for lp in loops for a in lp.args if a.kind != DAT] + [-1])
    size = [1, 1, 1]
    for d in range(ndim):
        size[d] = max(lp.rng[d][1] for lp in loops) + 2
    dats = [ops.ops_decl_dat(ctx, b, size, [4 if d < ndim else 0 for d in range(3)],
                             [4 if d < ndim else 0 for d in range(3)]) for _ in range(ndats)]
    st = [ops.ops_decl_stencil(ctx, ndim, s) for s in stencils]
    reds = [ops.ops_decl_reduction(ctx, ops.OPS_RED_SUM) for _ in range(nreds)]
    for lp in loops:
        args = [(a.kind, dats[a.handle], st[a.stencil], a.access) if a.kind == DAT else
                (a.kind, reds[a.handle], -1, a.access) for a in lp.args]
        # a minimal valid body: store 0 into every written arg
        bb = BodyBuilder()
        for i, a in enumerate(lp.args):
            if a.kind == DAT and a.access != READ:
                bb.st(i, 0)
        code, K = bb.build()
        ops.ops_par_loop(ctx, b, ndim, lp.rng[:ndim], args, code, K, lp.name)
    if overlapped_owned is not None:
        out = [ops.ops_plan_overlapped(ctx, o, len(loops), ndats) for o in overlapped_owned]
    elif wavefront:
        out = ops.ops_plan_wavefront(ctx, tile)
    else:
        out = ops.ops_plan_skewed(ctx, tile, ndim, len(loops))
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)
    return out


def test_worked_example_through_abi(lib):
    c = W.worked_example_1d()
    out = _abi_plan(c, c.loops, c.stencils, 1, [4])
    assert out[0][:, 0].tolist() == [[0, 5], [5, 8]]
    assert out[0][:, 1].tolist() == [[0, 4], [4, 8]]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_library_plan_matches_oracle_plan(lib, ndim):
    """The C++ planner and the oracle's restatement of Algorithm 1 must give
    identical integer ranges; the brute-force check validates them."""
    rnd = random.Random(3000 + ndim)
    sizes = {1: (30,), 2: (12, 10), 3: (7, 6, 5)}[ndim]
    for trial in range({1: 60, 2: 30, 3: 10}[ndim]):
        n = [rnd.randint(max(2, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 7))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        got = _abi_plan(None, loops, st, ndim, ts)
        nt, rg, _ = oplan.skewed_plan(loops, st, ndim, ts)
        for d in range(ndim):
            want = np.array([[list(rg[d][t][l]) for l in range(len(loops))] for t in range(nt[d])])
            assert got[d].shape == want.shape
            assert (got[d] == want).all(), f"dim {d}: library {got[d].tolist()} oracle {want.tolist()}"
        if trial < 8:
            check_skewed(loops, st, ndim, nt, rg)


def test_cloverleaf_shaped_plan_matches_oracle(lib):
    c = W.cloverleaf2d(n=200, steps=1)
    for tile in ([200, 17], [64, 50], [210, 210]):
        got = _abi_plan(c, c.loops, c.stencils, 2, tile)
        nt, rg, _ = oplan.skewed_plan(c.loops, c.stencils, 2, tile)
        for d in range(2):
            want = np.array([[list(rg[d][t][l]) for l in range(len(c.loops))] for t in range(nt[d])])
            assert (got[d] == want).all()


def _check_wavefront(loops, st, ndim, tile, rnd):
    """The library's wavefront plan against the oracle: the same phases in
    Algorithm 2 order, every exact conflict among its dependencies, levels
    and work units as documented, and random orders of its dependency DAG
    valid under the brute-force version check."""
    ph, deps, nunits, nlevels = _abi_plan(None, loops, st, ndim, tile, wavefront=True)
    nt, rg, _ = oplan.skewed_plan(loops, st, ndim, tile)
    want = oplan.phases_in_order(loops, nt, rg, ndim)
    assert len(ph) == len(want)
    for q, (l, box) in enumerate(want):
        assert ph[q, 0] == l
        assert [(int(ph[q, 6 + 2 * d]), int(ph[q, 7 + 2 * d])) for d in range(ndim)] == list(box)
    lib_deps = [deps[ph[q, 3]:ph[q, 3] + ph[q, 4]].tolist() for q in range(len(ph))]
    exact = oplan.phase_conflicts(loops, st, ndim, want)
    for q in range(len(ph)):
        assert all(p < q for p in lib_deps[q])
        assert set(exact[q]) <= set(lib_deps[q]), f"phase {q}: missing {set(exact[q]) - set(lib_deps[q])}"
        lv = max([ph[p, 5] + 1 for p in lib_deps[q]] + [0])
        assert ph[q, 5] == lv
        assert ph[q, 1] >= 1
    assert nlevels == (int(ph[:, 5].max()) + 1 if len(ph) else 0)
    assert nunits == int(ph[:, 1].sum())
    # units: each phase's chunks contiguous, every dependency handed out first
    order = sorted(range(len(ph)), key=lambda q: ph[q, 2])
    pos = 0
    for q in order:
        assert ph[q, 2] == pos
        pos += ph[q, 1]
        assert all(ph[p, 2] < ph[q, 2] for p in lib_deps[q])
    if len(ph) <= 400:
        for k in range(2):
            check_phase_order(loops, st, ndim, want, random_topological(lib_deps, rnd))
    return ph, lib_deps


def test_wavefront_plan_worked_example(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_example_1d_wavefront.json")))
    c = W.worked_example_1d()
    ph, deps = _check_wavefront(c.loops, c.stencils, 1, g["tile"], random.Random(1))
    assert deps == g["deps"]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_library_wavefront_plan(lib, ndim):
    rnd = random.Random(5000 + ndim)
    sizes = {1: (30,), 2: (12, 10), 3: (7, 6, 5)}[ndim]
    for trial in range({1: 40, 2: 20, 3: 8}[ndim]):
        n = [rnd.randint(max(3, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 7))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        _check_wavefront(loops, st, ndim, ts, rnd)


def test_cloverleaf_shaped_wavefront_plan(lib):
    """The bench chain's shape at 40^2 with 4-row tiles: the library finds
    every conflict, and the phases of a level are many (the wavefront's
    parallelism)."""
    c = W.cloverleaf2d(n=40, steps=1)
    ph, deps = _check_wavefront(c.loops, c.stencils, 2, [44, 4], random.Random(2))
    levels = np.bincount(ph[:, 5])
    assert levels.max() >= 8
    assert len(levels) < len(ph) // 4


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_library_overlapped_tiles_match_oracle(lib, ndim):
    """The C++ overlapped-tile geometry (Sec. 4.D) and the oracle's
    restatement agree on every loop box and every read footprint; the oracle's
    is validated by brute force in the oracle pins."""
    import itertools
    rnd = random.Random(4000 + ndim)
    sizes = {1: (30,), 2: (12, 10), 3: (7, 6, 5)}[ndim]
    for trial in range({1: 40, 2: 25, 3: 10}[ndim]):
        n = [rnd.randint(max(3, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 7))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        cuts = [list(range(-2, n[d] + 2, ts[d])) for d in range(ndim)]
        tiles = [tuple((lo, min(lo + ts[d], n[d] + 2)) for d, lo in enumerate(lows))
                 for lows in itertools.product(*cuts)]
        got = _abi_plan(None, loops, st, ndim, None, overlapped_owned=tiles)
        for owned, (boxes, foot) in zip(tiles, got):
            wb, wf = oplan.overlapped_plan(loops, st, ndim, owned)
            for l in range(len(loops)):
                want = [list(wb[l][d]) for d in range(ndim)]
                have = boxes[l, :ndim].tolist()
                if any(hi <= lo for lo, hi in want):
                    assert all(hi <= lo for lo, hi in have), f"tile {owned} loop {l}: {have} vs empty"
                else:
                    assert have == want, f"tile {owned} loop {l}: library {have} oracle {want}"
            for k in range(foot.shape[0]):
                if k in wf:
                    assert foot[k, :ndim].tolist() == [list(x) for x in wf[k]], f"tile {owned} dat {k}"
                else:
                    assert all(foot[k, d, 1] < foot[k, d, 0] for d in range(ndim)), f"tile {owned} dat {k} unread"


@pytest.mark.parametrize("name,fp32", [("small2d", False), ("cloverleaf2d", False), ("cloverleaf3d", False),
                                       ("opensbli3d", False), ("edge", False), ("cloverleaf2d", True),
                                       ("edge", True)])
def test_generated_loop_bodies_compile(lib, name, fp32):
    """The CUDA generated from each workload's IR (untiled / skewed kernels
    and overlapped-tile kernels, FP64 or FP32) compiles for sm_103a (NVRTC,
    no device needed), and every loop gets its kernel."""
    from paper_1704_00693_gb300.chain import ChainRunner
    if name == "edge":
        from test_gpu_chain import edge_chain
        c = edge_chain()
    elif name == "small2d":
        c = W.small2d(n=40, reps=1)
    elif name == "cloverleaf2d":
        c = W.cloverleaf2d(n=40, steps=1)
    elif name == "cloverleaf3d":
        c = W.cloverleaf3d(n=12, steps=1)
    else:
        c = W.opensbli3d(n=12, steps=1)
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    cfg.real = ops.OPS_REAL_F32 if fp32 else ops.OPS_REAL_F64
    ctx = ops.ops_init(cfg)
    r = ChainRunner(c, ctx=ctx, upload=False, mode="untiled")
    r.enqueue_step()
    try:
        src, n, ms = ops.ops_compile_queued(ctx, want_source=True)
    except ops.OpsError as e:
        if e.code == ops.OPS_ERR_NO_DEVICE:
            pytest.skip("NVRTC is not installed")
        raise
    assert n == len(src)
    for i in range(len(c.loops)):
        assert f" u{i}(" in src
    assert ("fp32" in src) == fp32 and ("__fmaf_rn" in src) == fp32
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


@pytest.mark.parametrize("name,fp32", [("small2d", False), ("edge", False), ("edge", True)])
def test_generated_wavefront_kernel_compiles(lib, name, fp32):
    """The wavefront kernel (every loop body of the segment behind one
    dispatch on the phase's loop) compiles for sm_103a, FP64 or FP32."""
    from paper_1704_00693_gb300.chain import ChainRunner
    if name == "edge":
        from test_gpu_chain import edge_chain
        c = edge_chain()
    else:
        c = W.small2d(n=40, reps=1)
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    cfg.real = ops.OPS_REAL_F32 if fp32 else ops.OPS_REAL_F64
    ctx = ops.ops_init(cfg)
    r = ChainRunner(c, ctx=ctx, upload=False, mode="wavefront")
    r.enqueue_step()
    try:
        src, n, ms = ops.ops_compile_queued(ctx, want_source=True, wavefront=True)
    except ops.OpsError as e:
        if e.code == ops.OPS_ERR_NO_DEVICE:
            pytest.skip("NVRTC is not installed")
        raise
    assert " wf(" in src and src.count("      case ") == len(c.loops)
    assert ("fp32" in src) == fp32
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


@pytest.mark.parametrize("name,fp32,batch", [("edge", True, False), ("edge", False, True),
                                             ("opensbli3d", False, True)])
def test_generated_tilewave_kernels_compile(lib, name, fp32, batch):
    """The tile-wavefront kernel and its batch form (one launch over several
    instances' tiles) compile for sm_103a, FP64 or FP32, 2D or 3D; the batch
    form maps tickets through its (instance, tile) table and stages each
    instance's arguments in shared memory."""
    from paper_1704_00693_gb300.chain import ChainRunner
    if name == "edge":
        from test_gpu_chain import edge_chain
        c = edge_chain()
    elif name == "cloverleaf2d":
        c = W.cloverleaf2d(n=40, steps=1)
    else:
        c = W.opensbli3d(n=12, steps=1)
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    cfg.real = ops.OPS_REAL_F32 if fp32 else ops.OPS_REAL_F64
    ctx = ops.ops_init(cfg)
    r = ChainRunner(c, ctx=ctx, upload=False, mode="tilewave")
    r.enqueue_step()
    try:
        src, n, ms = ops.ops_compile_queued(ctx, want_source=True, tilewave=True, batch=batch)
    except ops.OpsError as e:
        if e.code == ops.OPS_ERR_NO_DEVICE:
            pytest.skip("NVRTC is not installed")
        raise
    assert n == len(src)
    if batch:
        assert " twb(" in src and " tw(" not in src and "tmap[tk]" in src and "s_A = AA[inst]" in src
    else:
        assert " tw(" in src and " twb(" not in src
    assert src.count("          case ") == len(c.loops)
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


def test_noalloc_rejects_overlapping_views_and_short_pitches(lib):
    """ops_loop_noalloc checks its views on the host before any device work
    (so fake device addresses do here): two views of overlapping memory
    with one of them written, and a pitch shorter than the view's rows, are
    OPS_ERR_INVALID_ARG; overlapping views that are only read are allowed
    up to the first device call."""
    from synth.program import BodyBuilder, DAT, READ, WRITE
    n = 16

    def view(addr, pitch=n + 2):
        v = ops.ops_dat_view()
        v.ptr0 = addr
        v.pitch, v.plane = pitch, pitch * (n + 2)
        v.lo[:] = [-1, -1, 0]
        v.hi[:] = [n + 1, n + 1, 1]
        return v

    code, K = BodyBuilder().wsum(0, 0, [0.2] * 5).st(1, 0).build()
    s5 = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
    base = 1 << 20
    rng = ((0, n), (0, n))
    with pytest.raises(ops.OpsError) as e:  # the same memory read through a stencil and written
        ops.ops_loop_noalloc(2, rng, [(DAT, READ), (DAT, WRITE)], [view(base), view(base)], [s5, [(0, 0, 0)]],
                             code, K)
    assert e.value.code == ops.OPS_ERR_INVALID_ARG
    with pytest.raises(ops.OpsError) as e:  # overlapping by one row
        ops.ops_loop_noalloc(2, rng, [(DAT, READ), (DAT, WRITE)],
                             [view(base), view(base + 8 * (n + 2) * (n + 1))], [s5, [(0, 0, 0)]], code, K)
    assert e.value.code == ops.OPS_ERR_INVALID_ARG
    with pytest.raises(ops.OpsError) as e:  # rows shorter than the view's x extent
        ops.ops_loop_noalloc(2, rng, [(DAT, READ), (DAT, WRITE)],
                             [view(base, pitch=n), view(base + (1 << 20))], [s5, [(0, 0, 0)]], code, K)
    assert e.value.code == ops.OPS_ERR_INVALID_ARG


def test_scalars_share_the_handle_space_but_not_reductions(lib):
    """A scalar handle can be read by SCALAR arguments but is not a
    reduction: a RED argument targeting it is rejected at enqueue, and
    ops_reduction_result refuses it."""
    from synth.program import BodyBuilder, DAT, SCALAR, REDARG, READ, WRITE
    ctx = host_ctx()
    try:
        b = ops.ops_decl_block(ctx, 2)
        d0 = ops.ops_decl_dat(ctx, b, (8, 8, 1), (1, 1, 0), (1, 1, 0))
        d1 = ops.ops_decl_dat(ctx, b, (8, 8, 1), (1, 1, 0), (1, 1, 0))
        p0 = ops.ops_decl_stencil(ctx, 2, [(0, 0, 0)])
        red = ops.ops_decl_reduction(ctx, ops.OPS_RED_SUM)
        sc = ops.ops_decl_scalar(ctx, 0.5)
        assert sc == red + 1
        code, K = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).emit(5, 2, 0, 1).st(2, 2).build()
        ops.ops_par_loop(ctx, b, 2, ((0, 8), (0, 8)), [(DAT, d0, p0, READ), (SCALAR, sc, -1, READ),
                                                        (DAT, d1, p0, WRITE)], code, K, "reads a scalar")
        code, K = BodyBuilder().ld(0, 0, 0).red(1, 0).build()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_par_loop(ctx, b, 2, ((0, 8), (0, 8)), [(DAT, d0, p0, READ), (REDARG, sc, -1, READ)], code, K,
                             "reduces into a scalar")
        assert e.value.code == ops.OPS_ERR_INVALID_ARG and "scalar" in str(e.value)
        with pytest.raises(ops.OpsError):
            ops.ops_reduction_result(ctx, sc)
        ops.ops_queue_clear(ctx)
    finally:
        ops.ops_finalize(ctx)


@pytest.mark.parametrize("name,fp32", [("edge", True), ("opensbli3d", False)])
def test_generated_tile_per_warp_kernel_compiles(lib, name, fp32):
    """The tile-per-warp kernel (warp-level ordering, per-warp shared-memory
    slices) compiles for sm_103a, 2D and 3D, FP32 and FP64."""
    from paper_1704_00693_gb300.chain import ChainRunner
    if name == "edge":
        from test_gpu_chain import edge_chain
        c = edge_chain()
    else:
        c = W.opensbli3d(n=12, steps=1)
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    cfg.real = ops.OPS_REAL_F32 if fp32 else ops.OPS_REAL_F64
    ctx = ops.ops_init(cfg)
    r = ChainRunner(c, ctx=ctx, upload=False, mode="tilewarp")
    r.enqueue_step()
    try:
        src, n, ms = ops.ops_compile_queued(ctx, want_source=True, tilewarp=True)
    except ops.OpsError as e:
        if e.code == ops.OPS_ERR_NO_DEVICE:
            pytest.skip("NVRTC is not installed")
        raise
    assert " tww(" in src and "flush_red_warp(" in src and src.count("            case ") == len(c.loops)
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


@pytest.mark.parametrize("fp32", [False, True])
def test_generated_persistent_skewed_kernel_compiles(lib, fp32):
    """The persistent skewed kernel (every body behind one switch, bounded
    grid barriers at the plan's marked phases) compiles for sm_103a."""
    from paper_1704_00693_gb300.chain import ChainRunner
    from test_gpu_chain import edge_chain
    c = edge_chain()
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    cfg.real = ops.OPS_REAL_F32 if fp32 else ops.OPS_REAL_F64
    ctx = ops.ops_init(cfg)
    r = ChainRunner(c, ctx=ctx, upload=False, mode="skewed")
    r.enqueue_step()
    try:
        src, n, ms = ops.ops_compile_queued(ctx, want_source=True, skewed=True)
    except ops.OpsError as e:
        if e.code == ops.OPS_ERR_NO_DEVICE:
            pytest.skip("NVRTC is not installed")
        raise
    assert " sk(" in src and "sk_barrier" in src and src.count("      case ") == len(c.loops)
    ops.ops_queue_clear(ctx)
    ops.ops_finalize(ctx)


def test_execute_batch_argument_checks(lib):
    """ops_execute_batch: no contexts, a NULL entry -> OPS_ERR_INVALID_ARG;
    host-only contexts cannot execute -> OPS_ERR_NO_DEVICE, queues kept."""
    import ctypes as C
    L = ops.load()
    assert L.ops_execute_batch(None, 0) == ops.OPS_ERR_INVALID_ARG
    arr = (C.c_void_p * 2)(None, None)
    assert L.ops_execute_batch(arr, 2) == ops.OPS_ERR_INVALID_ARG
    cfg = ops.ops_config_default()
    cfg.device = ops.OPS_DEVICE_NONE
    ctxs = [ops.ops_init(cfg) for _ in range(2)]
    try:
        from paper_1704_00693_gb300.chain import ChainRunner
        for ctx in ctxs:
            r = ChainRunner(W.small2d(n=16, reps=1), ctx=ctx, upload=False, mode="tilewave")
            r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_execute_batch(ctxs)
        assert e.value.code == ops.OPS_ERR_NO_DEVICE
        assert L.ops_execute_batch((C.c_void_p * 1)(ctxs[0].value), 0) == ops.OPS_ERR_INVALID_ARG
    finally:
        for ctx in ctxs:
            ops.ops_queue_clear(ctx)
            ops.ops_finalize(ctx)
