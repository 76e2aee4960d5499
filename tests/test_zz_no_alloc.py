"""ops_loop_noalloc, the loop entry point for callers that must not allocate
device memory (their memory belongs to another allocator, or a cudaMalloc
would stall a GPU shared with other streams), checked against the regular
ops_par_loop path on two calls in a row and against the oracle, with SCALAR
arguments, in 3D, on an empty range and on a loop larger than the scratch's
grid.  Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from synth import rng as R
from synth import workloads as W
from synth.program import (Arg, BodyBuilder, Chain, DatSpec, Loop, DAT, SCALAR, REDARG, READ, WRITE, RW, RSUM,
                           RMIN, RMAX, MIN, MUL)

pytestmark = pytest.mark.gpu
RED_TOL = 1e-12


def _loop():
    """Reads a (9-point) and b (point), updates c in place (RW), writes d,
    and reduces sum / min / max of the new c."""
    bb = BodyBuilder().wsum(0, 0, [0.05, 0.1, 0.05, 0.1, 0.2, 0.1, 0.05, 0.1, 0.05])
    bb.wacc(0, 1, [0.15]).ld(1, 2, 0).cst(2, 0.25).emit(6, 0, 1, 2, 0)  # r0 += 0.25 c
    bb.st(2, 0).poly(3, 0, [0.1, 0.5, -0.2]).emit(MIN, 3, 3, 1).st(3, 3)
    bb.red(4, 0).red(5, 0).red(6, 3)
    return bb.build()


def test_noalloc_matches_regular_path_two_calls():
    import torch
    from paper_1704_00693_gb300 import _build
    _build.build()
    n, h = 200, 2
    ext = n + 2 * h
    inits = [R.uniform(R.subseed(5, "noalloc", k), (1, ext, ext), 0.5, 1.5) for k in range(4)]
    code, K = _loop()
    rng = ((0, n), (0, n))
    # regular path: a context with library-owned dats
    cfg = ops.ops_config_default()
    ctx = ops.ops_init(cfg)
    try:
        b = ops.ops_decl_block(ctx, 2)
        dats = [ops.ops_decl_dat(ctx, b, (n, n, 1), (h, h, 0), (h, h, 0)) for _ in range(4)]
        for d, a in zip(dats, inits):
            ops.ops_dat_upload(ctx, d, a)
        s9 = ops.ops_decl_stencil(ctx, 2, W.S9)
        p0 = ops.ops_decl_stencil(ctx, 2, W.P0)
        reds = [ops.ops_decl_reduction(ctx, op) for op in (RSUM, RMIN, RMAX)]
        args = [(DAT, dats[0], s9, READ), (DAT, dats[1], p0, READ), (DAT, dats[2], p0, RW),
                (DAT, dats[3], p0, WRITE), (REDARG, reds[0], -1, 0), (REDARG, reds[1], -1, 0),
                (REDARG, reds[2], -1, 0)]
        # caller-owned dats for the allocation-free path (torch tensors, pitch 224)
        pitch = 224
        tens = []
        for a in inits:
            t = torch.zeros((ext, pitch), dtype=torch.float64, device="cuda")
            t[:, :ext] = torch.from_numpy(a[0])
            tens.append(t)
        torch.cuda.synchronize()
        views = []
        for t in tens:
            v = ops.ops_dat_view()
            v.ptr0 = t.data_ptr() + 8 * (h + pitch * h)
            v.pitch, v.plane = pitch, pitch * ext
            v.lo[:] = [-h, -h, 0]
            v.hi[:] = [n + h, n + h, 1]
            views.append(v)
        na_args = [(DAT, READ), (DAT, READ), (DAT, RW), (DAT, WRITE), (REDARG, 0), (REDARG, 0), (REDARG, 0)]
        stencils = [W.S9, W.P0, W.P0, W.P0, None, None, None]
        red_ops = [0, 0, 0, 0, RSUM, RMIN, RMAX]
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            ops.ops_par_loop(ctx, b, 2, rng, args, code, K, "regular")
            want = [ops.ops_reduction_result(ctx, r) for r in reds]
            got = ops.ops_loop_noalloc(2, rng, na_args, views + [None] * 3, stencils, code, K,
                                       red_ops=red_ops, stream=stream)[4:]
            torch.cuda.synchronize()
            for k in (2, 3):
                ref = ops.ops_dat_fetch(ctx, dats[k])[0]
                mine = tens[k][:, :ext].cpu().numpy()
                assert np.array_equal(ref, mine), f"call {call}: dat {k} differs"
            assert abs(got[0] - want[0]) <= RED_TOL * abs(want[0]), (call, got[0], want[0])
            assert got[1] == want[1] and got[2] == want[2], (call, got, want)
    finally:
        ops.ops_finalize(ctx)


def test_noalloc_rejects_requests_beyond_scratch():
    from paper_1704_00693_gb300 import _build
    _build.build()
    ops.load()
    code = np.zeros((65, 6), dtype=np.int32)  # one instruction more than OPS_MAX_INS
    with pytest.raises(ops.OpsError) as e:
        ops.ops_loop_noalloc(2, ((0, 4), (0, 4)), [], [], [], code, [0.0])
    assert e.value.code == ops.OPS_ERR_NOMEM


def _views(tens, h, ext_xyz, dims, pitch):
    views = []
    for t in tens:
        v = ops.ops_dat_view()
        plane = pitch * ext_xyz[1]
        v.ptr0 = t.data_ptr() + 8 * (h + pitch * h + (plane * h if dims == 3 else 0))
        v.pitch, v.plane = pitch, plane
        v.lo[:] = [-h, -h, -h if dims == 3 else 0]
        v.hi[:] = [ext_xyz[0] - h, ext_xyz[1] - h, ext_xyz[2] - h if dims == 3 else 1]
        views.append(v)
    return views


def _oracle_one_loop(dims, n, h, inits, stencils, arg_list, code, K, red_ops):
    """The oracle's result for one loop over [0, n)^dims (dats with halo h)."""
    st = []
    args = []
    ndat = 0
    for (kind, acc), sp in zip(arg_list, stencils):
        if kind == DAT:
            st.append(list(sp))
            args.append(Arg(DAT, ndat, len(st) - 1, acc))
            ndat += 1
        else:
            args.append(Arg(REDARG, len([a for a in args if a.kind == REDARG])))
    size = tuple(n if d < dims else 1 for d in range(3))
    hh = tuple(h if d < dims else 0 for d in range(3))
    rng = tuple((0, n) if d < dims else (0, 1) for d in range(3))
    lp = Loop("one", rng[:dims] if dims < 3 else rng, args, code, K)
    reds = [r for (kind, _), r in zip(arg_list, red_ops) if kind == REDARG]
    ch = Chain("one", dims, size, hh, hh, [DatSpec(f"d{k}", a) for k, a in enumerate(inits)], st, reds, [lp])
    return oracle.run_chain(ch)


def test_noalloc_matches_oracle_3d_and_2d():
    """The dats the loop writes equal the oracle's bit for bit; the sum
    within 1e-12 relative of the exactly rounded one, min and max exactly;
    in 2D (pitched rows) and in 3D (pitched planes)."""
    import torch
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()
    code, K = _loop()
    arg_list = [(DAT, READ), (DAT, READ), (DAT, RW), (DAT, WRITE), (REDARG, 0), (REDARG, 0), (REDARG, 0)]
    red_ops = [0, 0, 0, 0, RSUM, RMIN, RMAX]
    for dims, n in ((2, 150), (3, 40)):
        h = 2
        ext = n + 2 * h
        shape = (ext if dims == 3 else 1, ext, ext)
        s9 = W.S9 if dims == 2 else W.S27
        stencils = [s9, W.P0, W.P0, W.P0, None, None, None]
        if dims == 3:
            bb = BodyBuilder().wsum(0, 0, [1.0 / 27] * 27)
            bb.wacc(0, 1, [0.15]).ld(1, 2, 0).cst(2, 0.25).emit(6, 0, 1, 2, 0)
            bb.st(2, 0).poly(3, 0, [0.1, 0.5, -0.2]).emit(MIN, 3, 3, 1).st(3, 3)
            bb.red(4, 0).red(5, 0).red(6, 3)
            code, K = bb.build()
        inits = [R.uniform(R.subseed(6, "noalloc3", dims, k), shape, 0.5, 1.5) for k in range(4)]
        ref, hist = _oracle_one_loop(dims, n, h, inits, stencils, arg_list, code, K, red_ops)
        pitch = ext + 3
        tens = []
        for a in inits:
            t = torch.zeros((shape[0], ext, pitch), dtype=torch.float64, device="cuda")
            t[:, :, :ext] = torch.from_numpy(a)
            tens.append(t)
        torch.cuda.synchronize()
        views = _views(tens, h, (ext, ext, ext), dims, pitch)
        rng = tuple((0, n) for _ in range(dims))
        stream = torch.cuda.current_stream().cuda_stream
        got = ops.ops_loop_noalloc(dims, rng, arg_list, views + [None] * 3, stencils, code, K,
                                   red_ops=red_ops, stream=stream)[4:]
        torch.cuda.synchronize()
        for k in (2, 3):
            assert np.array_equal(tens[k][:, :, :ext].cpu().numpy(), ref[k]), f"{dims}D dat {k}"
        assert abs(got[0] - hist[0][0]) <= RED_TOL * abs(hist[0][0])
        assert got[1] == hist[0][1] and got[2] == hist[0][2]


def test_noalloc_scalar_arguments_and_empty_range():
    """SCALAR arguments read the values passed in (w = a * s0 + s1, each
    rounded as the IR says); an empty range leaves the dats alone and
    returns every reduction's identity."""
    import torch
    from paper_1704_00693_gb300 import _build
    _build.build()
    n, h = 64, 1
    ext = n + 2
    a = R.uniform(R.subseed(8, "noalloc_s"), (1, ext, ext), 0.5, 1.5)
    ta = torch.from_numpy(a[0].copy()).cuda()
    tw = torch.zeros((ext, ext), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    views = _views([ta, tw], h, (ext, ext, 1), 2, ext)
    bb = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).ld(2, 2, 0).emit(6, 3, 0, 1, 2).st(3, 3).red(4, 3)
    code, K = bb.build()
    s0, s1 = 0.3125, -0.7
    args = [(DAT, READ), (SCALAR, READ), (SCALAR, READ), (DAT, WRITE), (REDARG, 0)]
    st = [W.P0, None, None, W.P0, None]
    got = ops.ops_loop_noalloc(2, ((0, n), (0, n)), args, [views[0], None, None, views[1], None], st, code, K,
                               scalar_values=[0, s0, s1, 0, 0], red_ops=[0, 0, 0, 0, RMAX])
    torch.cuda.synchronize()
    from fractions import Fraction
    inner = a[0, h:h + n, h:h + n]
    want = np.vectorize(lambda v: float(Fraction(float(v)) * Fraction(s0) + Fraction(s1)))(inner)
    w = tw.cpu().numpy()
    assert np.array_equal(w[h:h + n, h:h + n], want)
    assert got[4] == want.max()
    # empty range: identities, nothing written
    tw.zero_()
    torch.cuda.synchronize()
    bb = BodyBuilder().ld(0, 0, 0).st(1, 0).red(2, 0).red(3, 0).red(4, 0)
    code, K = bb.build()
    got = ops.ops_loop_noalloc(2, ((5, 5), (0, n)), [(DAT, READ), (DAT, WRITE), (REDARG, 0), (REDARG, 0),
                                                     (REDARG, 0)],
                               [views[0], views[1], None, None, None], [W.P0, W.P0, None, None, None], code, K,
                               red_ops=[0, 0, RSUM, RMIN, RMAX])
    torch.cuda.synchronize()
    assert got[2] == 0.0 and got[3] == float("inf") and got[4] == float("-inf")
    assert not tw.any().item()


def test_noalloc_bounds_and_large_loop():
    """A view too small for the stencil returns OPS_ERR_BOUNDS; on a loop
    with more enumeration units than the scratch holds CTAs (3840^2) the
    dats still equal the regular path's and the sum agrees within 1e-12."""
    import torch
    from paper_1704_00693_gb300 import _build
    _build.build()
    n, h = 3840, 1
    ext = n + 2
    a = R.uniform(R.subseed(9, "noalloc_big"), (1, ext, ext), 0.5, 1.5)
    ta = torch.from_numpy(a[0].copy()).cuda()
    tw = torch.zeros((ext, ext), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    views = _views([ta, tw], h, (ext, ext, 1), 2, ext)
    code, K = BodyBuilder().wsum(0, 0, [0.2, 0.1, 0.3, 0.15, 0.25]).st(1, 0).red(2, 0).build()
    args = [(DAT, READ), (DAT, WRITE), (REDARG, 0)]
    small = ops.ops_dat_view()
    small.ptr0, small.pitch, small.plane = views[0].ptr0, ext, ext * ext
    small.lo[:] = [0, 0, 0]
    small.hi[:] = [n, n, 1]
    with pytest.raises(ops.OpsError) as e:
        ops.ops_loop_noalloc(2, ((0, n), (0, n)), args, [small, views[1], None], [W.S5, W.P0, None], code, K,
                             red_ops=[0, 0, RSUM])
    assert e.value.code == ops.OPS_ERR_BOUNDS
    got = ops.ops_loop_noalloc(2, ((0, n), (0, n)), args, [views[0], views[1], None], [W.S5, W.P0, None], code, K,
                               red_ops=[0, 0, RSUM])
    torch.cuda.synchronize()
    cfg = ops.ops_config_default()
    cfg.mode = ops.OPS_MODE_UNTILED
    ctx = ops.ops_init(cfg)
    try:
        b = ops.ops_decl_block(ctx, 2)
        d0 = ops.ops_decl_dat(ctx, b, (n, n, 1), (h, h, 0), (h, h, 0))
        d1 = ops.ops_decl_dat(ctx, b, (n, n, 1), (h, h, 0), (h, h, 0))
        ops.ops_dat_upload(ctx, d0, a)
        s5 = ops.ops_decl_stencil(ctx, 2, W.S5)
        p0 = ops.ops_decl_stencil(ctx, 2, W.P0)
        red = ops.ops_decl_reduction(ctx, RSUM)
        ops.ops_par_loop(ctx, b, 2, ((0, n), (0, n)), [(DAT, d0, s5, READ), (DAT, d1, p0, WRITE),
                                                       (REDARG, red, -1, 0)], code, K, "big")
        want = ops.ops_reduction_result(ctx, red)
        ref = ops.ops_dat_fetch(ctx, d1)[0]
    finally:
        ops.ops_finalize(ctx)
    assert np.array_equal(tw.cpu().numpy()[h:h + n, h:h + n], ref[h:h + n, h:h + n])
    assert abs(got[2] - want) <= RED_TOL * abs(want)
