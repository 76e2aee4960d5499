"""ops_loop_noalloc, the loop entry point for callers that must not allocate
device memory (their memory belongs to another allocator, or a cudaMalloc
would stall a GPU shared with other streams), checked against the regular
ops_par_loop path on two calls in a row.  Kept in a file of its own that
pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import paper_1704_00693_gb300 as ops
from synth import rng as R
from synth import workloads as W
from synth.program import BodyBuilder, DAT, REDARG, READ, WRITE, RW, RSUM, RMIN, RMAX, MIN

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
