"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Every execution mode must reproduce the untiled program-order result of the
oracle bit for bit (explicitly rounded IEEE operations on both sides, no
contraction); reductions, whose summation order differs, within 1e-12
relative of the exactly rounded oracle value (min/max exactly).
"""
import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from paper_1704_00693_gb300.chain import ChainRunner
from synth import workloads as W
from synth.program import (Arg, BodyBuilder, Chain, DatSpec, Loop, DAT, REDARG, SCALAR, READ, WRITE, RW, INC,
                           RSUM, RMIN, RMAX, FMA, ADD, MUL)
from synth import rng as R

pytestmark = pytest.mark.gpu

RED_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()


def run_gpu(chain, mode, tile=None, steps=None, **kw):
    r = ChainRunner(chain, mode=mode, tile=tile, **kw)
    try:
        hist = r.run(steps)
        dats = r.fetch()
        stats = r.stats()
    finally:
        r.close()
    return dats, hist, stats


def assert_same(chain, got, ref, hist=None, ref_hist=None, what=""):
    for k, (a, b) in enumerate(zip(got, ref)):
        if not np.array_equal(a, b):
            diff = np.argwhere(a != b)
            raise AssertionError(f"{what}: dat {chain.dats[k].name} differs at {len(diff)} points, first {diff[:3]}, "
                                 f"max abs diff {np.nanmax(np.abs(a - b))}")
    if hist is not None:
        for s, (h1, h2) in enumerate(zip(hist, ref_hist)):
            for i, (v1, v2) in enumerate(zip(h1, h2)):
                op = chain.reductions[i]
                if op == RSUM:
                    assert abs(v1 - v2) <= RED_TOL * abs(v2), f"{what}: step {s} sum {v1} vs {v2}"
                else:
                    assert v1 == v2, f"{what}: step {s} min/max {v1} vs {v2}"


def test_worked_example_1d():
    c = W.worked_example_1d()
    ref, _ = oracle.run_chain(c)
    for mode, tile in [("untiled", None), ("skewed", (4,)), ("skewed", (1,)), ("skewed", (3,)),
                       ("overlapped", (4,)), ("overlapped", (1,)), ("overlapped", (3,)),
                       ("wavefront", (4,)), ("wavefront", (1,)), ("wavefront", (3,))]:
        for interp in (False, True):
            got, _, st = run_gpu(c, mode, tile, interpret=interp)
            assert_same(c, got, ref, what=f"{mode} {tile} interpret={interp}")


@pytest.mark.parametrize("interpret", [False, True])
@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 0, 0)), ("skewed", (0, 40, 0)),
                                       ("skewed", (100, 33, 0)), ("overlapped", (0, 0, 0)),
                                       ("overlapped", (64, 16, 0)), ("overlapped", (100, 33, 0)),
                                       ("wavefront", (0, 0, 0)), ("wavefront", (0, 4, 0)),
                                       ("wavefront", (100, 33, 0))])
def test_small2d_chain_bit_exact(mode, tile, interpret):
    """8 loops x 10 repetitions on 256^2 (radius-1 stencils, zero halo)."""
    c = W.small2d(n=256, reps=10)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, mode, tile, interpret=interpret)
    assert_same(c, got, ref, what=f"{mode} {tile}")
    if mode == "skewed":
        assert st["mode"] == ops.OPS_MODE_SKEWED
    if mode == "wavefront":
        # interpreted bodies take the persistent skewed kernel instead
        assert st["mode"] == (ops.OPS_MODE_SKEWED if interpret else ops.OPS_MODE_WAVEFRONT)
    if mode == "overlapped":
        # one run of the 8 loops of a step: radius-1 halos grow to 8 points
        assert st["mode"] == ops.OPS_MODE_OVERLAPPED and st["segments"] >= 1
        assert st["redundant_points"] > 0 and st["loops"] == len(c.loops)


@pytest.mark.parametrize("interpret", [False, True])
@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 32, 0)), ("skewed", (0, 17, 0)),
                                       ("skewed", (37, 23, 0)), ("skewed", (0, 0, 0)), ("auto", None),
                                       ("overlapped", None), ("overlapped", (32, 8, 0)),
                                       ("overlapped", (40, 100, 0)), ("wavefront", (0, 0, 0)),
                                       ("wavefront", (0, 5, 0)), ("wavefront", (37, 8, 0))])
def test_cloverleaf_shaped_chain(mode, tile, interpret):
    """83-loop CloverLeaf-shaped steps on a 100^2 grid (ragged tiles), with
    node ranges, thin halo strips, RW updates and two reductions per step;
    the min reduction feeds the next step's constants.  Loop bodies run
    compiled from the IR, or through the interpreter kernels."""
    c = W.cloverleaf2d(n=100, steps=3)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, mode, tile, interpret=interpret)
    assert_same(c, got, ref, hist, ref_hist, what=f"{mode} {tile} interpret={interpret}")
    if mode in ("untiled", "skewed"):
        assert st["compiled"] == (0 if interpret else 1)


@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 0, 0)), ("skewed", (0, 9, 7)),
                                       ("overlapped", None), ("auto", None), ("wavefront", (0, 0, 3))])
def test_cloverleaf3d_shaped_chain(mode, tile):
    """141-loop CloverLeaf-3D-shaped steps on 40^3 (7-, 27- and one-sided
    8-point stencils, node ranges, halo planes, two reductions per step)."""
    c = W.cloverleaf3d(n=40, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, mode, tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"3d hydro {mode} {tile}")


@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 0, 0)), ("skewed", (0, 16, 0)),
                                       ("overlapped", None), ("overlapped", (64, 16, 0)), ("auto", None),
                                       ("wavefront", (0, 0, 0)), ("wavefront", (0, 3, 0))])
def test_ppcg_shaped_chain(mode, tile):
    """The TeaLeaf-PPCG-shaped chain: setup loops, then 10 Chebyshev inner
    iterations (three loops each, no reduction) in one segment, and z.r."""
    c = W.ppcg2d(n=100, inner=10, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, mode, tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"ppcg {mode} {tile}")


def test_jacobi_eigenmode_closed_form_on_gpu():
    n, K, nu = 63, 30, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=2, q=1)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "skewed", (0, 16, 0))
    assert_same(c, got, ref, what="jacobi")
    import math
    lam = -4 * math.sin(math.pi * 2 / (2 * (n + 1))) ** 2 - 4 * math.sin(math.pi * 1 / (2 * (n + 1))) ** 2
    want = c.dats[0].init * (1 + nu * lam) ** K
    assert np.abs(got[0] - want).max() <= 1e-13 * np.abs(want).max()
    assert st["barriers"] > 0 and st["tiles"] == 4


def test_jacobi_overlapped_closed_form():
    """Overlapped tiles recompute halo points redundantly; the result is still
    the program-order one, and the eigenmode decays by the closed form."""
    n, K, nu = 63, 30, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=2, q=1)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "overlapped", (32, 16, 0))
    assert_same(c, got, ref, what="jacobi overlapped")
    # 60 loops in one flush: cut into runs whose recomputation stays bounded
    assert st["mode"] == ops.OPS_MODE_OVERLAPPED and st["redundant_points"] > 0
    assert st["segments"] > 1 and st["loops"] == len(c.loops)


def test_constant_and_linear_fields():
    c = W.small2d(n=48, reps=2, constant=0.75)
    got, _, _ = run_gpu(c, "skewed", (0, 10, 0))
    for d in got:
        assert (d == 0.75).all()
    a0, bx, by = 0.5, 0.25, -0.375
    c = W.linear2d(40, a0, bx, by)
    ref, _ = oracle.run_chain(c)
    got, _, _ = run_gpu(c, "skewed", (0, 7, 0))
    assert_same(c, got, ref, what="linear")


def test_opensbli_shaped_3d():
    c = W.opensbli3d(n=20, steps=1)
    ref, _ = oracle.run_chain(c)
    for mode, tile, interp in [("untiled", None, False), ("skewed", (0, 0, 6), False), ("skewed", (0, 7, 5), False),
                               ("untiled", None, True), ("skewed", (0, 7, 5), True),
                               ("overlapped", (0, 0, 0), False), ("overlapped", (8, 7, 5), False),
                               ("wavefront", (0, 0, 0), False), ("wavefront", (0, 7, 2), False)]:
        got, _, st = run_gpu(c, mode, tile, interpret=interp)
        assert_same(c, got, ref, what=f"3d {mode} {tile} interpret={interp}")


def edge_chain(n=30):
    """Edge cases: an empty range, a one-point range, INC and RW updates, a
    1-wide strip, a loop reading a reduction through a SCALAR argument
    (splits the segment), MIN/MAX/SUM reductions, DIV and SGT."""
    size, d_m, d_p = (n, n, 1), (2, 2, 0), (2, 2, 0)
    shp = (1, n + 4, n + 4)
    dats = [DatSpec(f"e{k}", R.uniform(R.subseed(99, "edge", k), shp, 0.5, 1.5)) for k in range(4)]
    st = [[(0, 0, 0)], W.S5, W.S4P, [(-2, 0, 0), (2, 0, 0), (0, -2, 0), (0, 2, 0)]]
    loops = []
    c, K = BodyBuilder().wsum(0, 0, [0.2] * 5).st(1, 0).build()
    loops.append(Loop("empty", ((5, 5), (0, n)), [Arg(DAT, 0, 1, READ), Arg(DAT, 1, 0, WRITE)], c, K))
    loops.append(Loop("onept", ((3, 4), (7, 8)), [Arg(DAT, 0, 1, READ), Arg(DAT, 1, 0, WRITE)], c, K))
    c, K = BodyBuilder().wsum(0, 0, [0.1, 0.2, 0.3, 0.1]).st(1, 0).build()
    loops.append(Loop("inc", ((0, n), (0, n)), [Arg(DAT, 0, 2, READ), Arg(DAT, 2, 0, INC)], c, K))
    bb = BodyBuilder().ld(0, 1, 0).ld(1, 0, 0).emit(7, 2, 0, 1)  # DIV
    bb.cst(3, 1.0).emit(10, 4, 2, 3, 0, 1).st(1, 4)  # SGT
    c, K = bb.build()
    loops.append(Loop("rw_div_sgt", ((-1, n + 1), (0, n)), [Arg(DAT, 0, 0, READ), Arg(DAT, 1, 0, RW)], c, K))
    c, K = BodyBuilder().wsum(0, 0, [0.25, 0.25, 0.25, 0.25]).st(1, 0).build()
    loops.append(Loop("strip", ((0, n), (0, 1)), [Arg(DAT, 1, 3, READ), Arg(DAT, 3, 0, WRITE)], c, K))
    bb = BodyBuilder().wsum(0, 0, [0.3, -0.1, 0.2, 0.05, 0.15]).red(1, 0).red(2, 0).red(3, 0)
    c, K = bb.build()
    loops.append(Loop("reds", ((0, n), (0, n)), [Arg(DAT, 2, 1, READ), Arg(REDARG, 0), Arg(REDARG, 1),
                                                 Arg(REDARG, 2)], c, K))
    bb = BodyBuilder().ld(0, 1, 0).ld(1, 2, 0).ld(2, 0, 0).emit(FMA, 3, 0, 2, 1).st(3, 3)
    c, K = bb.build()
    # min and max are exact whatever the order, so the dats stay bit-exact
    loops.append(Loop("use_scalar", ((0, n), (0, n)), [Arg(DAT, 0, 0, READ), Arg(SCALAR, 1), Arg(SCALAR, 2),
                                                       Arg(DAT, 3, 0, WRITE)], c, K))
    c, K = BodyBuilder().wsum(0, 0, [0.5] + [0.125] * 4).st(1, 0).build()
    loops.append(Loop("after", ((0, n), (0, n)), [Arg(DAT, 3, 1, READ), Arg(DAT, 0, 0, WRITE)], c, K))
    return Chain("edge", 2, size, d_m, d_p, dats, st, [RSUM, RMIN, RMAX], loops, steps=2)


@pytest.mark.parametrize("interpret", [False, True])
@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 7, 0)), ("skewed", (11, 5, 0)),
                                       ("overlapped", None), ("overlapped", (11, 5, 0)), ("wavefront", (0, 3, 0)),
                                       ("wavefront", (11, 5, 0))])
def test_edge_cases(mode, tile, interpret):
    c = edge_chain()
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, mode, tile, interpret=interpret)
    assert_same(c, got, ref, hist, ref_hist, what=f"edge {mode} {tile}")


def test_checked_mode_same_result():
    c = W.cloverleaf2d(n=64, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, _ = run_gpu(c, "skewed", (0, 16, 0), check=True)
    assert_same(c, got, ref, hist, ref_hist, what="checked")


def test_barrier_timeout_reports_and_context_recovers():
    """One CTA never arrives at grid barriers: every wait gives up after the
    limit, the kernel returns, the host sees OPS_ERR_TIMEOUT; a new context
    on the same device then runs normally."""
    c = W.small2d(n=64, reps=1)
    # the persistent skewed kernel (interpreted bodies) is the one with grid barriers
    r = ChainRunner(c, mode="skewed", tile=(0, 8, 0), timeout_ms=200, skip_barrier_block=0, interpret=True)
    try:
        r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(r.ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
    finally:
        r.close()
    ref, _ = oracle.run_chain(c)
    got, _, _ = run_gpu(c, "skewed", (0, 8, 0))
    assert_same(c, got, ref, what="after timeout")


def test_compiled_skewed_barrier_timeout_reports_and_context_recovers():
    """The same with compiled bodies: the persistent skewed kernel's grid
    barriers give up after the limit, every CTA leaves, OPS_ERR_TIMEOUT."""
    c = W.small2d(n=64, reps=1)
    r = ChainRunner(c, mode="skewed", tile=(0, 8, 0), timeout_ms=200, skip_barrier_block=0,
                    skewed_persistent=True)
    try:
        r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(r.ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
        assert r.stats()["kernel_launches"] == 1  # one persistent launch, not one per phase
    finally:
        r.close()
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "skewed", (0, 8, 0), skewed_persistent=True)
    assert_same(c, got, ref, what="after timeout")
    assert st["kernel_launches"] == st["segments"]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("name,tile", [("cloverleaf2d", (0, 0, 0)), ("cloverleaf2d", (0, 40, 0)),
                                       ("ppcg2d", (0, 24, 0)), ("cloverleaf3d", (0, 0, 8))])
def test_persistent_skewed_kernel_bit_exact(name, tile, fp32):
    """The persistent skewed kernel (one cooperative launch per segment, grid
    barriers only at the plan's marked phases) against the oracle."""
    c = {"cloverleaf2d": lambda: W.cloverleaf2d(n=130, steps=2), "ppcg2d": lambda: W.ppcg2d(n=100, inner=10, steps=2),
         "cloverleaf3d": lambda: W.cloverleaf3d(n=24, steps=1)}[name]()
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, "skewed", tile, fp32=fp32, skewed_persistent=True)
    assert_same(c, got, ref, hist, ref_hist, what=f"persistent skewed {name} {tile} fp32={fp32}")
    assert st["mode"] == ops.OPS_MODE_SKEWED and 4 * st["kernel_launches"] <= st["phases"]


def test_wavefront_timeout_reports_and_context_recovers():
    """The wavefront kernel's first work unit never reports completion: the
    phases waiting on it give up after the limit, every CTA leaves, the host
    sees OPS_ERR_TIMEOUT; a new context on the same device then runs the
    same chain in wavefront mode normally."""
    c = W.small2d(n=64, reps=1)
    r = ChainRunner(c, mode="wavefront", tile=(0, 4, 0), timeout_ms=200, skip_barrier_block=0)
    try:
        r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(r.ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
    finally:
        r.close()
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "wavefront", (0, 4, 0))
    assert st["mode"] == ops.OPS_MODE_WAVEFRONT
    assert_same(c, got, ref, what="after timeout")


def test_wavefront_jacobi_closed_form_and_stats():
    """Jacobi steps in wavefront mode reproduce the Dirichlet eigenmode's
    closed-form decay; the plan is cached and one kernel runs per flush."""
    import math
    n, K, nu = 62, 30, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=2, q=1)
    ref, _ = oracle.run_chain(c)
    r = ChainRunner(c, mode="wavefront", tile=(0, 4, 0))
    try:
        r.run()
        got = r.fetch()
        st = r.stats()
        r.run()
        st2 = r.stats()
    finally:
        r.close()
    assert_same(c, got, ref, what="jacobi wavefront")
    assert st["mode"] == ops.OPS_MODE_WAVEFRONT and st["barriers"] == 0
    assert st["kernel_launches"] == st["segments"] >= 1
    assert st["tiles"] == math.ceil(n / 4) and st["tile"][1] == 4
    assert st2["plan_cache_hits"] >= 1
    lam = -4 * math.sin(math.pi * 2 / (2 * (n + 1))) ** 2 - 4 * math.sin(math.pi * 1 / (2 * (n + 1))) ** 2
    want = c.dats[0].init * (1 + nu * lam) ** K
    assert np.abs(got[0] - want).max() <= 1e-13 * np.abs(want).max()


def test_wavefront_segments_and_single_loop_segments():
    """A flush cut into segments of at most 10 loops runs one wavefront
    kernel per segment of several loops; a segment length of 1 runs every
    loop untiled.  Both give the program-order result."""
    c = W.cloverleaf2d(n=90, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "wavefront", (0, 8, 0), segment=10)
    assert_same(c, got, ref, hist, ref_hist, what="wavefront segments")
    assert st["segments"] >= 8 and st["kernel_launches"] == st["segments"]
    got, hist, st = run_gpu(c, "wavefront", (0, 8, 0), segment=1)
    assert_same(c, got, ref, hist, ref_hist, what="wavefront one-loop segments")
    assert st["mode"] == ops.OPS_MODE_UNTILED


def test_plan_cache_reuse_and_stats():
    c = W.cloverleaf2d(n=80, steps=3)
    r = ChainRunner(c, mode="skewed", tile=(0, 20, 0))
    try:
        r.step()
        s1 = r.stats()
        r.step()
        s2 = r.stats()
    finally:
        r.close()
    assert s1["plan_cache_hits"] == 0 and s1["plan_ms"] > 0
    assert s2["plan_cache_hits"] >= 1 and s2["plan_ms"] == 0
    assert s2["tiles"] == 5 and s2["loops"] == len(c.loops)


def test_autotuner_settles_and_stays_exact():
    """AUTO mode times one candidate schedule per step (untiled, skewed tiles
    of growing height, overlapped), round robin until each has two samples,
    then keeps the fastest; every step's dats stay bit-identical to the
    oracle whichever candidate ran."""
    c = W.cloverleaf2d(n=120, steps=20)
    ref, ref_hist = oracle.run_chain(c)
    r = ChainRunner(c, mode="auto")
    try:
        tuning = []
        for _ in range(c.steps):
            r.step()
            tuning.append(r.stats()["tuning"])
        got = r.fetch()
        hist = r.history
    finally:
        r.close()
    assert tuning[0] == 1 and tuning[-1] == 0
    assert_same(c, got, ref, hist, ref_hist, what="auto")


def test_full_size_cloverleaf_one_step():
    """The benchmark's workload (3840^2, 83 loops, automatic tiles, the
    benchmark's launch configuration) for one step, every point checked."""
    c = W.cloverleaf2d(n=3840, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "skewed")
    assert_same(c, got, ref, hist, ref_hist, what="full size skewed")
    assert st["tiles"] > 1 and st["compiled"] == 1
    got, hist, st = run_gpu(c, "untiled")
    assert_same(c, got, ref, hist, ref_hist, what="full size untiled")
    assert st["compiled"] == 1


def test_async_dat_copies_match_blocking_ones():
    """ops_dat_upload_async / ops_dat_fetch_async queue the same copies as the
    blocking calls: a step run on asynchronously uploaded dats and fetched
    asynchronously equals the oracle."""
    import torch
    c = W.cloverleaf2d(n=64, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    r = ChainRunner(c, mode="untiled", upload=False)
    try:
        host_in = [torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True).numpy() for d in c.dats]
        for a, d in zip(host_in, c.dats):
            a[...] = d.init
        for h, a in zip(r.dats, host_in):
            ops.ops_dat_upload_async(r.ctx, h, a)
        r.step()
        out = [torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True).numpy() for d in c.dats]
        for h, a in zip(r.dats, out):
            ops.ops_dat_fetch_async(r.ctx, h, a)
        ops.ops_sync(r.ctx)
        hist = r.history
    finally:
        r.close()
    assert_same(c, out, ref, hist, ref_hist, what="async copies")


def test_full_size_opensbli_one_step():
    """The OpenSBLI-shaped chain at its full size (320^3, 15 dats, 40 loops,
    radius-2 stencils in all three directions) for one step, every point
    checked, untiled and in the autotuner's first skewed candidate."""
    c = W.opensbli3d(n=320, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    for mode in ("untiled", "skewed"):
        got, hist, st = run_gpu(c, mode)
        assert_same(c, got, ref, hist, ref_hist, what=f"opensbli 320^3 {mode}")
        assert st["compiled"] == 1
        del got


@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 16, 0)), ("overlapped", None),
                                       ("auto", None), ("wavefront", (0, 8, 0)), ("tilewave", (0, 0, 0))])
def test_borrowed_device_dats(mode, tile):
    """Dats declared on caller-owned device memory (torch tensors with a pitch
    of their own): the chain reads and writes them in place in every mode
    (overlapped tiles need library-owned dats and run the segment skewed)."""
    import torch
    c = W.cloverleaf2d(n=70, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    ez, ey, ex = c.dats[0].init.shape
    pitch = ex + 5  # rows padded unlike the library's own layout
    ctx = ops.ops_init()
    try:
        ts = []
        for d in c.dats:
            t = torch.zeros((ez, ey, pitch), dtype=torch.float64, device="cuda")
            t[:, :, :ex] = torch.from_numpy(d.init)
            ts.append(t)
        torch.cuda.synchronize()
        r = ChainRunner(c, mode=mode, tile=tile, ctx=ctx, upload=False)
        # replace the library's dats by borrowed ones (same order, same shapes)
        r.dats = []
        for t in ts:
            p0 = t.data_ptr() + 8 * (c.d_m[0] + pitch * c.d_m[1])
            r.dats.append(ops.ops_decl_dat(ctx, r.block, c.size, c.d_m, c.d_p, p0, pitch, pitch * ey))
        hist = r.run()
        torch.cuda.synchronize()
        got = [t[:, :, :ex].cpu().numpy() for t in ts]
        st = r.stats()
    finally:
        ops.ops_finalize(ctx)
    assert_same(c, got, ref, hist, ref_hist, what=f"borrowed {mode}")
    if mode == "overlapped":
        assert st["mode"] == ops.OPS_MODE_SKEWED
    if mode == "wavefront":
        assert st["mode"] == ops.OPS_MODE_WAVEFRONT
    if mode == "tilewave":
        assert st["mode"] == ops.OPS_MODE_TILEWAVE


@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 17, 0)), ("skewed", (0, 0, 0)),
                                       ("overlapped", None), ("auto", None), ("wavefront", (0, 0, 0)),
                                       ("wavefront", (0, 6, 0))])
def test_fp32_chains_bit_exact(mode, tile):
    """An OPS_REAL_F32 context: float dats, single-precision arithmetic with
    explicit rounding on both sides, constants rounded to float on load; the
    compiled kernels match the oracle's FP32 execution bit for bit in every
    schedule (reductions of the float values within the usual bound)."""
    for c in (W.cloverleaf2d(n=100, steps=3), W.small2d(n=256, reps=4), edge_chain()):
        ref, ref_hist = oracle.run_chain(c, fp32=True)
        got, hist, st = run_gpu(c, mode, tile, fp32=True)
        assert got[0].dtype == np.float32
        assert_same(c, got, ref, hist, ref_hist, what=f"fp32 {c.name} {mode} {tile}")
        assert st["compiled"] == 1


def test_fp32_refuses_interpreted_and_checked_modes():
    c = W.small2d(n=32, reps=1)
    for kw in (dict(interpret=True), dict(check=True)):
        r = ChainRunner(c, mode="untiled", fp32=True, **kw)
        try:
            with pytest.raises(ops.OpsError):
                r.step()
        finally:
            r.close()


def test_compare_select_on_signed_zeros_and_nan():
    """MIN, MAX and SGT bodies over data full of ties, signed zeros, NaN and
    infinities: the compiled kernels (whose FP64 compares run on the
    integer pipe) and the interpreter give the oracle's bit patterns in
    every mode, FP64 and FP32."""
    import math
    from synth.program import MIN as IMIN, MAX as IMAX, SGT as ISGT
    n = 40
    shp = (1, n + 2, n + 2)
    special = np.array([0.0, -0.0, 1.0, -1.0, math.nan, math.inf, -math.inf, 1.0, 5e-324, -5e-324])
    rnd = np.random.default_rng(21)
    dats = [DatSpec(f"s{k}", special[rnd.integers(0, len(special), shp)]) for k in range(3)]
    dats.append(DatSpec("o", np.zeros(shp)))
    st = [[(0, 0, 0)], [(0, 0, 0), (1, 0, 0)]]
    loops = []
    for k, op in enumerate((IMIN, IMAX)):
        code, K = BodyBuilder().ld(0, 0, 0).ld(1, 1, 1).emit(op, 2, 0, 1).st(2, 2).build()
        loops.append(Loop(f"mm{k}", ((0, n), (0, n)), [Arg(DAT, k, 0, READ), Arg(DAT, 2, 1, READ),
                                                       Arg(DAT, 3, 0, WRITE)], code, K))
    code, K = BodyBuilder().ld(0, 0, 0).ld(1, 1, 0).ld(2, 2, 0).ld(3, 3, 0).emit(ISGT, 4, 0, 1, 2, 3).st(3, 4).build()
    loops.append(Loop("sgt", ((0, n), (0, n)), [Arg(DAT, 0, 0, READ), Arg(DAT, 1, 0, READ), Arg(DAT, 2, 0, READ),
                                                Arg(DAT, 3, 0, RW)], code, K))
    c = Chain("special", 2, (n, n, 1), (1, 1, 0), (1, 1, 0), dats, st, [], loops, steps=2)
    for fp32 in (False, True):
        ref, _ = oracle.run_chain(c, fp32=fp32)
        ut = np.uint32 if fp32 else np.uint64
        for mode, tile, interp in (("untiled", None, False), ("untiled", None, True), ("tilewave", (16, 16, 0), False),
                                   ("wavefront", (0, 8, 0), False), ("skewed", (0, 8, 0), False)):
            if fp32 and interp:
                continue
            got, _, _ = run_gpu(c, mode, tile, interpret=interp, fp32=fp32)
            for k, (a, b) in enumerate(zip(got, ref)):
                assert np.array_equal(a.view(ut), b.view(ut)), f"{mode} interpret={interp} fp32={fp32} dat {k}"


@pytest.mark.parametrize("mode,tile", [("untiled", None), ("skewed", (0, 32, 0)), ("skewed", (0, 0, 0)),
                                       ("overlapped", None), ("wavefront", (0, 0, 0)), ("tilewave", (0, 0, 0)),
                                       ("tilewarp", (0, 0, 0)), ("auto", None)])
def test_cloverleaf_shaped_chain_wide_rows(mode, tile):
    """The mode matrix on 160^2, where rows are wider than the compiled
    kernels' 128-point threshold, so every mode runs its full-width units."""
    c = W.cloverleaf2d(n=160, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, mode, tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"160^2 {mode} {tile}")


@pytest.mark.parametrize("fp32,mode,tile", [(False, "wavefront", (0, 0, 0)), (True, "untiled", None),
                                            (True, "skewed", (0, 1024, 0)), (True, "wavefront", (0, 0, 0))])
def test_bench_size_schedules(fp32, mode, tile):
    """The bench's CloverLeaf-shaped step at 3840^2 in the schedules it
    times beside the headline: every point of every dat against the oracle."""
    c = W.cloverleaf2d(n=3840, steps=1)
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, mode, tile, fp32=fp32)
    assert_same(c, got, ref, hist, ref_hist, what=f"3840^2 {mode} {tile} fp32={fp32}")


def test_overlapped_at_1024():
    c = W.cloverleaf2d(n=1024, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "overlapped", None)
    assert_same(c, got, ref, hist, ref_hist, what="1024^2 overlapped")
    assert st["redundant_points"] > 0
