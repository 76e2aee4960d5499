"""GPU parity of the tile-per-warp form of the tile wavefront
(OPS_MODE_TILEWARP) against the FP64 / FP32 oracle, through the C ABI.

The plan is the tile wavefront's; only the execution differs (a warp per
tile, warp-level ordering between a tile's loops).  Every dat must equal the
oracle's untiled program-order result bit for bit, sums within 1e-12
relative, min and max exactly."""
import math

import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from paper_1704_00693_gb300.chain import ChainRunner
from synth import workloads as W

from test_gpu_chain import assert_same, edge_chain, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()


def test_worked_example_1d():
    c = W.worked_example_1d()
    ref, _ = oracle.run_chain(c)
    for tile in ((4,), (3,), (8,)):
        got, _, st = run_gpu(c, "tilewarp", tile)
        assert_same(c, got, ref, what=f"tilewarp {tile}")
        assert st["mode"] == ops.OPS_MODE_TILEWARP


@pytest.mark.parametrize("tile", [(0, 0, 0), (32, 16, 0), (100, 33, 0)])
def test_small2d_chain_bit_exact(tile):
    c = W.small2d(n=256, reps=10)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "tilewarp", tile)
    assert_same(c, got, ref, what=f"tilewarp {tile}")
    assert st["mode"] == ops.OPS_MODE_TILEWARP and st["kernel_launches"] == st["segments"]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("n,tile", [(100, (0, 0, 0)), (100, (37, 23, 0)), (300, (0, 0, 0)), (300, (64, 40, 0))])
def test_cloverleaf_shaped_chain(n, tile, fp32):
    c = W.cloverleaf2d(n=n, steps=3)
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, "tilewarp", tile, fp32=fp32)
    assert_same(c, got, ref, hist, ref_hist, what=f"tilewarp {n} {tile} fp32={fp32}")
    assert st["mode"] == ops.OPS_MODE_TILEWARP


@pytest.mark.parametrize("tile", [(0, 0, 0), (20, 20, 20)])
def test_cloverleaf3d_shaped_chain(tile):
    c = W.cloverleaf3d(n=40, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "tilewarp", tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"3d hydro tilewarp {tile}")


def test_ppcg_and_opensbli_shaped_chains():
    for c in (W.ppcg2d(n=100, inner=10, steps=2), W.opensbli3d(n=24, steps=2)):
        ref, ref_hist = oracle.run_chain(c)
        got, hist, st = run_gpu(c, "tilewarp", (0, 0, 0))
        assert_same(c, got, ref, hist, ref_hist, what=f"tilewarp {c.name}")


@pytest.mark.parametrize("fp32", [False, True])
def test_edge_cases(fp32):
    c = edge_chain()
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    for tile in ((0, 0, 0), (11, 9, 0)):
        got, hist, st = run_gpu(c, "tilewarp", tile, fp32=fp32)
        assert_same(c, got, ref, hist, ref_hist, what=f"edge tilewarp {tile} fp32={fp32}")


def test_jacobi_closed_form():
    n, K, nu = 62, 30, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=2, q=1)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "tilewarp", (16, 16, 0))
    assert_same(c, got, ref, what="jacobi tilewarp")
    lam = -4 * math.sin(math.pi * 2 / (2 * (n + 1))) ** 2 - 4 * math.sin(math.pi * 1 / (2 * (n + 1))) ** 2
    want = c.dats[0].init * (1 + nu * lam) ** K
    assert np.abs(got[0] - want).max() <= 1e-13 * np.abs(want).max()


def test_timeout_reports_and_context_recovers():
    """Tile 0 never reports its progress: the warps waiting on it give up
    after the limit, every warp leaves, the host sees OPS_ERR_TIMEOUT."""
    c = W.small2d(n=64, reps=1)
    r = ChainRunner(c, mode="tilewarp", tile=(16, 16, 0), timeout_ms=200, skip_barrier_block=0)
    try:
        r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(r.ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
    finally:
        r.close()
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "tilewarp", (16, 16, 0))
    assert st["mode"] == ops.OPS_MODE_TILEWARP
    assert_same(c, got, ref, what="after timeout")


def test_full_size_jacobi_fp32():
    """The bench's heat-equation flush at full size: 8192^2 FP32, 10
    iterations, automatic tiles, every point against the oracle."""
    c = W.jacobi2d(8192, 10, init="rand")
    ref, _ = oracle.run_chain(c, fp32=True)
    got, _, st = run_gpu(c, "tilewarp", (0, 0, 0), fp32=True)
    assert st["mode"] == ops.OPS_MODE_TILEWARP
    assert_same(c, got, ref, what="8192^2 jacobi tilewarp")


def test_full_size_cloverleaf_fp32():
    c = W.cloverleaf2d(n=3840, steps=1)
    ref, ref_hist = oracle.run_chain(c, fp32=True)
    got, hist, st = run_gpu(c, "tilewarp", (0, 0, 0), fp32=True)
    assert st["mode"] == ops.OPS_MODE_TILEWARP
    assert_same(c, got, ref, hist, ref_hist, what="3840^2 tilewarp fp32")
