"""GPU parity of the tile wavefront (OPS_MODE_TILEWAVE) against the FP64 /
FP32 oracle, through the C ABI.

Every dat must equal the oracle's untiled program-order result bit for bit;
reduction sums within 1e-12 relative of the exactly rounded value, min and
max exactly.  The cases span ragged tiles, tiles the library must grow to
cover the chain's skew, 1D/2D/3D chains, the edge-case chain (empty and
one-point ranges, INC/RW, SCALAR splits, all reductions), segment cuts, the device-wait timeout, and the bench workloads at full size.
"""
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
    for tile in ((4,), (3,), (2,), (8,)):
        got, _, st = run_gpu(c, "tilewave", tile)
        assert_same(c, got, ref, what=f"tilewave {tile}")
        assert st["mode"] == ops.OPS_MODE_TILEWAVE


@pytest.mark.parametrize("tile", [(0, 0, 0), (32, 16, 0), (100, 33, 0), (256, 256, 0)])
def test_small2d_chain_bit_exact(tile):
    c = W.small2d(n=256, reps=10)
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "tilewave", tile)
    assert_same(c, got, ref, what=f"tilewave {tile}")
    assert st["mode"] == ops.OPS_MODE_TILEWAVE and st["kernel_launches"] == st["segments"]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("n,tile", [(100, (0, 0, 0)), (100, (32, 16, 0)), (100, (37, 23, 0)),
                                    (300, (0, 0, 0)), (300, (128, 32, 0)), (300, (64, 40, 0))])
def test_cloverleaf_shaped_chain(n, tile, fp32):
    """83-loop CloverLeaf-shaped steps (node ranges, thin halo strips, RW
    updates, a sum and a min reduction per step, the min feeding the next
    step's constants); 300^2 rows are wider than the 128-point x tiles."""
    c = W.cloverleaf2d(n=n, steps=3)
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, "tilewave", tile, fp32=fp32)
    assert_same(c, got, ref, hist, ref_hist, what=f"tilewave {n} {tile} fp32={fp32}")
    assert st["mode"] == ops.OPS_MODE_TILEWAVE
    for d in range(2):
        if tile[d]:
            assert st["tile"][d] >= tile[d]  # grown where the skew reaches across a tile


@pytest.mark.parametrize("tile", [(0, 0, 0), (48, 32, 32), (20, 20, 20)])
def test_cloverleaf3d_shaped_chain(tile):
    c = W.cloverleaf3d(n=40, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "tilewave", tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"3d hydro tilewave {tile}")


@pytest.mark.parametrize("tile", [(0, 0, 0), (64, 24, 0), (101, 101, 0)])
def test_ppcg_shaped_chain(tile):
    c = W.ppcg2d(n=100, inner=10, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "tilewave", tile)
    assert_same(c, got, ref, hist, ref_hist, what=f"ppcg tilewave {tile}")


def test_opensbli_shaped_3d():
    c = W.opensbli3d(n=24, steps=2)
    ref, _ = oracle.run_chain(c)
    for tile in ((0, 0, 0), (28, 14, 14), (16, 16, 8)):
        got, _, st = run_gpu(c, "tilewave", tile)
        assert_same(c, got, ref, what=f"3d tilewave {tile}")


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("tile", [(0, 0, 0), (11, 9, 0)])
def test_edge_cases(tile, fp32):
    c = edge_chain()
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, "tilewave", tile, fp32=fp32)
    assert_same(c, got, ref, hist, ref_hist, what=f"edge tilewave {tile}")


def test_segments_and_single_loop_segments():
    """A flush cut into segments of at most 10 loops runs one tile-wavefront
    kernel per segment; one-loop segments run untiled."""
    c = W.cloverleaf2d(n=90, steps=2)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "tilewave", (0, 0, 0), segment=10)
    assert_same(c, got, ref, hist, ref_hist, what="tilewave segments")
    got, hist, st = run_gpu(c, "tilewave", (0, 0, 0), segment=1)
    assert_same(c, got, ref, hist, ref_hist, what="tilewave one-loop segments")


def test_jacobi_closed_form_and_stats():
    """Jacobi steps reproduce the Dirichlet eigenmode's closed-form decay;
    the plan is cached and one kernel runs per flush."""
    n, K, nu = 62, 30, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=2, q=1)
    ref, _ = oracle.run_chain(c)
    r = ChainRunner(c, mode="tilewave", tile=(32, 32, 0))
    try:
        r.run()
        got = r.fetch()
        st = r.stats()
        r.run()
        st2 = r.stats()
    finally:
        r.close()
    assert_same(c, got, ref, what="jacobi tilewave")
    assert st["mode"] == ops.OPS_MODE_TILEWAVE and st["kernel_launches"] == st["segments"] >= 1
    assert st2["plan_cache_hits"] >= 1 and st2["plan_ms"] == 0.0
    lam = -4 * math.sin(math.pi * 2 / (2 * (n + 1))) ** 2 - 4 * math.sin(math.pi * 1 / (2 * (n + 1))) ** 2
    want = c.dats[0].init * (1 + nu * lam) ** K
    assert np.abs(got[0] - want).max() <= 1e-13 * np.abs(want).max()


def test_timeout_reports_and_context_recovers():
    """Tile 0 never reports its progress: the tiles waiting on it give up
    after the limit, every CTA leaves, the host sees OPS_ERR_TIMEOUT; a new
    context on the same device then runs the same chain normally."""
    c = W.small2d(n=64, reps=1)
    r = ChainRunner(c, mode="tilewave", tile=(16, 16, 0), timeout_ms=200, skip_barrier_block=0)
    try:
        r.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(r.ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
    finally:
        r.close()
    ref, _ = oracle.run_chain(c)
    got, _, st = run_gpu(c, "tilewave", (16, 16, 0))
    assert st["mode"] == ops.OPS_MODE_TILEWAVE
    assert_same(c, got, ref, what="after timeout")


@pytest.mark.parametrize("fp32", [True, False])
def test_full_size_cloverleaf_one_step(fp32):
    """The bench workload: one CloverLeaf-shaped step at 3840^2 with the
    automatic tiles, every point of every dat against the oracle."""
    c = W.cloverleaf2d(n=3840, steps=1)
    ref, ref_hist = oracle.run_chain(c, fp32=fp32)
    got, hist, st = run_gpu(c, "tilewave", (0, 0, 0), fp32=fp32)
    assert st["mode"] == ops.OPS_MODE_TILEWAVE
    assert_same(c, got, ref, hist, ref_hist, what=f"3840^2 tilewave fp32={fp32}")


def test_full_size_ppcg():
    """The PPCG-shaped chain at 4000^2 (FP64), every point against the oracle."""
    c = W.ppcg2d(n=4000, inner=10, steps=1)
    ref, ref_hist = oracle.run_chain(c)
    got, hist, st = run_gpu(c, "tilewave", (0, 0, 0))
    assert st["mode"] == ops.OPS_MODE_TILEWAVE
    assert_same(c, got, ref, hist, ref_hist, what="ppcg 4000^2 tilewave")
