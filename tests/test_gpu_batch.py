"""GPU parity of batched chains (ops_execute_batch): several grids' chains in
one tile-wavefront launch per segment, through the C ABI.

Each instance's dats must equal the oracle's untiled program-order result
for that instance bit for bit, sums within 1e-12 relative, min and max
exactly; and each instance must end exactly as it does when its context
runs the same chain alone.  The instances differ in their field values,
hence in their reductions and in the time-step constants derived from
them.
"""
import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from paper_1704_00693_gb300.chain import ChainRunner, run_batch
from synth import workloads as W

from test_gpu_chain import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()


def batched(chains, mode, tile=None, fp32=False, steps=None, **kw):
    runners = [ChainRunner(c, mode=mode, tile=tile, fp32=fp32, **kw) for c in chains]
    try:
        hists = run_batch(runners, steps)
        dats = [r.fetch() for r in runners]
        stats = [r.stats() for r in runners]
    finally:
        for r in runners:
            r.close()
    return dats, hists, stats


def check_batch(chains, mode, tile=None, fp32=False, alone=True, steps=None, **kw):
    dats, hists, stats = batched(chains, mode, tile, fp32=fp32, steps=steps, **kw)
    for k, c in enumerate(chains):
        ref, ref_hist = oracle.run_chain(c, steps=steps, fp32=fp32)
        assert_same(c, dats[k], ref, hists[k], ref_hist, what=f"instance {k} {mode} {tile} fp32={fp32}")
    if alone:
        # the same instances, each on its own context: identical dats and reductions
        for k in (0, len(chains) - 1):
            r = ChainRunner(chains[k], mode=mode, tile=tile, fp32=fp32, **kw)
            try:
                h = r.run(steps)
                d = r.fetch()
            finally:
                r.close()
            for a, b in zip(d, dats[k]):
                assert np.array_equal(a, b), f"instance {k}: alone and in the batch differ"
            assert h == hists[k], f"instance {k}: reductions alone {h} in the batch {hists[k]}"
    return stats


@pytest.mark.parametrize("tile", [(0, 0, 0), (32, 32, 0), (1 << 20, 1 << 20, 0), (40, 24, 0)])
def test_small2d_instances(tile):
    """Six 128^2 grids of the 16-loop small chain: automatic tiles, small
    tiles (many per instance), the whole grid as one tile, ragged tiles."""
    chains = W.instances(W.small2d(n=128, reps=2), 6)
    stats = check_batch(chains, "tilewave", tile)
    for st in stats:
        assert st["mode"] == ops.OPS_MODE_TILEWAVE and st["batched"] == 6
    assert stats[0]["kernel_launches"] == stats[0]["segments"]


@pytest.mark.parametrize("fp32", [False, True])
def test_cloverleaf_instances(fp32):
    """Four 96^2 CloverLeaf-shaped grids, two steps: segments cut at the
    time-step reduction, per-instance sums and minima, per-instance
    constants (each grid's own time step)."""
    chains = W.instances(W.cloverleaf2d(n=96, steps=2), 4)
    stats = check_batch(chains, "tilewave", (0, 0, 0), fp32=fp32)
    assert all(st["batched"] == 4 for st in stats)


def test_opensbli3d_instances():
    chains = W.instances(W.opensbli3d(n=16, steps=1), 3)
    check_batch(chains, "tilewave", (0, 0, 0))


def test_one_instance_and_many_instances():
    """A batch of one is the tile wavefront alone; 40 instances of a
    64^2 grid run more tickets than CTAs resident."""
    check_batch(W.instances(W.small2d(n=64, reps=1), 1), "tilewave", (16, 16, 0))
    check_batch(W.instances(W.small2d(n=64, reps=1), 40), "tilewave", (16, 16, 0), alone=False)


@pytest.mark.parametrize("fp32", [False, True])
def test_untiled_batch_one_launch_per_loop(fp32):
    """Untiled batches launch each loop once for all instances (a CTA row
    per instance) and fold every instance's reductions in one launch."""
    chains = W.instances(W.cloverleaf2d(n=64, steps=2), 5)
    stats = check_batch(chains, "untiled", fp32=fp32)
    assert all(st["batched"] == 5 and st["mode"] == ops.OPS_MODE_UNTILED for st in stats)
    assert stats[0]["kernel_launches"] == len(chains[0].loops)


def test_other_modes_run_each_context():
    chains = W.instances(W.cloverleaf2d(n=64, steps=2), 3)
    stats = check_batch(chains, "skewed", (0, 32, 0))
    assert all(st["batched"] == 0 and st["mode"] == ops.OPS_MODE_SKEWED for st in stats)


def test_autotuned_batch():
    """Under OPS_MODE_AUTO the batch autotuner times its candidates over the
    first flushes and keeps the fastest; every flush is exact."""
    chains = W.instances(W.small2d(n=128, reps=2), 5)
    stats = check_batch(chains, "auto", steps=12, alone=False)
    assert stats[0]["tuning"] == 0


def test_mismatched_batches_are_rejected_and_keep_their_queues():
    a = ChainRunner(W.small2d(n=64, reps=1), mode="tilewave")
    b = ChainRunner(W.small2d(n=72, reps=1), mode="tilewave")
    try:
        a.enqueue_step()
        b.enqueue_step()
        with pytest.raises(ops.OpsError) as e:
            ops.ops_execute_batch([a.ctx, b.ctx])
        assert e.value.code == ops.OPS_ERR_INVALID_ARG
        with pytest.raises(ops.OpsError) as e:
            ops.ops_execute_batch([a.ctx, a.ctx])
        assert e.value.code == ops.OPS_ERR_INVALID_ARG
        # nothing ran and the queues are intact: each context still runs its chain
        ops.ops_execute(a.ctx)
        ops.ops_execute(b.ctx)
        ops.ops_sync(a.ctx)
        ops.ops_sync(b.ctx)
        for r in (a, b):
            ref, _ = oracle.run_chain(r.chain, steps=1)
            assert_same(r.chain, r.fetch(), ref, what="after a rejected batch")
    finally:
        a.close()
        b.close()


def test_batch_timeout_reports_on_the_first_context():
    """Tile 0 of instance 0 never reports its progress: the CTAs waiting on
    it give up after the limit, every CTA leaves, ops_sync of the first
    context returns OPS_ERR_TIMEOUT; new contexts then batch normally."""
    chains = W.instances(W.small2d(n=64, reps=1), 3)
    runners = [ChainRunner(c, mode="tilewave", tile=(16, 16, 0), timeout_ms=200,
                           skip_barrier_block=0 if k == 0 else -1) for k, c in enumerate(chains)]
    try:
        for r in runners:
            r.enqueue_step()
        ops.ops_execute_batch([r.ctx for r in runners])
        with pytest.raises(ops.OpsError) as e:
            ops.ops_sync(runners[0].ctx)
        assert e.value.code == ops.OPS_ERR_TIMEOUT
    finally:
        for r in runners:
            r.close()
    check_batch(chains, "tilewave", (16, 16, 0), alone=False)


def test_bench_batch_workload():
    """The bench's batch: 64 CloverLeaf-shaped 256^2 grids, one step each,
    automatic tiles; every instance against the oracle."""
    chains = W.instances(W.cloverleaf2d(n=256, steps=1), 64)
    stats = check_batch(chains, "tilewave", (0, 0, 0), alone=False)
    assert all(st["batched"] == 64 for st in stats)
