"""Continuous-batching server: correctness, batch independence, admission."""
import time

import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from synth import rng as R
from synth import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()


def problems(sizes, tag):
    return [W.cg_problem(n, 1e-1, 1e1, seed=R.subseed(21, tag, i)) for i, n in enumerate(sizes)]


def max_concurrency(stats):
    ev = []
    for s in stats:
        a = s["submit_ms"] + s["queue_ms"]
        ev += [(a, 1), (s["done_ms"], -1)]
    cur = best = 0
    for _, d in sorted(ev):
        cur += d
        best = max(best, cur)
    return best


def test_served_results_equal_solo_solves():
    """Every request solved in the served mix is bit-identical to the same
    request solved alone, and meets the tolerance (FP64 residual recomputed
    by the oracle)."""
    sizes = [64, 192, 128, 320, 64, 256, 512, 100]
    probs = problems(sizes, "mix")
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=2 << 30)
    try:
        ids = [ops.ops_serve_submit(srv, k, b) for k, b in probs]
        results = [ops.ops_serve_poll(srv, i, n) for i, n in zip(ids, sizes)]
    finally:
        ops.ops_serve_close(srv)
    ctx = ops.ops_init()
    try:
        for (k, b), (x, st) in zip(probs, results):
            assert st["converged"] == 1
            assert oracle.relres(k, b, x) <= TOL
            xa, sta = ops.ops_cg_solve(ctx, k, b, TOL, ops.OPS_PREC_MIXED)
            assert np.array_equal(x, xa)
            assert st["iterations"] == sta["iterations"] and st["outer"] == sta["outer"]
    finally:
        ops.ops_finalize(ctx)


def test_requests_join_a_running_batch():
    """Requests submitted while a large solve runs are admitted at once and
    run alongside it (continuous batching, not a queue behind it)."""
    big, small = problems([1024], "big")[0], problems([64, 96], "small")
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=2 << 30)
    try:
        ib = ops.ops_serve_submit(srv, *big)
        time.sleep(0.002)
        isx = [ops.ops_serve_submit(srv, k, b) for k, b in small]
        rs = [ops.ops_serve_poll(srv, i, k.shape[0]) for i, (k, b) in zip(isx, small)]
        rb = ops.ops_serve_poll(srv, ib, 1024)
    finally:
        ops.ops_serve_close(srv)
    big_admit = rb[1]["submit_ms"] + rb[1]["queue_ms"]
    for (x, st), (k, b) in zip(rs, small):
        admit = st["submit_ms"] + st["queue_ms"]
        assert st["queue_ms"] < 50.0
        assert big_admit <= admit < rb[1]["done_ms"]
        assert oracle.relres(k, b, x) <= TOL
    assert oracle.relres(*big, rb[0]) <= TOL


def test_admission_by_footprint():
    """With a pool that holds two 256^2 problems, at most two run at once and
    all complete."""
    from paper_1704_00693_gb300 import _build  # noqa: F401
    sizes = [256] * 6
    probs = problems(sizes, "budget")
    one = 92 * 256 * 256 + 16 * 4096
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=2 * one + one // 2)
    try:
        ids = [ops.ops_serve_submit(srv, k, b) for k, b in probs]
        res = [ops.ops_serve_poll(srv, i, 256) for i in ids]
    finally:
        ops.ops_serve_close(srv)
    stats = [s for _, s in res]
    assert max_concurrency(stats) <= 2
    for (k, b), (x, st) in zip(probs, res):
        assert oracle.relres(k, b, x) <= TOL


def test_oversized_request_is_refused():
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=1 << 20)
    try:
        k, b = problems([256], "big2")[0]
        with pytest.raises(ops.OpsError) as e:
            ops.ops_serve_submit(srv, k, b)
        assert e.value.code == ops.OPS_ERR_NOMEM
    finally:
        ops.ops_serve_close(srv)


def test_per_request_tolerance_and_precision():
    """Requests carry their own tolerance and precision: an FP64 request and
    a mixed one at a tighter tolerance share the batch, each meets its own
    tolerance and equals the same request solved alone."""
    probs = problems([128, 192, 96], "perreq")
    want = [(1e-6, ops.OPS_PREC_FP64), (1e-10, ops.OPS_PREC_MIXED), (0.0, -1)]
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=1 << 30)
    try:
        ids = [ops.ops_serve_submit(srv, k, b, tol, prec) for (k, b), (tol, prec) in zip(probs, want)]
        res = [ops.ops_serve_poll(srv, i, k.shape[0]) for i, (k, b) in zip(ids, probs)]
    finally:
        ops.ops_serve_close(srv)
    ctx = ops.ops_init()
    try:
        for (k, b), (tol, prec), (x, st) in zip(probs, want, res):
            t, p = (tol, prec) if tol > 0 else (TOL, ops.OPS_PREC_MIXED)
            assert st["converged"] == 1 and oracle.relres(k, b, x) <= t
            xa, sta = ops.ops_cg_solve(ctx, k, b, t, p)
            assert np.array_equal(x, xa)
    finally:
        ops.ops_finalize(ctx)


def test_many_requests_reuse_fixed_tables():
    """A stream of 40 small requests of mixed sizes through a server whose
    batch can hold 8: every result meets the tolerance (admission keeps the
    fixed tables within their capacity while solves come and go)."""
    sizes = [64 + 32 * (i % 9) for i in range(40)]
    probs = problems(sizes, "stream")
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=1 << 30, max_batch=8)
    try:
        ids = [ops.ops_serve_submit(srv, k, b) for k, b in probs]
        res = [ops.ops_serve_poll(srv, i, n) for i, n in zip(ids, sizes)]
    finally:
        ops.ops_serve_close(srv)
    assert max_concurrency([s for _, s in res]) <= 8
    for (k, b), (x, st) in zip(probs, res):
        assert st["converged"] == 1 and oracle.relres(k, b, x) <= TOL



def test_worker_counters():
    """ops_serve_stats accounts for every request and for the worker's time."""
    sizes = [64, 96, 128, 160]
    probs = problems(sizes, "counters")
    srv = ops.ops_serve_open(TOL, ops.OPS_PREC_MIXED, hbm_budget=1 << 30)
    try:
        ids = [ops.ops_serve_submit(srv, k, b) for k, b in probs]
        res = [ops.ops_serve_poll(srv, i, n) for i, n in zip(ids, sizes)]
        c = ops.ops_serve_stats(srv)
    finally:
        ops.ops_serve_close(srv)
    assert c["admitted"] == len(sizes) and c["completed"] == len(sizes)
    assert c["rounds"] >= 1 and c["run_ms"] > 0.0
    assert all(c[k] >= 0.0 for k in ("upload_ms", "fetch_ms", "idle_ms"))
    for (k, b), (x, st) in zip(probs, res):
        assert oracle.relres(k, b, x) <= TOL
