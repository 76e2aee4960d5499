"""GPU parity of the heat-conduction solvers against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
import paper_1704_00693_gb300 as ops
from synth import workloads as W
from synth import rng as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1704_00693_gb300 import _build
    _build.build()
    oracle.build()
    c = ops.ops_init()
    yield c
    ops.ops_finalize(c)


@pytest.mark.parametrize("n", [1, 7, 64, 301])
def test_operator_bit_exact(ctx, n):
    """One application of A in FP64 and in FP32 matches the oracle bit for
    bit (same faces, same fma order) on grids that span several work units
    and a ragged last unit."""
    kappa, _ = W.cg_problem(n, 1e-2, 1e2)
    u = R.uniform(R.subseed(3, "u", n), (n, n), -1.0, 1.0)
    w64 = ops.ops_heat_apply(ctx, kappa, u, ops.OPS_PREC_FP64)
    assert np.array_equal(w64, oracle.matvec(kappa, u))
    w32 = ops.ops_heat_apply(ctx, kappa, u, ops.OPS_PREC_MIXED)
    assert np.array_equal(w32, oracle.matvec32(kappa, u))


def test_cg64_eigenmode_one_iteration(ctx):
    n, kap, p, q = 40, 0.7, 3, 2
    i = np.arange(n)
    b = np.outer(np.sin(np.pi * q * (i + 1) / (n + 1)), np.sin(np.pi * p * (i + 1) / (n + 1)))
    mu = 1 + kap * (4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 + 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2)
    x, st = ops.ops_cg_solve(ctx, np.full((n, n), kap), b, 1e-10, ops.OPS_PREC_FP64)
    assert st["iterations"] == 1 and st["converged"] == 1
    assert np.abs(x - b / mu).max() < 1e-14


@pytest.mark.parametrize("n", [33, 128])
def test_cg64_matches_oracle(ctx, n):
    kappa, b = W.cg_problem(n, 1e-2, 1e2)
    x_ref, it_ref, _ = oracle.cg64(kappa, b, tol=1e-10)
    x, st = ops.ops_cg_solve(ctx, kappa, b, 1e-10, ops.OPS_PREC_FP64)
    assert st["converged"] == 1
    assert abs(st["iterations"] - it_ref) <= max(2, it_ref // 50)
    assert oracle.relres(kappa, b, x) <= 1.5e-10
    assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


@pytest.mark.parametrize("n", [33, 200])
def test_mixed_refinement_matches_oracle(ctx, n):
    kappa, b = W.cg_problem(n, 1e-2, 1e2)
    x64, _, _ = oracle.cg64(kappa, b, tol=1e-12)
    xr, it, rel, outer = oracle.cg_refine(kappa, b, tol=1e-10, inner_tol=1e-4)
    x, st = ops.ops_cg_solve(ctx, kappa, b, 1e-10, ops.OPS_PREC_MIXED)
    assert st["converged"] == 1 and st["outer"] >= 2
    true_rel = oracle.relres(kappa, b, x)
    assert true_rel <= 1e-10
    assert abs(true_rel - st["relres"]) <= 1e-3 * true_rel + 1e-16
    assert abs(st["outer"] - outer) <= 1
    # the same refinement scheme: a wrong restart (say, a stale beta on the
    # first inner direction) shows up as extra inner iterations
    assert abs(st["iterations"] - it) <= max(4, 0.1 * it), (st["iterations"], it)
    assert np.abs(x - x64).max() <= 1e-7 * np.abs(x64).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_results_independent_of_batch(ctx, prec):
    """Each problem solved inside a batch of mixed sizes gives bit-identical
    x and iteration counts to the same problem solved alone."""
    sizes = [17, 64, 130, 300, 64]
    probs = [W.cg_problem(n, 1e-1, 1e1, seed=R.subseed(11, "b", i)) for i, n in enumerate(sizes)]
    xs, sts = ops.ops_cg_solve_batch(ctx, [p[0] for p in probs], [p[1] for p in probs], 1e-8, prec)
    for (k, b), x, st in zip(probs, xs, sts):
        xa, sta = ops.ops_cg_solve(ctx, k, b, 1e-8, prec)
        assert np.array_equal(x, xa)
        assert st == sta
        assert oracle.relres(k, b, x) <= 1e-8 * (1.0 if prec == 1 else 1.5)


def test_iteration_cap_reports_not_converged(ctx):
    kappa, b = W.cg_problem(64, 1e-2, 1e2)
    x, st = ops.ops_cg_solve(ctx, kappa, b, 1e-12, ops.OPS_PREC_FP64, maxit=5)
    assert st["converged"] == 0 and st["iterations"] == 5


def test_full_size_mixed_solve():
    """The 4000^2 TeaLeaf-shaped problem (conductivity log-uniform in
    [1e-2, 1e2]) with FP32 sweeps and FP64 refinement to 1e-10; the FP64
    residual is recomputed by the oracle."""
    from paper_1704_00693_gb300 import _build
    _build.build()
    c = ops.ops_init()
    try:
        kappa, b = W.cg_problem(4000, 1e-2, 1e2)
        x, st = ops.ops_cg_solve(c, kappa, b, 1e-10, ops.OPS_PREC_MIXED)
    finally:
        ops.ops_finalize(c)
    assert st["converged"] == 1
    assert oracle.relres(kappa, b, x) <= 1e-10


@pytest.mark.parametrize("n", [1, 33, 128])
def test_chain_cg_matches_oracle(n):
    """CG written as a loop chain (setup loops for the faces and diagonal,
    three loops per iteration, host-read reductions) converges like the
    oracle's FP64 CG, and its operator is the engine's bit for bit (one
    iteration from x = 0 gives w = A b)."""
    from cg_loopchain import ChainCG
    kappa, b = W.cg_problem(n, 1e-2, 1e2)
    x_ref, it_ref, _ = oracle.cg64(kappa, b, tol=1e-10)
    for mode in ("untiled", "skewed"):
        cg = ChainCG(n, mode=mode)
        try:
            x, it, rel = cg.solve(kappa, b, 1e-10)
            assert rel <= 1e-10
            assert abs(it - it_ref) <= max(2, it_ref // 50)
            assert oracle.relres(kappa, b, x) <= 1.5e-10
            assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
            cg.solve(kappa, b, 1e-10, maxit=1)
            w = ops.ops_dat_fetch(cg.ctx, cg.d["w"]).reshape(n + 2, n + 2)[1:n + 1, 1:n + 1]
            assert np.array_equal(w, oracle.matvec(kappa, b))
        finally:
            cg.close()
