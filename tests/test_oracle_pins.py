"""Pins for the CPU oracle: checks against facts fixed by the paper and by the
mathematics, never against the oracle itself or the CUDA library."""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import plan as oplan
from synth import workloads as W
from synth import rng as R

from bruteforce import check_overlapped, check_phase_order, check_skewed, random_chain, random_topological

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fma_exact(a, b, c):
    """a*b + c rounded once (exact rational arithmetic, correctly rounded)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


# ---------------------------------------------------------------- exact sums
def test_fsum_matches_library_and_exact_rationals():
    rnd = np.random.default_rng(1)
    for trial in range(20):
        n = int(rnd.integers(1, 2000))
        x = rnd.standard_normal(n) * 10.0 ** rnd.integers(-20, 20, size=n)
        assert oracle.fsum(x) == math.fsum(x)
    # heavy cancellation; the exact rational sum rounded once
    for trial in range(50):
        n = int(rnd.integers(2, 40))
        x = rnd.standard_normal(n) * 10.0 ** rnd.integers(-30, 30, size=n)
        x = np.concatenate([x, -x[: n // 2] * (1 + 2.0 ** -52)])
        exact = sum((Fraction(float(v)) for v in x), Fraction(0))
        assert oracle.fsum(x) == float(exact)
    # a tie that naive left-to-right summation rounds the wrong way
    assert oracle.fsum([1.0, 2.0 ** -53, 2.0 ** -106]) == 1.0 + 2.0 ** -52


# ----------------------------------------------------------- interpreter pins
def test_constant_preservation_bit_exact():
    """All dats and halos = 0.75, positive dyadic weights summing to 1: every
    weighted sum is exact and must return 0.75 exactly (any dropped or extra
    term, or a wrong coefficient index, changes the value)."""
    c = W.small2d(n=24, reps=3, constant=0.75)
    dats, _ = oracle.run_chain(c)
    for d in dats:
        assert (d == 0.75).all()


def test_linear_field_reproduction():
    """f = a0 + bx x + by y (dyadic): a symmetric 9-point average returns f,
    the 5-point Laplacian returns 0 and the one-sided 4-point average returns
    f + bx/2 + 5 by/8, all exactly; bx != by catches a transposed offset."""
    a0, bx, by = 0.5, 0.25, -0.375
    n = 20
    c = W.linear2d(n, a0, bx, by)
    dats, _ = oracle.run_chain(c)
    h = 2
    y = np.arange(n)[:, None]
    x = np.arange(n)[None, :]
    f = a0 + bx * x + by * y
    inner = (0, slice(h, h + n), slice(h, h + n))
    assert (dats[1][inner] == f).all()
    assert (dats[2][inner] == 0.0).all()
    assert (dats[3][inner] == f + bx / 2 + 5 * by / 8).all()


@pytest.mark.parametrize("p,q", [(1, 1), (2, 3)])
def test_jacobi_eigenmode_closed_form(p, q):
    """u = sin(pi p (i+1)/(N+1)) sin(pi q (j+1)/(N+1)) is an eigenvector of the
    5-point Dirichlet Laplacian with eigenvalue
    -4 sin^2(pi p / (2(N+1))) - 4 sin^2(pi q / (2(N+1))); K Jacobi steps
    u <- u + nu L u multiply it by (1 + nu lambda)^K."""
    n, K, nu = 31, 40, 0.125
    c = W.jacobi2d(n, K, nu=nu, p=p, q=q)
    init = c.dats[0].init.copy()
    dats, _ = oracle.run_chain(c)
    lam = -4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 - 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2
    g = (1 + nu * lam) ** K
    want = init * g
    err = np.abs(dats[0] - want).max() / np.abs(want).max()
    assert err < 1e-13, err


def test_reductions_sum_min_against_scalar_loops():
    """A loop over U(0,1) data with a SUM and a MIN reduction: the sum must be
    the exactly rounded sum of the per-point values, the min the plain min."""
    from synth.program import Arg, BodyBuilder, Chain, DatSpec, Loop, DAT, REDARG, READ, RSUM, RMIN
    n = 37
    shp = (1, n + 2, n + 2)
    a = R.uniform(R.subseed(7, "a"), shp)
    b = R.uniform(R.subseed(7, "b"), shp)
    st = [[(0, 0, 0)], [(0, 0, 0), (1, 0, 0)]]
    code, K = (BodyBuilder().wsum(0, 0, [0.75, -0.5]).wacc(0, 1, [1.25]).red(2, 0).red(3, 0).build())
    lp = Loop("red", ((0, n), (0, n)), [Arg(DAT, 0, 1, READ), Arg(DAT, 1, 0, READ),
                                        Arg(REDARG, 0), Arg(REDARG, 1)], code, K)
    ch = Chain("red", 2, (n, n, 1), (1, 1, 0), (1, 1, 0), [DatSpec("a", a), DatSpec("b", b)], st,
               [RSUM, RMIN], [lp])
    _, hist = oracle.run_chain(ch)
    vals = []
    for j in range(n):
        for i in range(n):
            t = 0.75 * a[0, j + 1, i + 1]
            t = fma_exact(-0.5, a[0, j + 1, i + 2], t)
            t = fma_exact(1.25, b[0, j + 1, i + 1], t)
            vals.append(t)
    assert hist[0][0] == math.fsum(vals)
    assert hist[0][1] == min(vals)


def test_oracle_rejects_out_of_allocation_access():
    from synth.program import Arg, BodyBuilder, Chain, DatSpec, Loop, DAT, READ, WRITE
    n = 8
    st = [[(0, 0, 0)], [(3, 0, 0)]]
    code, K = BodyBuilder().wsum(0, 0, [1.0]).st(1, 0).build()
    lp = Loop("bad", ((0, n), (0, n)), [Arg(DAT, 0, 1, READ), Arg(DAT, 1, 0, WRITE)], code, K)
    ch = Chain("bad", 2, (n, n, 1), (1, 1, 0), (1, 1, 0),
               [DatSpec("a", np.zeros((1, n + 2, n + 2))), DatSpec("b", np.zeros((1, n + 2, n + 2)))],
               st, [], [lp])
    with pytest.raises(oracle.OracleError):
        oracle.run_chain(ch)


# ------------------------------------------------------------------ plan pins
def test_worked_example_plan_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_1d.json")))
    c = W.worked_example_1d()
    nt, rg, un = oplan.skewed_plan(c.loops, c.stencils, 1, [g["tilesize"]])
    assert nt == [2]
    assert [list(rg[0][t][0]) for t in range(2)] == g["loop1"]
    assert [list(rg[0][t][1]) for t in range(2)] == g["loop2"]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_skewed_plan_bruteforce(ndim):
    rnd = random.Random(1000 + ndim)
    sizes = {1: (24,), 2: (11, 9), 3: (6, 5, 4)}[ndim]
    trials = {1: 150, 2: 60, 3: 15}[ndim]
    for trial in range(trials):
        n = [rnd.randint(max(2, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 6))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        nt, rg, _ = oplan.skewed_plan(loops, st, ndim, ts)
        check_skewed(loops, st, ndim, nt, rg)


def test_skewed_plan_bruteforce_catches_planted_mistake():
    """Dropping the WAR/WAW extension (Algorithm 1, second tile pass) must
    make the brute-force check fail on some random chain."""
    import oracle.plan as P
    orig = P._ext

    def no_negative(stencil, d):
        lo, hi = orig(stencil, d)
        return 0, hi

    rnd = random.Random(7)
    failures = 0
    P._ext = no_negative
    try:
        for trial in range(60):
            loops, st = random_chain(rnd, 1, [20], ndats=3, nloops=4)
            nt, rg, _ = P.skewed_plan(loops, st, 1, [rnd.randint(2, 6)])
            try:
                check_skewed(loops, st, 1, nt, rg)
            except AssertionError:
                failures += 1
    finally:
        P._ext = orig
    assert failures > 0


@pytest.mark.parametrize("ndim", [1, 2])
def test_overlapped_plan_bruteforce(ndim):
    rnd = random.Random(2000 + ndim)
    sizes = {1: (24,), 2: (10, 9)}[ndim]
    for trial in range(25 if ndim == 2 else 80):
        n = [rnd.randint(max(3, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 6))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        tiles = []
        import itertools
        cuts = [list(range(-2, n[d] + 2, ts[d])) for d in range(ndim)]
        for lows in itertools.product(*cuts):
            tiles.append(tuple((lo, min(lo + ts[d], n[d] + 2)) for d, lo in enumerate(lows)))
        check_overlapped(loops, st, ndim, tiles, oplan.overlapped_plan)


def test_ppcg_chain_eigenmode_closed_form():
    """The TeaLeaf-PPCG-shaped chain with constant conductivity k applied to
    the Dirichlet eigenmode v of I + k L (eigenvalue lam = 1 + k (4 sin^2 +
    4 sin^2)) keeps every vector a multiple of v: sd_0 = v / theta, rt = v,
    z = sd, then rt -= lam sd, sd = alpha sd + beta rt, z += sd.  The oracle's
    z must be that scalar recurrence times v, and z.r its sum."""
    n, kap, p, q, inner = 24, 0.7, 3, 2, 8
    c = W.ppcg2d(n=n, inner=inner, kappa_const=kap, r_mode=(p, q))
    ref, hist = oracle.run_chain(c)
    lam = 1 + kap * (4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 + 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2)
    theta, delta = c.meta["theta"], c.meta["delta"]
    sigma = theta / delta
    sd, rt = 1.0 / theta, 1.0
    z = sd
    rho_old = 1.0 / sigma
    for _ in range(inner):
        rt = rt - lam * sd
        rho = 1.0 / (2 * sigma - rho_old)
        alpha, beta = rho * rho_old, 2 * rho / delta
        rho_old = rho
        sd = alpha * sd + beta * rt
        z = z + sd
    v = c.dats[1].init
    zz = ref[5]
    assert np.abs(zz - z * v).max() <= 1e-13 * np.abs(v).max()
    assert abs(hist[0][0] - z * float((v * v).sum())) <= 1e-12 * abs(z * float((v * v).sum()))


@pytest.mark.parametrize("name,tile", [("cloverleaf2d", (64, 9)), ("cloverleaf2d", (17, 64)), ("small2d", (40, 7)),
                                       ("opensbli3d", (12, 5, 4)), ("ppcg2d", (50, 6))])
def test_tiled_execution_equals_program_order(name, tile):
    """Algorithm 1's ranges executed as Algorithm 2 does (tile by tile, loops
    in order within a tile) give the program-order result bit for bit and
    the same exact reductions: the oracle's plan and executor agree with the
    definition of the method on whole workloads, not only on the brute-force
    grids."""
    c = {"cloverleaf2d": lambda: W.cloverleaf2d(n=48, steps=2), "small2d": lambda: W.small2d(n=60, reps=3),
         "opensbli3d": lambda: W.opensbli3d(n=14, steps=1), "ppcg2d": lambda: W.ppcg2d(n=50, inner=4)}[name]()
    ref, ref_hist = oracle.run_chain(c)
    got, hist = oracle.run_chain_tiled(c, tile)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert hist == ref_hist


# ---------------------------------------------------------- wavefront orders
def test_phase_conflicts_worked_example():
    """The conflict relation of the Sec. 4.B worked example, derived by hand
    in the golden file: loop 1 of tile 1 depends on nothing of tile 0."""
    g = json.load(open(os.path.join(GOLDEN, "worked_example_1d_wavefront.json")))
    c = W.worked_example_1d()
    nt, rg, _ = oplan.skewed_plan(c.loops, c.stencils, 1, g["tile"])
    ph = oplan.phases_in_order(c.loops, nt, rg, 1)
    assert [[l, list(b[0])] for l, b in ph] == g["phases"]
    assert oplan.phase_conflicts(c.loops, c.stencils, 1, ph) == g["deps"]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_phase_conflicts_allow_any_topological_order(ndim):
    """Brute force on tiny random chains: every order of a skewed plan's
    phases that respects phase_conflicts gives program-order versions at
    every read and every cell (random orders and the order that runs each
    phase as late as possible)."""
    rnd = random.Random(7000 + ndim)
    sizes = {1: (24,), 2: (10, 9), 3: (6, 5, 5)}[ndim]
    for trial in range({1: 40, 2: 20, 3: 8}[ndim]):
        n = [rnd.randint(max(3, s // 2), s) for s in sizes]
        loops, st = random_chain(rnd, ndim, n, ndats=rnd.randint(3, 5), nloops=rnd.randint(2, 7))
        ts = [rnd.randint(1, n[d] + 2) for d in range(ndim)]
        nt, rg, _ = oplan.skewed_plan(loops, st, ndim, ts)
        ph = oplan.phases_in_order(loops, nt, rg, ndim)
        deps = oplan.phase_conflicts(loops, st, ndim, ph)
        assert all(p < q for q, d in enumerate(deps) for p in d)
        for k in range(3):
            check_phase_order(loops, st, ndim, ph, random_topological(deps, rnd))
        # latest first: always take the highest-numbered ready phase
        users = [[] for _ in ph]
        for q, d in enumerate(deps):
            for p in d:
                users[p].append(q)
        waiting, ready, order = [len(d) for d in deps], [q for q, d in enumerate(deps) if not d], []
        while ready:
            ready.sort()
            q = ready.pop()
            order.append(q)
            for u in users[q]:
                waiting[u] -= 1
                if waiting[u] == 0:
                    ready.append(u)
        check_phase_order(loops, st, ndim, ph, order)


@pytest.mark.parametrize("name,tile", [("cloverleaf2d", (44, 5)), ("small2d", (40, 4)), ("jacobi2d", (26, 3)),
                                       ("opensbli3d", (14, 14, 2))])
def test_wavefront_order_equals_program_order(name, tile):
    """Whole workloads in random conflict-respecting orders of their phases
    give the program-order dats bit for bit and the same exact reductions;
    with every dependency list cut to its first half (a planted mistake) some
    order goes wrong."""
    c = {"cloverleaf2d": lambda: W.cloverleaf2d(n=40, steps=1), "small2d": lambda: W.small2d(n=36, reps=2),
         "jacobi2d": lambda: W.jacobi2d(n=24, iters=4, init="random"),
         "opensbli3d": lambda: W.opensbli3d(n=10, steps=1)}[name]()
    ref, ref_hist = oracle.run_chain(c)
    for seed in range(2):
        got, hist = oracle.run_chain_wavefront(c, tile, seed=seed)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        assert hist == ref_hist
    wrong = 0
    for seed in range(4):
        got, _ = oracle.run_chain_wavefront(c, tile, seed=seed, drop=lambda q, d: d[:len(d) // 2])
        wrong += any(not np.array_equal(a, b) for a, b in zip(got, ref))
    assert wrong > 0


def test_fp32_oracle_pins():
    """The oracle's FP32 execution: constants preserved exactly (dyadic
    weights), linear fields reproduced exactly by symmetric stencils, and
    every result within a few float roundings per loop of the FP64 one."""
    c = W.small2d(n=48, reps=2, constant=0.75)
    got, _ = oracle.run_chain(c, fp32=True)
    assert all(d.dtype == np.float32 and (d == np.float32(0.75)).all() for d in got)
    a0, bx, by = 0.5, 0.25, -0.375
    c = W.linear2d(40, a0, bx, by)
    got32, _ = oracle.run_chain(c, fp32=True)
    got64, _ = oracle.run_chain(c)
    for a, b in zip(got32, got64):
        assert np.array_equal(a.astype(np.float64), b)
    c = W.small2d(n=64, reps=3)
    r32, _ = oracle.run_chain(c, fp32=True)
    r64, _ = oracle.run_chain(c)
    nloops = len(c.loops) * c.steps
    for a, b in zip(r32, r64):
        assert np.abs(a.astype(np.float64) - b).max() <= 20 * nloops * 2.0 ** -24 * max(1.0, np.abs(b).max())
