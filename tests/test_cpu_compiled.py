"""The compiled CPU execution (oracle.cpu_compiled, the paper's CPU scheme
timed as context beside the oracle) against the oracle: dats bit for bit,
untiled and tiled, reductions within rounding."""
import numpy as np
import pytest

import oracle
from oracle import cpu_compiled
from synth import workloads as W

from test_gpu_chain import edge_chain


def _same(c, got, hist, ref, ref_hist):
    for k, (a, b) in enumerate(zip(got, ref)):
        assert np.array_equal(a, b), f"{c.name}: dat {k} differs"
    for h1, h2 in zip(hist, ref_hist):
        for v1, v2, op in zip(h1, h2, c.reductions):
            if op == 0:
                assert abs(v1 - v2) <= 1e-12 * max(1.0, abs(v2))
            else:
                assert v1 == v2


@pytest.mark.parametrize("name,tile", [("cloverleaf2d", (52, 7)), ("small2d", (40, 5)), ("opensbli3d", (14, 14, 3)),
                                       ("ppcg2d", (44, 6)), ("edge", (11, 5)), ("cloverleaf3d", (16, 16, 4))])
def test_compiled_cpu_matches_oracle(name, tile):
    c = {"cloverleaf2d": lambda: W.cloverleaf2d(n=48, steps=2), "small2d": lambda: W.small2d(n=36, reps=2),
         "opensbli3d": lambda: W.opensbli3d(n=10, steps=1), "ppcg2d": lambda: W.ppcg2d(n=40, inner=4),
         "edge": edge_chain, "cloverleaf3d": lambda: W.cloverleaf3d(n=12, steps=1)}[name]()
    ref, ref_hist = oracle.run_chain(c)
    for t in (None, tile):
        got, hist = cpu_compiled.run_chain(c, t)
        _same(c, got, hist, ref, ref_hist)


def test_compiled_cpu_splits_at_reduction_consumers():
    """A loop that reads a reduction through a scalar starts a new schedule,
    so it sees the final value, as in program order."""
    c = edge_chain()
    cc = cpu_compiled.CompiledChain(c)
    segs = cc._segments(c.loops)
    names = [c.loops[s0].name for s0, _ in segs]
    assert names == ["empty", "use_scalar"]
