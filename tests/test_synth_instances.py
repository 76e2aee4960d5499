"""The batch workload generator (synth.workloads.instances): grids that share
every loop, stencil and reduction of a chain and differ only in their field
values, drawn like the original's (zero halos kept zero, constant dats kept)."""
import numpy as np

from synth import workloads as W


def test_instances_share_the_chain_and_redraw_the_fields():
    base = W.cloverleaf2d(n=24, steps=1)
    inst = W.instances(base, 4, seed=7)
    assert len(inst) == 4 and inst[0] is base
    for c in inst[1:]:
        assert c.loops is base.loops and c.stencils is base.stencils and c.reductions is base.reductions
        assert c.size == base.size and c.d_m == base.d_m and c.d_p == base.d_p
        for d0, d in zip(base.dats, c.dats):
            a0, a = d0.init, d.init
            assert a.shape == a0.shape
            assert np.array_equal(a0 == 0.0, a == 0.0)  # zeros where the original has them, only there
            nz = a0 != 0.0
            if nz.any() and a0[nz].min() < a0[nz].max():
                assert a[nz].min() >= a0[nz].min() and a[nz].max() <= a0[nz].max()
                assert not np.array_equal(a, a0)  # a fresh draw
    # distinct instances get distinct fields, and the draw is reproducible
    assert not np.array_equal(inst[1].dats[0].init, inst[2].dats[0].init)
    again = W.instances(base, 4, seed=7)
    for c1, c2 in zip(inst[1:], again[1:]):
        for d1, d2 in zip(c1.dats, c2.dats):
            assert np.array_equal(d1.init, d2.init)


def test_instances_keep_zero_halos_of_the_small_chain():
    base = W.small2d(n=16, reps=1)
    c = W.instances(base, 2, seed=3)[1]
    h = base.d_m[0]
    for d in c.dats:
        a = d.init[0]
        assert np.all(a[:h, :] == 0.0) and np.all(a[:, :h] == 0.0)
        assert np.all(a[h:-h, h:-h] > 0.0)
