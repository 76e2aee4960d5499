"""Conjugate gradients written as a loop chain, TeaLeaf's form (Sec. 5).

The 5-point heat-conduction operator (A u)_c = d_c u_c - sum_f k_f u_nb, with
k_f the harmonic mean of the two cells' conductivity (a boundary face takes
the cell's own) and d_c = 1 + sum_f k_f, applied through ops_par_loop: the
face coefficients and the diagonal are set up by loops on the device, and
every CG iteration is three loops,

    w = A p          with the reduction p.w
    x += a p, r -= a w   with the reduction r.r
    p = r + b p

where the host reads both reductions (the flush points of Sec. 4.A) to form
a and b and to test convergence, and hands them to the loops as
device-resident scalars (ops_decl_scalar / ops_scalar_set).  All arithmetic
is FP64.  This is the application code of the plain OPS-style solver that
the batched engine (ops_cg_solve_batch) and the served solves are measured
against; run with mode "untiled" it is one kernel per loop.  It sits beside
the benchmark, outside the library package: the library only runs the loops
it is given.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import numpy as np

from paper_1704_00693_gb300 import (OPS_ARG_DAT, OPS_ARG_RED, OPS_ARG_SCALAR, MODES, OPS_READ, OPS_RED_SUM, OPS_RW,
                                    OPS_WRITE, OPS_IR_ADD, OPS_IR_CST, OPS_IR_DIV, OPS_IR_FMA, OPS_IR_LD, OPS_IR_MUL,
                                    OPS_IR_RED, OPS_IR_ST, OPS_IR_SUB, _check, load, ops_arg, ops_config_default,
                                    ops_dat_fetch, ops_dat_upload, ops_decl_block, ops_decl_dat, ops_decl_reduction,
                                    ops_decl_scalar, ops_decl_stencil, ops_finalize, ops_init, ops_reduction_result,
                                    ops_scalar_set)


def _ins(*rows):
    """IR rows (op, d, a, b, c, e), padded with zeros, as an int32 array."""
    out = np.zeros((len(rows), 6), dtype=np.int32)
    for i, r in enumerate(rows):
        out[i, :len(r)] = r
    return out


class ChainCG:
    """One n x n problem size; solve() may be called for many problems."""

    def __init__(self, n: int, mode: str = "untiled", device: int = 0, stream: int = 0):
        self.n = n
        cfg = ops_config_default()
        cfg.device = device
        cfg.mode = MODES[mode]
        cfg.stream = stream or None
        self.ctx = ops_init(cfg)
        ctx = self.ctx
        blk = ops_decl_block(ctx, 2, "heat")
        size, h = [n, n, 1], [1, 1, 0]
        names = ["kappa", "b", "x", "r", "p", "w", "dg", "nkx", "nky"]
        self.d = {nm: ops_decl_dat(ctx, blk, size, h, h, name=nm) for nm in names}
        st = {
            "P": [(0, 0, 0)],
            "S5": [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)],
            "EX": [(0, 0, 0), (1, 0, 0)], "EY": [(0, 0, 0), (0, 1, 0)],
            "WX": [(0, 0, 0), (-1, 0, 0)], "SY": [(0, 0, 0), (0, -1, 0)],
        }
        self.s = {k: ops_decl_stencil(ctx, 2, v) for k, v in st.items()}
        self.pw = ops_decl_reduction(ctx, OPS_RED_SUM)
        self.rr = ops_decl_reduction(ctx, OPS_RED_SUM)
        # the step lengths a, -a and b live on the device; the loops read them as SCALAR arguments
        self.sa = ops_decl_scalar(ctx, 0.0)
        self.sna = ops_decl_scalar(ctx, 0.0)
        self.sb = ops_decl_scalar(ctx, 0.0)
        self.blk = blk
        self._ext = (n + 2, n + 2)
        self._host = np.zeros(self._ext, dtype=np.float64)
        self._build_loops()

    # ---- loop descriptors, marshalled once ----
    def _loop(self, rng, args, code, consts):
        r = np.zeros(6, dtype=np.int32)
        for d in range(2):
            r[2 * d], r[2 * d + 1] = rng[d]
        arr = (ops_arg * len(args))(*[ops_arg(k, h, s, a) for k, h, s, a in args])
        consts = np.ascontiguousarray(np.asarray(consts, dtype=np.float64).reshape(-1))
        if consts.size == 0:
            consts = np.zeros(1)
        code = np.ascontiguousarray(code)
        cargs = (C.c_int(self.blk), C.c_int(2), r.ctypes.data_as(C.POINTER(C.c_int)), C.c_int(len(args)), arr,
                 C.c_int(code.shape[0]), code.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int(consts.size),
                 consts.ctypes.data_as(C.POINTER(C.c_double)), b"cg")
        return (r, arr, code, consts, cargs)

    def _build_loops(self):
        n, d, s = self.n, self.d, self.s
        D, RD, SC = OPS_ARG_DAT, OPS_ARG_RED, OPS_ARG_SCALAR
        LD, CST, ADD, SUB, MUL, DIV, FMA, ST, RED = (OPS_IR_LD, OPS_IR_CST, OPS_IR_ADD, OPS_IR_SUB, OPS_IR_MUL,
                                                     OPS_IR_DIV, OPS_IR_FMA, OPS_IR_ST, OPS_IR_RED)
        cells = ((0, n), (0, n))
        # negated face coefficients: -hmean(k_west, k_here) inside, -k at the boundary faces
        hm = _ins((LD, 0, 0, 1), (LD, 1, 0, 0), (CST, 2, 0), (MUL, 3, 2, 0), (MUL, 3, 3, 1), (ADD, 4, 0, 1),
                  (DIV, 5, 3, 4), (CST, 6, 1), (SUB, 7, 6, 5), (ST, 1, 7))
        own = _ins((LD, 0, 0, 0), (CST, 6, 1), (SUB, 7, 6, 0), (ST, 1, 7))
        nbr = _ins((LD, 0, 0, 1), (CST, 6, 1), (SUB, 7, 6, 0), (ST, 1, 7))
        self.setup = [
            self._loop(((1, n), (0, n)), [(D, d["kappa"], s["WX"], OPS_READ), (D, d["nkx"], s["P"], OPS_WRITE)],
                       hm, [2.0, 0.0]),
            self._loop(((0, 1), (0, n)), [(D, d["kappa"], s["WX"], OPS_READ), (D, d["nkx"], s["P"], OPS_WRITE)],
                       own, [2.0, 0.0]),
            self._loop(((n, n + 1), (0, n)), [(D, d["kappa"], s["WX"], OPS_READ), (D, d["nkx"], s["P"], OPS_WRITE)],
                       nbr, [2.0, 0.0]),
            self._loop(((0, n), (1, n)), [(D, d["kappa"], s["SY"], OPS_READ), (D, d["nky"], s["P"], OPS_WRITE)],
                       hm, [2.0, 0.0]),
            self._loop(((0, n), (0, 1)), [(D, d["kappa"], s["SY"], OPS_READ), (D, d["nky"], s["P"], OPS_WRITE)],
                       own, [2.0, 0.0]),
            self._loop(((0, n), (n, n + 1)), [(D, d["kappa"], s["SY"], OPS_READ), (D, d["nky"], s["P"], OPS_WRITE)],
                       nbr, [2.0, 0.0]),
            # d = 1 + k_W + k_E + k_S + k_N
            self._loop(cells, [(D, d["nkx"], s["EX"], OPS_READ), (D, d["nky"], s["EY"], OPS_READ),
                               (D, d["dg"], s["P"], OPS_WRITE)],
                       _ins((CST, 0, 0), (LD, 1, 0, 0), (SUB, 0, 0, 1), (LD, 1, 0, 1), (SUB, 0, 0, 1),
                            (LD, 1, 1, 0), (SUB, 0, 0, 1), (LD, 1, 1, 1), (SUB, 0, 0, 1), (ST, 2, 0)), [1.0]),
            # x = 0, r = p = b, r.r
            self._loop(cells, [(D, d["b"], s["P"], OPS_READ), (D, d["x"], s["P"], OPS_WRITE),
                               (D, d["r"], s["P"], OPS_WRITE), (D, d["p"], s["P"], OPS_WRITE),
                               (RD, self.rr, -1, OPS_READ)],
                       _ins((CST, 0, 0), (ST, 1, 0), (LD, 1, 0, 0), (ST, 2, 1), (ST, 3, 1), (MUL, 2, 1, 1),
                            (RED, 4, 2)), [0.0]),
        ]
        # w = A p (the engine's term order) and p.w
        self.matvec = self._loop(
            cells, [(D, d["p"], s["S5"], OPS_READ), (D, d["dg"], s["P"], OPS_READ), (D, d["nkx"], s["EX"], OPS_READ),
                    (D, d["nky"], s["EY"], OPS_READ), (D, d["w"], s["P"], OPS_WRITE), (RD, self.pw, -1, OPS_READ)],
            _ins((LD, 0, 1, 0), (LD, 1, 0, 0), (MUL, 2, 0, 1),
                 (LD, 0, 2, 0), (LD, 1, 0, 1), (FMA, 2, 0, 1, 2),
                 (LD, 0, 2, 1), (LD, 1, 0, 2), (FMA, 2, 0, 1, 2),
                 (LD, 0, 3, 0), (LD, 1, 0, 3), (FMA, 2, 0, 1, 2),
                 (LD, 0, 3, 1), (LD, 1, 0, 4), (FMA, 2, 0, 1, 2),
                 (ST, 4, 2), (LD, 1, 0, 0), (MUL, 3, 1, 2), (RED, 5, 3)), [0.0])
        # x += a p; r -= a w; r.r   (scalars a and -a)
        self.update = self._loop(
            cells, [(D, d["p"], s["P"], OPS_READ), (D, d["w"], s["P"], OPS_READ), (D, d["x"], s["P"], OPS_RW),
                    (D, d["r"], s["P"], OPS_RW), (RD, self.rr, -1, OPS_READ), (SC, self.sa, -1, OPS_READ),
                    (SC, self.sna, -1, OPS_READ)],
            _ins((LD, 0, 5, 0), (LD, 1, 0, 0), (LD, 2, 2, 0), (FMA, 3, 0, 1, 2), (ST, 2, 3),
                 (LD, 0, 6, 0), (LD, 1, 1, 0), (LD, 2, 3, 0), (FMA, 3, 0, 1, 2), (ST, 3, 3),
                 (MUL, 4, 3, 3), (RED, 4, 4)), [0.0])
        # p = r + b p   (scalar b)
        self.direction = self._loop(
            cells, [(D, d["r"], s["P"], OPS_READ), (D, d["p"], s["P"], OPS_RW), (SC, self.sb, -1, OPS_READ)],
            _ins((LD, 0, 2, 0), (LD, 1, 1, 0), (LD, 2, 0, 0), (FMA, 3, 0, 1, 2), (ST, 1, 3)), [0.0])

    def _enqueue(self, loop):
        rc = load().ops_par_loop(self.ctx, *loop[4])
        if rc:
            _check(self.ctx, rc)

    def _red(self, h) -> float:
        out = C.c_double(0.0)
        _check(self.ctx, load().ops_reduction_result(self.ctx, C.c_int(h), C.byref(out)))
        return out.value

    def _upload(self, name, a):
        self._host[1:self.n + 1, 1:self.n + 1] = a
        ops_dat_upload(self.ctx, self.d[name], self._host)

    def solve(self, kappa: np.ndarray, b: np.ndarray, tol: float, maxit: int = 100000
              ) -> Tuple[np.ndarray, int, float]:
        """x with |b - A x| <= tol |b| (recursive residual), the iteration
        count and the final relative residual."""
        n = self.n
        assert kappa.shape == (n, n) and b.shape == (n, n)
        self._upload("kappa", kappa)
        self._upload("b", b)
        for lp in self.setup:
            self._enqueue(lp)
        rr = self._red(self.rr)
        nb = float(np.sqrt(rr))
        it = 0
        relres = 0.0 if nb == 0.0 else 1.0
        while nb > 0.0 and it < maxit:
            self._enqueue(self.matvec)
            pw = self._red(self.pw)
            a = rr / pw
            ops_scalar_set(self.ctx, self.sa, a)
            ops_scalar_set(self.ctx, self.sna, -a)
            self._enqueue(self.update)
            rr_new = self._red(self.rr)
            it += 1
            relres = float(np.sqrt(rr_new)) / nb
            if relres <= tol:
                break
            ops_scalar_set(self.ctx, self.sb, rr_new / rr)
            self._enqueue(self.direction)
            rr = rr_new
        x = ops_dat_fetch(self.ctx, self.d["x"]).reshape(n + 2, n + 2)[1:n + 1, 1:n + 1].copy()
        return x, it, relres

    def close(self):
        if self.ctx is not None:
            ops_finalize(self.ctx)
            self.ctx = None
