"""Submit a loop-chain program through the C ABI (argument marshalling only).

A program object has the fields of the interchange format described in
`synth.program` (block geometry, dat initial values, stencils, reductions,
the loops of one step); this helper declares everything once and then, per
step, queues the loops with ops_par_loop and reads every reduction with
ops_reduction_result, which is the flush point of the step (Sec. 4.A).
"""
from __future__ import annotations

import time
from typing import List, Optional

import numpy as np

from . import (OPS_ARG_DAT, OPS_MODE_AUTO, MODES, ops_config_default, ops_dat_fetch, ops_dat_upload,
               ops_decl_block, ops_decl_dat, ops_decl_reduction, ops_decl_stencil, ops_execute, ops_execute_batch,
               ops_finalize, ops_init, ops_last_stats, ops_par_loop, ops_reduction_result, ops_set_mode, ops_sync)


class ChainRunner:
    def __init__(self, chain, mode: str = "auto", tile=None, segment: int = 0, check: bool = False,
                 stream: int = 0, device: int = 0, ctx=None, blocks_per_sm: int = 0, timeout_ms: int = 0,
                 skip_barrier_block: int = -1, upload: bool = True, timing: bool = False,
                 interpret: bool = False, fp32: bool = False, skewed_persistent: bool = False):
        self.chain = chain
        self.dtype = np.float32 if fp32 else np.float64
        self.own_ctx = ctx is None
        if ctx is None:
            cfg = ops_config_default()
            cfg.device = device
            cfg.mode = MODES[mode]
            if tile is not None:
                for d, t in enumerate(tile):
                    cfg.tile[d] = int(t)
            cfg.segment = segment
            cfg.check = 1 if check else 0
            cfg.stream = stream or None
            cfg.blocks_per_sm = blocks_per_sm
            if timeout_ms:
                cfg.timeout_ms = timeout_ms
            cfg.test_skip_barrier_block = skip_barrier_block
            cfg.timing = 1 if timing else 0
            cfg.interpret = 1 if interpret else 0
            cfg.real = 1 if fp32 else 0
            cfg.skewed_persistent = 1 if skewed_persistent else 0
            ctx = ops_init(cfg)
        else:
            ops_set_mode(ctx, MODES[mode], tile, segment)
        self.ctx = ctx
        c = chain
        self.block = ops_decl_block(ctx, c.ndim, c.name)
        self.dats = [ops_decl_dat(ctx, self.block, c.size, c.d_m, c.d_p, name=d.name) for d in c.dats]
        if upload:
            for h, d in zip(self.dats, c.dats):
                ops_dat_upload(ctx, h, d.init, self.dtype)
        self.stencils = [ops_decl_stencil(ctx, c.ndim, pts) for pts in c.stencils]
        self.reds = [ops_decl_reduction(ctx, op) for op in c.reductions]
        self.dt = 1.0
        self.history: List[List[float]] = []

    def set_timing(self, on: bool):
        """Per-kernel timing events on or off for later steps (kernel_ms in stats)."""
        from . import ops_set_timing
        ops_set_timing(self.ctx, on)

    def upload(self):
        for h, d in zip(self.dats, self.chain.dats):
            ops_dat_upload(self.ctx, h, d.init, self.dtype)

    def _marshal(self):
        """ctypes arguments of every loop, built once; only constants change per step."""
        import ctypes as C
        from . import load, ops_arg
        L = load()
        self._calls = []
        c = self.chain
        for lp in c.loops:
            r = np.zeros(6, dtype=np.int32)
            for d in range(c.ndim):
                r[2 * d], r[2 * d + 1] = lp.rng[d]
            args = []
            for a in lp.args:
                if a.kind == OPS_ARG_DAT:
                    args.append(ops_arg(a.kind, self.dats[a.handle], self.stencils[a.stencil], a.access))
                else:
                    args.append(ops_arg(a.kind, self.reds[a.handle], -1, a.access))
            arr = (ops_arg * max(1, len(args)))(*args)
            code = np.ascontiguousarray(lp.code.astype(np.int32))
            consts = np.ascontiguousarray(lp.consts.astype(np.float64))
            # ctypes arguments converted once (the arrays stay alive in the tuple)
            cargs = (C.c_int(self.block), C.c_int(self.chain.ndim), r.ctypes.data_as(C.POINTER(C.c_int)),
                     C.c_int(len(args)), arr, C.c_int(code.shape[0]), code.ctypes.data_as(C.POINTER(C.c_int32)),
                     C.c_int(consts.size), consts.ctypes.data_as(C.POINTER(C.c_double)), lp.name.encode())
            self._calls.append((lp, r, code, consts, cargs))
        self._L = L

    def enqueue_step(self, dt: Optional[float] = None):
        import ctypes as C
        from . import _check
        if not hasattr(self, "_calls"):
            self._marshal()
        dt = self.dt if dt is None else dt
        L = self._L
        par_loop, ctx = L.ops_par_loop, self.ctx
        for lp, r, code, consts, cargs in self._calls:
            if lp.dt_slot >= 0:
                consts[lp.dt_slot] = lp.dt_scale * dt
            rc = par_loop(ctx, *cargs)
            if rc:
                _check(ctx, rc)

    def step(self) -> List[float]:
        """Queue one step and flush it by reading every reduction."""
        self.enqueue_step()
        if self.reds:
            vals = [ops_reduction_result(self.ctx, r) for r in self.reds]
        else:
            ops_execute(self.ctx)
            vals = []
        self.history.append(vals)
        if self.chain.dt_red >= 0:
            self.dt = vals[self.chain.dt_red]
        return vals

    def run(self, steps: Optional[int] = None):
        n = self.chain.steps if steps is None else steps
        for _ in range(n):
            self.step()
        ops_sync(self.ctx)
        return self.history

    def fetch(self) -> List[np.ndarray]:
        return [ops_dat_fetch(self.ctx, h, dtype=self.dtype) for h in self.dats]

    def stats(self) -> dict:
        return ops_last_stats(self.ctx)

    def close(self):
        if self.own_ctx and self.ctx is not None:
            ops_finalize(self.ctx)
            self.ctx = None


def run_batch(runners: List[ChainRunner], steps: Optional[int] = None, sync: bool = True):
    """Step the runners' chains together: per step every chain is queued,
    all are flushed by one ops_execute_batch, then every reduction of every
    runner is read (each runner's next dt comes from its own)."""
    n = runners[0].chain.steps if steps is None else steps
    ctxs = [r.ctx for r in runners]
    for _ in range(n):
        for r in runners:
            r.enqueue_step()
        ops_execute_batch(ctxs)
        for r in runners:
            vals = [ops_reduction_result(r.ctx, h) for h in r.reds]
            r.history.append(vals)
            if r.chain.dt_red >= 0:
                r.dt = vals[r.chain.dt_red]
    if sync:
        for r in runners:
            ops_sync(r.ctx)
    return [r.history for r in runners]
