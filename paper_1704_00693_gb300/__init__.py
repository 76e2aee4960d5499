"""Python binding of libopstile (include/opstile.h): argument marshalling only.

Every function keeps the C name and signature shape; handles are ints,
host arrays are numpy arrays, device addresses are ints.  A non-zero status
raises OpsError carrying the code and ops_last_error's message.  The CUDA
library must have been built (`paper_1704_00693_gb300._build.build()`, or
`__graft_entry__.build()`); importing this module without it fails loudly —
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

OPS_OK = 0
OPS_ERR_INVALID_ARG = -1
OPS_ERR_BOUNDS = -2
OPS_ERR_DEVICE_BOUNDS = -3
OPS_ERR_NOMEM = -4
OPS_ERR_TIMEOUT = -5
OPS_ERR_NOT_CONVERGED = -6
OPS_ERR_CUDA = -7
OPS_ERR_STATE = -8
OPS_ERR_NO_DEVICE = -9

(OPS_MODE_UNTILED, OPS_MODE_SKEWED, OPS_MODE_OVERLAPPED, OPS_MODE_AUTO, OPS_MODE_WAVEFRONT,
 OPS_MODE_TILEWAVE, OPS_MODE_TILEWARP) = 0, 1, 2, 3, 4, 5, 6
OPS_ARG_DAT, OPS_ARG_SCALAR, OPS_ARG_RED = 0, 1, 2
OPS_READ, OPS_WRITE, OPS_RW, OPS_INC = 0, 1, 2, 3
OPS_RED_SUM, OPS_RED_MIN, OPS_RED_MAX = 0, 1, 2
OPS_DEVICE_NONE = -1
OPS_REAL_F64, OPS_REAL_F32 = 0, 1
# loop-body IR opcodes (include/opstile.h)
(OPS_IR_LD, OPS_IR_CST, OPS_IR_ADD, OPS_IR_SUB, OPS_IR_MUL, OPS_IR_FMA, OPS_IR_DIV, OPS_IR_MIN, OPS_IR_MAX,
 OPS_IR_SGT, OPS_IR_WSUM, OPS_IR_WACC, OPS_IR_POLY, OPS_IR_ST, OPS_IR_RED) = range(1, 16)

MODES = {"untiled": OPS_MODE_UNTILED, "skewed": OPS_MODE_SKEWED, "overlapped": OPS_MODE_OVERLAPPED,
         "auto": OPS_MODE_AUTO, "wavefront": OPS_MODE_WAVEFRONT, "tilewave": OPS_MODE_TILEWAVE,
         "tilewarp": OPS_MODE_TILEWARP}


class OpsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"opstile error {code}: {msg}")
        self.code = code


class ops_config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("mode", C.c_int), ("tile", C.c_int * 3),
                ("segment", C.c_int), ("check", C.c_int), ("l2_bytes", C.c_int64), ("hbm_budget", C.c_int64),
                ("timeout_ms", C.c_int), ("blocks_per_sm", C.c_int), ("test_skip_barrier_block", C.c_int),
                ("timing", C.c_int), ("interpret", C.c_int), ("real", C.c_int), ("skewed_persistent", C.c_int)]


class ops_arg(C.Structure):
    _fields_ = [("kind", C.c_int), ("handle", C.c_int), ("stencil", C.c_int), ("access", C.c_int)]


class ops_flush_stats(C.Structure):
    _fields_ = [("plan_ms", C.c_double), ("segments", C.c_int), ("loops", C.c_int), ("tiles", C.c_int),
                ("phases", C.c_int), ("barriers", C.c_int), ("launches", C.c_int), ("plan_cache_hits", C.c_int),
                ("mode", C.c_int), ("tile", C.c_int * 3), ("redundant_points", C.c_int64), ("points", C.c_int64),
                ("skew", C.c_int * 3), ("kernel_ms", C.c_double), ("kernel_launches", C.c_int),
                ("tuning", C.c_int), ("compiled", C.c_int), ("compile_ms", C.c_double), ("batched", C.c_int)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k in ("tile", "skew") else getattr(self, k))
                for k, _ in self._fields_}


_lib = None
EXPORTS = []  # filled from the header at import


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libopstile.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise ImportError(f"libopstile.so not built at {p}: run paper_1704_00693_gb300._build.build()")
    L = C.CDLL(p)
    L.ops_last_error.restype = C.c_char_p
    L.ops_config_default.restype = None
    _lib = L
    return L


def _check(ctx, rc: int):
    if rc != OPS_OK:
        msg = load().ops_last_error(ctx).decode(errors="replace") if ctx else ""
        raise OpsError(rc, msg)


def _i3(v) -> C.Array:
    return (C.c_int * 3)(*[int(x) for x in v])


# ---------------------------------------------------------------- lifecycle
def ops_config_default() -> ops_config:
    cfg = ops_config()
    load().ops_config_default(C.byref(cfg))
    return cfg


def ops_init(cfg: Optional[ops_config] = None):
    L = load()
    if cfg is None:
        cfg = ops_config_default()
    ctx = C.c_void_p()
    rc = L.ops_init(C.byref(ctx), C.byref(cfg))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_init failed (no sm_103a device?)" if rc == OPS_ERR_NO_DEVICE else "ops_init failed")
    return ctx


def ops_finalize(ctx):
    _check(None, load().ops_finalize(ctx))


def ops_last_error(ctx) -> str:
    return load().ops_last_error(ctx).decode(errors="replace")


def ops_set_mode(ctx, mode: int, tile: Optional[Sequence[int]] = None, segment: int = 0):
    t = _i3(tile) if tile is not None else None
    _check(ctx, load().ops_set_mode(ctx, C.c_int(mode), t, C.c_int(segment)))


# ------------------------------------------------------------- declarations
def ops_decl_block(ctx, dims: int, name: str = "") -> int:
    out = C.c_int()
    _check(ctx, load().ops_decl_block(ctx, C.c_int(dims), name.encode(), C.byref(out)))
    return out.value


def ops_decl_dat(ctx, block: int, size, d_m, d_p, dev_ptr0: int = 0, pitch: int = 0, plane: int = 0,
                 name: str = "") -> int:
    out = C.c_int()
    _check(ctx, load().ops_decl_dat(ctx, C.c_int(block), _i3(size), _i3(d_m), _i3(d_p), C.c_void_p(dev_ptr0 or None),
                                    C.c_int64(pitch), C.c_int64(plane), name.encode(), C.byref(out)))
    return out.value


def ops_decl_stencil(ctx, dims: int, points, name: str = "") -> int:
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 3))
    out = C.c_int()
    _check(ctx, load().ops_decl_stencil(ctx, C.c_int(dims), C.c_int(pts.shape[0]),
                                        pts.ctypes.data_as(C.POINTER(C.c_int)), name.encode(), C.byref(out)))
    return out.value


def ops_decl_reduction(ctx, op: int) -> int:
    out = C.c_int()
    _check(ctx, load().ops_decl_reduction(ctx, C.c_int(op), C.byref(out)))
    return out.value


# -------------------------------------------------------------------- loops
def ops_decl_scalar(ctx, init: float = 0.0) -> int:
    out = C.c_int()
    _check(ctx, load().ops_decl_scalar(ctx, C.c_double(init), C.byref(out)))
    return out.value


def ops_scalar_set(ctx, h: int, value: float):
    _check(ctx, load().ops_scalar_set(ctx, C.c_int(h), C.c_double(value)))


def ops_scalar_get(ctx, h: int) -> float:
    v = C.c_double()
    _check(ctx, load().ops_scalar_get(ctx, C.c_int(h), C.byref(v)))
    return v.value


def ops_par_loop(ctx, block: int, dims: int, rng, args, code, consts, name: str = ""):
    r = np.zeros(6, dtype=np.int32)
    for d in range(dims):
        r[2 * d], r[2 * d + 1] = rng[d]
    a = (ops_arg * max(1, len(args)))(*[ops_arg(*x) for x in args])
    code = np.ascontiguousarray(np.asarray(code, dtype=np.int32).reshape(-1, 6))
    consts = np.ascontiguousarray(np.asarray(consts, dtype=np.float64).ravel())
    _check(ctx, load().ops_par_loop(ctx, C.c_int(block), C.c_int(dims), r.ctypes.data_as(C.POINTER(C.c_int)),
                                    C.c_int(len(args)), a, C.c_int(code.shape[0]),
                                    code.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int(consts.size),
                                    consts.ctypes.data_as(C.POINTER(C.c_double)), name.encode()))


def ops_execute(ctx):
    _check(ctx, load().ops_execute(ctx))


def ops_execute_batch(ctxs):
    """Flush the matching chains queued on every context of ctxs as one batch."""
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    _check(ctxs[0] if len(ctxs) else None, load().ops_execute_batch(arr, C.c_int(len(ctxs))))


def ops_sync(ctx):
    _check(ctx, load().ops_sync(ctx))


def ops_queue_clear(ctx):
    _check(ctx, load().ops_queue_clear(ctx))


def ops_reduction_result(ctx, red: int) -> float:
    v = C.c_double()
    _check(ctx, load().ops_reduction_result(ctx, C.c_int(red), C.byref(v)))
    return v.value


# ------------------------------------------------------------ data movement
def ops_dat_info(ctx, dat: int):
    p = C.c_void_p()
    pitch = C.c_int64()
    plane = C.c_int64()
    ext = (C.c_int * 3)()
    _check(ctx, load().ops_dat_info(ctx, C.c_int(dat), C.byref(p), C.byref(pitch), C.byref(plane), ext))
    return (p.value or 0), pitch.value, plane.value, tuple(ext)


def ops_dat_fetch(ctx, dat: int, out: Optional[np.ndarray] = None, dtype=np.float64) -> np.ndarray:
    """The dat's allocation box as a dense (ez, ey, ex) array of the
    context's element type (dtype float32 for an OPS_REAL_F32 context)."""
    _, _, _, ext = ops_dat_info(ctx, dat)
    if out is None:
        out = np.empty((ext[2], ext[1], ext[0]), dtype=dtype)
    assert out.dtype in (np.float64, np.float32) and out.flags.c_contiguous and out.size == ext[0] * ext[1] * ext[2]
    _check(ctx, load().ops_dat_fetch(ctx, C.c_int(dat), C.c_void_p(out.ctypes.data), C.c_int64(out.size)))
    return out


def ops_dat_upload(ctx, dat: int, host: np.ndarray, dtype=np.float64):
    h = np.ascontiguousarray(host, dtype=dtype)
    _check(ctx, load().ops_dat_upload(ctx, C.c_int(dat), C.c_void_p(h.ctypes.data), C.c_int64(h.size)))


def ops_dat_fetch_async(ctx, dat: int, out: np.ndarray):
    """Queue a fetch into `out` (C-contiguous float64, pinned for overlap);
    the values are there once ops_sync returns."""
    assert out.dtype in (np.float64, np.float32) and out.flags.c_contiguous
    _check(ctx, load().ops_dat_fetch_async(ctx, C.c_int(dat), C.c_void_p(out.ctypes.data), C.c_int64(out.size)))


def ops_dat_upload_async(ctx, dat: int, host: np.ndarray):
    """Queue an upload from `host` (C-contiguous float64, kept unchanged until
    ops_sync returns)."""
    assert host.dtype in (np.float64, np.float32) and host.flags.c_contiguous
    _check(ctx, load().ops_dat_upload_async(ctx, C.c_int(dat), C.c_void_p(host.ctypes.data), C.c_int64(host.size)))


def ops_last_stats(ctx) -> dict:
    s = ops_flush_stats()
    _check(ctx, load().ops_last_stats(ctx, C.byref(s)))
    return s.as_dict()


def ops_set_timing(ctx, timing: bool):
    _check(ctx, load().ops_set_timing(ctx, 1 if timing else 0))


def ops_plan_skewed(ctx, tile, ndim: int, nloops: int):
    """Algorithm 1 ranges for the queued loops: list over d of arrays
    [ntiles_d, nloops, 2]."""
    cap = 2 * nloops * sum(max(1, 4096) for _ in range(ndim)) * 64
    buf = np.zeros(cap, dtype=np.int32)
    nt = (C.c_int * 3)()
    t = _i3(list(tile) + [1] * (3 - len(tile)))
    _check(ctx, load().ops_plan_skewed(ctx, t, nt, buf.ctypes.data_as(C.POINTER(C.c_int)), C.c_int64(cap)))
    out, pos = [], 0
    for d in range(ndim):
        n = nt[d] * nloops * 2
        out.append(buf[pos:pos + n].reshape(nt[d], nloops, 2).copy())
        pos += n
    return out


def ops_plan_overlapped(ctx, owned, nloops: int, ndats: int):
    """Overlapped-tile geometry of one tile for the queued loops: (boxes
    [nloops, 3, 2], footprints [ndats, 3, 2]); owned = per-dimension (lo, hi)."""
    o = np.zeros(6, dtype=np.int32)
    for d in range(3):
        o[2 * d], o[2 * d + 1] = owned[d] if d < len(owned) else (0, 1)
    boxes = np.zeros(6 * max(1, nloops), dtype=np.int32)
    foot = np.zeros(6 * max(1, ndats), dtype=np.int32)
    ip = C.POINTER(C.c_int)
    _check(ctx, load().ops_plan_overlapped(ctx, o.ctypes.data_as(ip), boxes.ctypes.data_as(ip),
                                           foot.ctypes.data_as(ip)))
    return boxes[:6 * nloops].reshape(nloops, 3, 2).copy(), foot[:6 * ndats].reshape(ndats, 3, 2).copy()


def ops_plan_wavefront(ctx, tile):
    """Wavefront plan of the queued loops for the given tile sizes:
    (phases, deps, nunits, nlevels), phases an int32 array [nphases, 12] of
    (loop, chunks, first work unit, first dependency entry, dependency count,
    level, x0, x1, y0, y1, z0, z1) in Algorithm 2 order and deps the
    dependency entries (indices of earlier phases)."""
    counts = (C.c_int64 * 4)()
    t = _i3(list(tile) + [1] * (3 - len(tile)))
    _check(ctx, load().ops_plan_wavefront(ctx, t, counts, None, C.c_int64(0), None, C.c_int64(0)))
    nph, ndep = counts[0], counts[1]
    ph = np.zeros((max(1, nph), 12), dtype=np.int32)
    dp = np.zeros(max(1, ndep), dtype=np.int32)
    ip = C.POINTER(C.c_int)
    _check(ctx, load().ops_plan_wavefront(ctx, t, counts, ph.ctypes.data_as(ip), C.c_int64(ph.size),
                                          dp.ctypes.data_as(ip), C.c_int64(dp.size)))
    return ph[:nph].copy(), dp[:ndep].copy(), int(counts[2]), int(counts[3])


def ops_plan_tilewave(ctx, tile):
    """Tile-wavefront plan of the queued loops for the given tile sizes:
    (need, tile_class, order, steps), need an int32 array [classes,
    directions, loops], tile_class the class of each tile (x fastest), order
    the tile of each ticket and steps the first loop of each step of a tile
    followed by the number of loops."""
    counts = (C.c_int64 * 5)()
    t = _i3(list(tile) + [1] * (3 - len(tile)))
    _check(ctx, load().ops_plan_tilewave(ctx, t, counts, None, C.c_int64(0), None, None, C.c_int64(0), None))
    ntiles, ncl, ndirs, nloops, nsteps = (int(v) for v in counts)
    need = np.zeros(max(1, ncl * ndirs * nloops), dtype=np.int32)
    cls = np.zeros(max(1, ntiles), dtype=np.int32)
    order = np.zeros(max(1, ntiles), dtype=np.int32)
    steps = np.zeros(nsteps + 1, dtype=np.int32)
    ip = C.POINTER(C.c_int)
    _check(ctx, load().ops_plan_tilewave(ctx, t, counts, need.ctypes.data_as(ip), C.c_int64(need.size),
                                         cls.ctypes.data_as(ip), order.ctypes.data_as(ip), C.c_int64(ntiles),
                                         steps.ctypes.data_as(ip)))
    return (need[:ncl * ndirs * nloops].reshape(ncl, ndirs, nloops).copy(), cls[:ntiles].copy(), order[:ntiles].copy(),
            steps)


def ops_compile_queued(ctx, want_source: bool = False, wavefront: bool = False, tilewave: bool = False,
                       batch: bool = False, skewed: bool = False, tilewarp: bool = False):
    """Generate and compile (NVRTC, sm_103a, no device) the loop bodies of the
    queued loops -- the per-loop and overlapped-tile kernels, or with
    wavefront=True the wavefront kernel, with tilewave=True the
    tile-wavefront kernel (batch=True: its batch form), with skewed=True the
    persistent skewed kernel; returns (source or None, source length,
    compile ms)."""
    f = (load().ops_compile_queued_tilewarp if tilewarp else
         load().ops_compile_queued_skewed if skewed else
         load().ops_compile_queued_tilewave_batch if tilewave and batch else
         load().ops_compile_queued_tilewave if tilewave else
         load().ops_compile_queued_wavefront if wavefront else load().ops_compile_queued)
    n = C.c_int64(0)
    ms = C.c_double(0.0)
    buf = None
    if want_source:
        _check(ctx, f(ctx, None, C.c_int64(0), C.byref(n), C.byref(ms)))
        buf = C.create_string_buffer(n.value + 1)
    _check(ctx, f(ctx, buf, C.c_int64(n.value + 1 if buf is not None else 0), C.byref(n), C.byref(ms)))
    return (buf.value.decode() if buf is not None else None), n.value, ms.value


# ------------------------------------------------------------ hardware probes
class ops_probe_result(C.Structure):
    _fields_ = [("fp64_fma_tflops", C.c_double), ("fp64_add_tops", C.c_double), ("fp32_fma_tflops", C.c_double),
                ("l2_read_gbs", C.c_double), ("hbm_copy_gbs", C.c_double), ("grid_barrier_us", C.c_double),
                ("flag_roundtrip_us", C.c_double), ("l2_bytes", C.c_int64), ("persisting_l2_max_bytes", C.c_int64),
                ("num_sms", C.c_int), ("sm_clock_khz_max", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def ops_probe_device(device: int = 0) -> dict:
    """Measured FP64/FP32 rates, L2 and HBM bandwidth and synchronisation costs of `device`."""
    out = ops_probe_result()
    rc = load().ops_probe_device(C.c_int(device), C.byref(out))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_probe_device failed")
    return out.as_dict()


# ------------------------------------------------ one loop, no device allocation
class ops_dat_view(C.Structure):
    _fields_ = [("ptr0", C.c_void_p), ("pitch", C.c_int64), ("plane", C.c_int64), ("lo", C.c_int * 3),
                ("hi", C.c_int * 3)]


def ops_loop_noalloc(dims: int, rng, args, views, stencils, code, consts, scalar_values=None, red_ops=None,
                     stream: int = 0):
    """Run one loop over caller-owned dats without allocating device memory.

    args: (kind, access) per argument; views: per argument an ops_dat_view
    (or None for non-dat args); stencils: per argument a list of 3-int
    offsets (None for non-dat args); scalar_values / red_ops: per argument
    (ignored where not SCALAR / RED).  Returns the per-argument reduction
    results (None where not RED)."""
    n = len(args)
    r = np.zeros(6, dtype=np.int32)
    for d in range(dims):
        r[2 * d], r[2 * d + 1] = rng[d]
    a = (ops_arg * max(1, n))(*[ops_arg(k, 0, 0, acc) for k, acc in args])
    v = (ops_dat_view * max(1, n))(*[x if x is not None else ops_dat_view() for x in views])
    npts = np.array([len(s) if s is not None else 0 for s in stencils], dtype=np.int32)
    offs = [p for s in stencils if s is not None for p in s]
    offs = np.ascontiguousarray(np.asarray(offs if offs else [(0, 0, 0)], dtype=np.int32).reshape(-1, 3))
    code = np.ascontiguousarray(np.asarray(code, dtype=np.int32).reshape(-1, 6))
    consts = np.ascontiguousarray(np.asarray(consts, dtype=np.float64).ravel())
    sv = np.ascontiguousarray(np.asarray(scalar_values if scalar_values is not None else [0.0] * n, dtype=np.float64))
    ro = np.ascontiguousarray(np.asarray(red_ops if red_ops is not None else [0] * n, dtype=np.int32))
    out = np.full(max(1, n), np.nan)
    rc = load().ops_loop_noalloc(C.c_int(dims), r.ctypes.data_as(C.POINTER(C.c_int)), C.c_int(n), a, v,
                                 npts.ctypes.data_as(C.POINTER(C.c_int)), offs.ctypes.data_as(C.POINTER(C.c_int)),
                                 C.c_int(code.shape[0]), code.ctypes.data_as(C.POINTER(C.c_int32)),
                                 C.c_int(consts.size), consts.ctypes.data_as(C.POINTER(C.c_double)),
                                 sv.ctypes.data_as(C.POINTER(C.c_double)), ro.ctypes.data_as(C.POINTER(C.c_int)),
                                 out.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream or None))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_loop_noalloc failed")
    return [float(out[i]) if args[i][0] == OPS_ARG_RED else None for i in range(n)]


# ------------------------------------------------------ heat-conduction solves
OPS_PREC_FP64, OPS_PREC_MIXED = 0, 1


class ops_cg_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("precision", C.c_int), ("maxit", C.c_int),
                ("maxouter", C.c_int)]


class ops_cg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("converged", C.c_int), ("relres", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _cg_params(tol, precision, maxit, inner_tol, maxouter):
    return ops_cg_params(float(tol), float(inner_tol), int(precision), int(maxit), int(maxouter))


def ops_heat_apply(ctx, kappa: np.ndarray, u: np.ndarray, precision: int = OPS_PREC_FP64) -> np.ndarray:
    n = kappa.shape[0]
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    w = np.empty((n, n))
    P = C.POINTER(C.c_double)
    _check(ctx, load().ops_heat_apply(ctx, C.c_int(n), k.ctypes.data_as(P), uu.ctypes.data_as(P),
                                      C.c_int(precision), w.ctypes.data_as(P)))
    return w


def ops_cg_solve_batch(ctx, kappas, rhss, tol: float, precision: int, maxit: int = 100000, inner_tol: float = 0.0,
                       maxouter: int = 0):
    """Solve len(kappas) systems together; returns (list of x, list of stats
    dicts).  A solve that hits maxit is reported by stats['converged'] == 0."""
    cnt = len(kappas)
    ks = [np.ascontiguousarray(k, dtype=np.float64) for k in kappas]
    bs = [np.ascontiguousarray(b, dtype=np.float64) for b in rhss]
    xs = [np.empty_like(k) for k in ks]
    ns = (C.c_int * cnt)(*[k.shape[0] for k in ks])
    P = C.POINTER(C.c_double)
    kp = (P * cnt)(*[k.ctypes.data_as(P) for k in ks])
    bp = (P * cnt)(*[b.ctypes.data_as(P) for b in bs])
    xp = (P * cnt)(*[x.ctypes.data_as(P) for x in xs])
    st = (ops_cg_stats * cnt)()
    prm = _cg_params(tol, precision, maxit, inner_tol, maxouter)
    rc = load().ops_cg_solve_batch(ctx, C.c_int(cnt), ns, kp, bp, C.byref(prm), xp, st)
    if rc not in (OPS_OK, OPS_ERR_NOT_CONVERGED):
        _check(ctx, rc)
    return xs, [s.as_dict() for s in st]


def ops_cg_solve(ctx, kappa, rhs, tol: float, precision: int, maxit: int = 100000, inner_tol: float = 0.0,
                 maxouter: int = 0):
    xs, st = ops_cg_solve_batch(ctx, [kappa], [rhs], tol, precision, maxit, inner_tol, maxouter)
    return xs[0], st[0]


# ------------------------------------------------------------------ serving
class ops_serve_config(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget", C.c_int64), ("max_batch", C.c_int), ("ticks_per_poll", C.c_int),
                ("params", ops_cg_params)]


class ops_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("converged", C.c_int), ("relres", C.c_double),
                ("queue_ms", C.c_double), ("service_ms", C.c_double), ("latency_ms", C.c_double),
                ("submit_ms", C.c_double), ("done_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def ops_serve_open(tol: float, precision: int, hbm_budget: int, device: int = 0, max_batch: int = 0,
                   ticks_per_poll: int = 0, maxit: int = 100000, inner_tol: float = 0.0, maxouter: int = 0):
    cfg = ops_serve_config(device, int(hbm_budget), int(max_batch), int(ticks_per_poll),
                           _cg_params(tol, precision, maxit, inner_tol, maxouter))
    srv = C.c_void_p()
    rc = load().ops_serve_open(C.byref(srv), C.byref(cfg))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_serve_open failed")
    return srv


def ops_serve_submit(srv, kappa: np.ndarray, rhs: np.ndarray, tol: float = 0.0, precision: int = -1) -> int:
    """Queue a solve; tol <= 0 / precision < 0 take the server's parameters."""
    n = kappa.shape[0]
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    b = np.ascontiguousarray(rhs, dtype=np.float64)
    rid = C.c_uint64()
    P = C.POINTER(C.c_double)
    rc = load().ops_serve_submit(srv, C.c_int(n), k.ctypes.data_as(P), b.ctypes.data_as(P), C.c_double(tol),
                                 C.c_int(precision), C.byref(rid))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_serve_submit failed")
    return rid.value


def ops_serve_poll(srv, rid: int, n: int, wait: bool = True):
    """(x, stats) once done; None while pending (wait=False)."""
    x = np.empty((n, n))
    st = ops_solve_stats()
    rc = load().ops_serve_poll(srv, C.c_uint64(rid), C.c_int(1 if wait else 0),
                               x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
    if rc == OPS_ERR_STATE:
        return None
    if rc != OPS_OK:
        raise OpsError(rc, "ops_serve_poll failed")
    return x, st.as_dict()


class ops_serve_counters(C.Structure):
    _fields_ = [("admitted", C.c_int64), ("completed", C.c_int64), ("rounds", C.c_int64), ("upload_ms", C.c_double),
                ("run_ms", C.c_double), ("fetch_ms", C.c_double), ("idle_ms", C.c_double)]


def ops_serve_stats(srv) -> dict:
    out = ops_serve_counters()
    rc = load().ops_serve_stats(srv, C.byref(out))
    if rc != OPS_OK:
        raise OpsError(rc, "ops_serve_stats failed")
    return {k: getattr(out, k) for k, _ in out._fields_}


def ops_serve_close(srv):
    rc = load().ops_serve_close(srv)
    if rc != OPS_OK:
        raise OpsError(rc, "ops_serve_close failed")
