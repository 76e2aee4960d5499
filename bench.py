#!/usr/bin/env python3
"""Loop-chain benchmark on one GB300: effective GB/s of the CloverLeaf-2D-shaped
chain (3840^2 FP64, 25 dats, 83 loops and two reductions per step), tiled
(skewed, one persistent kernel per step) against the untiled
one-kernel-per-loop form on the same GPU.

A step is one pass of the whole chain (83 loops queued through the C ABI,
flushed by reading the step's two reductions).  Effective GB/s counts bytes
the paper's way (Sec. 6.A): every dat argument of a loop costs 8 B per
point of its range, RW twice, stencil re-use ignored.  The dats (3.0 GB)
are larger than the 126 MB L2, so no flush is needed between steps.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Prints one JSON line.  --impl reference times the CPU oracle (untiled,
program order, FP64) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_DEFAULT = 3840
def workload(n: int) -> str:
    return (f"cloverleaf2d-shaped chain: {n}^2 FP64, halo 2, 25 dats U(0.5,1.5), 83 loops + 1 sum + 1 min "
            "reduction per step")
PROFILE = os.path.join(ROOT, "profiles", "chain_cloverleaf2d_3840.md")
KERNEL_SRC = [os.path.join(ROOT, "paper_1704_00693_gb300", "csrc", f) for f in ("jit.cpp", "chain_kernels.cu", "device_common.cuh")]
# FP64 fallback when the probe is skipped: 2 DFMA per clock per SM on GB300, fma = 2 flops
FP64_DFMA_PER_CLK_SM = 2
NUM_SMS = 152
SCHEDULES = {0: "untiled", 1: "skewed", 2: "overlapped", 3: "auto", 4: "wavefront", 5: "tilewave", 6: "tilewarp"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--mode", default="auto", choices=["skewed", "untiled", "overlapped", "wavefront", "tilewave", "tilewarp", "auto"])
    p.add_argument("--no-probe", action="store_true", help="skip the hardware probes (FP64 rate, L2, barriers)")
    p.add_argument("--tile", default="", help="x,y tile (0 = automatic)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-untiled", action="store_true")
    p.add_argument("--no-serve", action="store_true", help="skip the served-solves measurement")
    p.add_argument("--no-cg", action="store_true", help="skip the 4000^2 CG measurement")
    p.add_argument("--no-3d", action="store_true", help="skip the other chains (OpenSBLI 3D, CloverLeaf 3D, PPCG)")
    p.add_argument("--serve-requests", type=int, default=512)
    p.add_argument("--no-batch", action="store_true", help="skip the batched small-grid chains")
    p.add_argument("--only", default="", choices=["", "chain", "fp32", "ppcg", "jacobi", "batch", "probe", "serve"],
                   help="run one section alone on grids of --n points per side and print its JSON (for "
                        "profiling and sweeps): chain = the CloverLeaf-shaped step in --mode (FP64), fp32 = the "
                        "same in FP32, ppcg, jacobi (FP32 heat-equation steps), batch (64 grids), probe (the "
                        "hardware probes with the SM clocks sampled while they run)")
    p.add_argument("--real", default="f64", choices=["f64", "f32"], help="element type of --only chain")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(ms: float, device: str = "cuda") -> float:
    """The slowest rank's time (every rank gets it); ranks are independent
    replicas, so this is the only collective of the benchmark."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(untiled_bytes: float, steps: int, world: int, ms: float) -> float:
    """Whole-job effective GB/s: every rank runs the same chain (weak scaling)."""
    return untiled_bytes * steps * world / (ms * 1e-3) / 1e9


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
def workload_numbers(chain):
    from synth.program import body_flops, loop_points, untiled_bytes
    U = untiled_bytes(chain)
    flops = sum(body_flops(lp, chain) * loop_points(lp) for lp in chain.loops)
    return U, flops


def profile_traffic(schedule, tile):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source with the same
    schedule (mode and tile)."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(open(f, "rb").read())
    src_hash = h.hexdigest()[:16]
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != src_hash:
        return None
    want = schedule if tile is None else f"{schedule} {tile[0]}x{tile[1]}"
    if vals.get("schedule") != want:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def time_mode(chain, mode, tile, steps, warmup, stream, torch, fp32=False):
    """Timed steps without per-kernel events (the value), then as many steps
    of the same settled schedule with per-kernel CUDA events on the launching
    stream (the kernels' durations for the roofline)."""
    from paper_1704_00693_gb300.chain import ChainRunner
    r = ChainRunner(chain, mode=mode, tile=tile, stream=stream.cuda_stream, timing=False, fp32=fp32)
    try:
        for w in range(warmup):
            r.step()
            if w == 0:
                time_mode.first = r.stats()  # plan building and run-time compilation happen here
        # in auto mode, keep warming up until the autotuner has timed every candidate
        extra = 0
        while mode == "auto" and r.stats()["tuning"] and extra < 40:
            r.step()
            extra += 1
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches = 0
        stats = None
        # an NVTX range marks the timed steps, so a profiler can select them
        torch.cuda.nvtx.range_push(f"timed_{mode}")
        e0.record(stream)
        for _ in range(steps):
            r.step()
            stats = r.stats()
            launches += stats["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
        # kernel durations: the same schedule, events around every chain kernel
        r.set_timing(True)
        kms, kl = 0.0, 0
        torch.cuda.nvtx.range_push(f"kernels_{mode}")
        for _ in range(steps):
            r.step()
            st = r.stats()
            kms += st["kernel_ms"]
            kl += st["kernel_launches"]
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    finally:
        r.close()
    return ms, kms, kl, launches, stats


def time_e2e(chain, mode, tile, steps, stream, torch, nctx=3):
    """End to end through the public API: every step uploads all dats from
    pinned host memory (ops_dat_upload_async), runs the step (queue, flush,
    reduction read) and fetches back every dat the step writes, its result
    (ops_dat_fetch_async; the dats it only reads are unchanged), copies
    inside the timed region.  Steps rotate over `nctx` contexts, each on its
    own stream, so one instance's copies overlap another's compute; the host
    waits for every copy before the clock stops."""
    from paper_1704_00693_gb300 import ops_dat_fetch_async, ops_dat_upload_async, ops_sync
    from paper_1704_00693_gb300.chain import ChainRunner
    streams = [torch.cuda.Stream() for _ in range(nctx)]
    runners = [ChainRunner(chain, mode=mode, tile=tile, stream=s.cuda_stream, upload=False) for s in streams]
    try:
        host_in, host_out = [], [[] for _ in range(nctx)]
        for d in chain.dats:
            t = torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = d.init
            host_in.append(t.numpy())
            for k in range(nctx):
                host_out[k].append(torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True).numpy())
        bi = sum(a.size * 8 for a in host_in)
        from synth.program import DAT, READ
        written = sorted({a.handle for lp in chain.loops for a in lp.args if a.kind == DAT and a.access != READ})
        bo = sum(host_in[k].size * 8 for k in written)

        def upload(r):
            for h, a in zip(r.dats, host_in):
                ops_dat_upload_async(r.ctx, h, a)

        # untimed: plans and compiled code of every context
        for r in runners:
            upload(r)
            r.step()
            ops_sync(r.ctx)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upload(runners[0])
        for k in range(steps):
            cur = runners[k % nctx]
            if k + 1 < steps:
                upload(runners[(k + 1) % nctx])
            cur.step()
            for d in written:
                ops_dat_fetch_async(cur.ctx, cur.dats[d], host_out[k % nctx][d])
        for r in runners:
            ops_sync(r.ctx)
        ms = (time.perf_counter() - t0) * 1e3
    finally:
        for r in runners:
            r.close()
    return ms, bi, bo


def time_e2e_sequential(chain, mode, tile, steps, stream, torch):
    """The same per-step copies with one context and blocking calls."""
    from paper_1704_00693_gb300 import ops_dat_fetch, ops_dat_upload
    from paper_1704_00693_gb300.chain import ChainRunner
    r = ChainRunner(chain, mode=mode, tile=tile, stream=stream.cuda_stream, upload=False)
    try:
        host_in, host_out = [], []
        for d in chain.dats:
            t = torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = d.init
            host_in.append(t)
            host_out.append(torch.empty(d.init.shape, dtype=torch.float64, pin_memory=True))
        for h, t in zip(r.dats, host_in):
            ops_dat_upload(r.ctx, h, t.numpy())
        r.step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for h, t in zip(r.dats, host_in):
                ops_dat_upload(r.ctx, h, t.numpy())
            r.step()
            for h, t in zip(r.dats, host_out):
                ops_dat_fetch(r.ctx, h, t.numpy())
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
    finally:
        r.close()
    return ms


def mem_available_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def bench_serving(nreq=512, seq_sample=None, tol=1e-8, budget=48 << 30):
    """Served mixed-size diffusion solves (FP32 sweeps + FP64 refinement,
    continuous batching) against sequential untiled FP64 CG solves on the
    same GPU.  Requests: n uniform over multiples of 64 in [64, 2048],
    conductivity log-uniform in [0.1, 10], RHS U(0,1), tolerance 1e-8."""
    import numpy as np
    import paper_1704_00693_gb300 as ops
    from synth import workloads as W
    reqs = W.serving_stream(nreq)
    need = sum(16 * n * n for _, n, _ in reqs) * 1.2
    reuse = need > 0.5 * mem_available_bytes()
    cache = {}

    def problem(i):
        _, n, s = reqs[i]
        if reuse:  # not enough host memory for every grid: one grid per size
            if n not in cache:
                cache[n] = W.cg_problem(n, 1e-1, 1e1, seed=s)
            return cache[n]
        return W.cg_problem(n, 1e-1, 1e1, seed=s)

    probs = [problem(i) for i in range(nreq)]
    # Sequential untiled FP64 baseline: every request in stream order, one
    # solve at a time, with CG written as a loop chain run untiled (three
    # loops per iteration, both reductions read by the host, Sec. 4.A);
    # compiled code and contexts per grid size are set up before the clock.
    from cg_loopchain import ChainCG
    sizes = sorted({n for _, n, _ in reqs})
    chains = {n: ChainCG(n, mode="untiled") for n in sizes}
    try:
        for n in sizes:
            chains[n].solve(*probs[next(i for i in range(nreq) if reqs[i][1] == n)], tol, maxit=1)
        t0 = time.perf_counter()
        for i in range(nreq):
            chains[reqs[i][1]].solve(*probs[i], tol)
        t_chain = time.perf_counter() - t0
    finally:
        for c in chains.values():
            c.close()
    chain_rate = nreq / t_chain
    # the same stream through the batched engine, one FP64 solve at a time
    seq_sample = nreq if seq_sample is None else min(seq_sample, nreq)
    ctx = ops.ops_init()
    try:
        ops.ops_cg_solve(ctx, *probs[0], tol, ops.OPS_PREC_FP64)  # warm-up
        t0 = time.perf_counter()
        for i in range(seq_sample):
            ops.ops_cg_solve(ctx, *probs[i], tol, ops.OPS_PREC_FP64)
        t_seq = time.perf_counter() - t0
    finally:
        ops.ops_finalize(ctx)
    seq_rate = seq_sample / t_seq
    # scale a sample's rate to the whole stream by the cells it holds
    cells_all = sum(n * n for _, n, _ in reqs)
    cells_sample = sum(reqs[i][1] ** 2 for i in range(seq_sample))
    seq_rate_all = seq_rate * (cells_sample / seq_sample) / (cells_all / nreq)

    def serve(arrivals):
        srv = ops.ops_serve_open(tol, ops.OPS_PREC_MIXED, hbm_budget=budget)
        try:
            ids = []
            t0 = time.perf_counter()
            for i in range(nreq):
                wait = arrivals[i] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                ids.append(ops.ops_serve_submit(srv, *probs[i]))
            res = [ops.ops_serve_poll(srv, rid, reqs[i][1]) for i, rid in enumerate(ids)]
            makespan = time.perf_counter() - t0
            counters = ops.ops_serve_stats(srv)
        finally:
            ops.ops_serve_close(srv)
        lat = np.array([st["latency_ms"] for _, st in res])
        conv = sum(st["converged"] for _, st in res)
        return {"solves_per_s": nreq / makespan, "makespan_s": makespan, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "converged": conv,
                "worker_ms": {k: round(counters[k], 1) for k in ("upload_ms", "run_ms", "fetch_ms", "idle_ms")},
                "rounds": counters["rounds"]}, res

    sat, res = serve([0.0] * nreq)
    # check a few results against the oracle's FP64 residual
    import oracle
    worst = max(oracle.relres(*probs[i], res[i][0]) for i in range(0, nreq, max(1, nreq // 8)))
    loads = {}
    for f in (0.8, 1.5):
        rate = f * chain_rate
        load, _ = serve([t / rate for t, _, _ in reqs])
        loads[f"offered_{f}x_seq"] = dict(load, offered_rate=rate)
    return {"requests": nreq, "sizes": "n uniform over multiples of 64 in [64, 2048]",
            "tol": tol, "precision": "fp32 sweeps + fp64 refinement", "distinct_grids": not reuse,
            "saturation": sat, **loads,
            "sequential_untiled_fp64": {"solves_per_s": chain_rate, "seconds": t_chain,
                                        "how": "CG as a loop chain, untiled, host-read reductions, one solve "
                                               "at a time over the whole stream"},
            "speedup_vs_sequential_untiled_fp64": sat["solves_per_s"] / chain_rate,
            "engine_fp64_one_at_a_time": {"solves_per_s": seq_rate_all, "sample": seq_sample,
                                          "sample_solves_per_s": seq_rate},
            "speedup_vs_engine_fp64_one_at_a_time": sat["solves_per_s"] / seq_rate_all,
            "worst_sampled_oracle_relres": worst}


def bench_cg(n=4000, tol=1e-10):
    """TeaLeaf-shaped solve: conductivity log-uniform in [1e-2, 1e2], RHS
    U(0,1); FP64 CG against FP32 sweeps with FP64 residual and refinement.
    Each form: one untimed full-size solve, then the best of two timed ones
    (host wall clock, uploads of kappa and b and the fetch of x included)."""
    import paper_1704_00693_gb300 as ops
    from synth import workloads as W
    kappa, b = W.cg_problem(n, 1e-2, 1e2)
    ctx = ops.ops_init()
    out = {"n": n, "tol": tol}
    try:
        runs = [("fp64", ops.OPS_PREC_FP64, 0.0), ("mixed_inner1e-4", ops.OPS_PREC_MIXED, 1e-4),
                ("mixed_inner1e-5", ops.OPS_PREC_MIXED, 1e-5), ("mixed_inner1e-6", ops.OPS_PREC_MIXED, 1e-6)]
        for name, prec, itol in runs:
            # a full-size solve first (allocation, graph capture), then the best of two timed ones
            ops.ops_cg_solve(ctx, kappa, b, tol, prec, inner_tol=itol)
            dt = float("inf")
            for _ in range(2):
                t0 = time.perf_counter()
                x, st = ops.ops_cg_solve(ctx, kappa, b, tol, prec, inner_tol=itol)
                dt = min(dt, time.perf_counter() - t0)
            out[name] = {"seconds": dt, "iterations": st["iterations"], "outer": st["outer"],
                         "converged": st["converged"], "relres": st["relres"],
                         "ms_per_iteration": dt * 1e3 / max(1, st["iterations"])}
    finally:
        ops.ops_finalize(ctx)
    # the same solve as a loop chain (three loops per iteration, host-read reductions)
    from cg_loopchain import ChainCG
    cg = ChainCG(n, mode="untiled")
    try:
        cg.solve(kappa, b, tol, maxit=2)  # compiled code and plans
        dt = float("inf")
        for _ in range(2):
            t0 = time.perf_counter()
            x, it, rel = cg.solve(kappa, b, tol)
            dt = min(dt, time.perf_counter() - t0)
        out["fp64_loop_chain_untiled"] = {"seconds": dt, "iterations": it, "relres": rel,
                                          "ms_per_iteration": dt * 1e3 / max(1, it)}
    finally:
        cg.close()
    best = min((k for k in out if k.startswith("mixed")), key=lambda k: out[k]["seconds"])
    out["best_mixed"] = best
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out[best]["seconds"]
    return out


def compare_schedules(chain, stream, torch, schedules, steps=5, fp32=False, bytes_per_elem=8):
    """Effective GB/s of each (mode, tile) schedule of one chain, with the
    speedup of each over the untiled form (the first entry)."""
    U, flops = workload_numbers(chain)
    U = U * bytes_per_elem // 8
    out = {"n": chain.size[0], "untiled_bytes_per_step": U, "flops_per_step": flops, "dtype": "f32" if fp32 else "f64"}
    for mode, tile, key in schedules:
        ms, kms, kl, launches, st = time_mode(chain, mode, tile, steps, 3, stream, torch, fp32=fp32)
        first = getattr(time_mode, "first", None) or {}
        out[key] = {"value": U * steps / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms / steps,
                    "kernel_ms_per_step": kms / steps, "schedule": SCHEDULES.get(st["mode"]), "tile": st["tile"],
                    "tiles": st["tiles"], "plan_ms": first.get("plan_ms"), "compile_ms": first.get("compile_ms")}
    for key in [k for k in out if isinstance(out[k], dict) and k != "untiled"]:
        out[f"speedup_{key}_vs_untiled"] = out["untiled"]["ms_per_step"] / out[key]["ms_per_step"]
    return out


def bench_chain(chain, stream, torch, steps=5):
    """Autotuned schedule and the tile wavefront against the untiled form on one chain."""
    return compare_schedules(chain, stream, torch, [("untiled", None, "untiled"), ("tilewave", None, "tilewave"),
                                                    ("auto", None, "auto")], steps)


def bench_opensbli3d(stream, torch, n=320, steps=5):
    """The OpenSBLI-shaped 3D chain (320^3, 15 dats, 40 loops per step)."""
    from synth import workloads as W
    return bench_chain(W.opensbli3d(n=n, steps=1), stream, torch, steps)


def bench_ppcg(stream, torch, n=4000, inner=10, steps=5):
    """The TeaLeaf-PPCG-shaped chain (one preconditioner application: 7
    setup loops, 10 Chebyshev iterations of three loops, z.r), the paper's
    best tiling case: every schedule against untiled."""
    from synth import workloads as W
    chain = W.ppcg2d(n=n, inner=inner)
    out = compare_schedules(chain, stream, torch, [("untiled", None, "untiled"), ("tilewave", None, "tilewave"),
                                                   ("skewed", None, "skewed"), ("wavefront", None, "wavefront"),
                                                   ("overlapped", None, "overlapped"), ("auto", None, "auto")], steps)
    out["inner"] = inner
    return out


def bench_fp32(stream, torch, n=3840, steps=5):
    """The CloverLeaf-shaped chain in an OPS_REAL_F32 context (float dats and
    arithmetic): every schedule, effective GB/s at 4 bytes per element.  With
    single-precision arithmetic the chain is bound by memory, not by the
    FP64 pipe, which is where tiling pays."""
    from synth import workloads as W
    chain = W.cloverleaf2d(n=n, steps=1)
    return compare_schedules(chain, stream, torch,
                             [("untiled", None, "untiled"), ("tilewave", None, "tilewave"),
                              ("skewed", [0, 1024, 0], "skewed_1024"), ("wavefront", None, "wavefront"),
                              ("auto", None, "auto")], steps, fp32=True, bytes_per_elem=4)


def bench_jacobi(stream, torch, n=8192, iters=10, steps=5):
    """The paper's heat-equation benchmark shape (Sec. 6.A): Jacobi steps of
    the 2D heat equation, `iters` iterations (2 loops each: the 5-point
    update into a second dat, the copy back) per flush, in an FP32 context
    on an n^2 grid (two 256 MB dats at 8192^2): untiled against the tile
    wavefront at its automatic tiles and at 128 x 128, and the autotuner."""
    from synth import workloads as W
    chain = W.jacobi2d(n, iters, init="rand")
    return compare_schedules(chain, stream, torch,
                             [("untiled", None, "untiled"), ("tilewave", None, "tilewave"),
                              ("tilewave", [128, 128, 0], "tilewave_128x128"), ("tilewarp", None, "tilewarp"),
                              ("auto", None, "auto")],
                             steps, fp32=True, bytes_per_elem=4)


def bench_cloverleaf3d(stream, torch, n=330, steps=3):
    """The CloverLeaf-3D-shaped chain (330^3 as in the paper, 30 dats, 141 loops per step)."""
    from synth import workloads as W
    return bench_chain(W.cloverleaf3d(n=n, steps=1), stream, torch, steps)


def bench_batch(torch, chain, count=64, steps=5, warmup=3):
    """Many small grids' chains: `count` instances of `chain` (same loops,
    own field values) stepped together.  Batched: per step every context
    queues its chain and one ops_execute_batch runs each segment of all of
    them: untiled with one launch per loop for all grids, the tile
    wavefront in one launch (automatic tiles), or as the batch autotuner
    picks (auto); sequential: every context flushes on its own (ops_execute,
    each on its own stream, so their kernels may overlap).
    Either way every reduction of every grid is read each step (the
    CloverLeaf time step feeds the next step).  Host wall clock over the
    timed steps, device idle on both sides."""
    from paper_1704_00693_gb300 import ops_execute, ops_reduction_result
    from paper_1704_00693_gb300.chain import ChainRunner, run_batch
    from synth import workloads as W
    chains = W.instances(chain, count)
    out = {"workload": f"{count} x {chain.name}", "count": count, "loops_per_chain": len(chain.loops),
           "unit": "chains/s", "how": "host wall clock, synchronize on both sides; a chain = one step of one grid"}

    def seq_step(runners):
        for r in runners:
            r.enqueue_step()
            ops_execute(r.ctx)
        for r in runners:
            vals = [ops_reduction_result(r.ctx, h) for h in r.reds]
            if r.chain.dt_red >= 0:
                r.dt = vals[r.chain.dt_red]

    shared = torch.cuda.Stream()
    for key, mode, batched in (("sequential_untiled", "untiled", False), ("sequential_auto", "auto", False),
                               ("batched_untiled", "untiled", True), ("batched_tilewave", "tilewave", True),
                               ("batched_auto", "auto", True)):
        # a batch's contexts share one stream (no cross-stream joins); the
        # sequential contexts each have their own, so their kernels may overlap
        runners = [ChainRunner(c, mode=mode, stream=shared.cuda_stream if batched else 0) for c in chains]
        try:
            def one():
                if batched:
                    run_batch(runners, 1, sync=False)
                else:
                    seq_step(runners)
            for _ in range(warmup):
                one()
            extra = 0
            while mode == "auto" and any(r.stats()["tuning"] for r in runners[:1]) and extra < 40:
                one()
                extra += 1
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                one()
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            st = runners[0].stats()
            out[key] = {"value": count * steps / sec, "ms_per_step": sec * 1e3 / steps,
                        "schedule": SCHEDULES.get(st["mode"]), "tile": st["tile"], "tiles_per_grid": st["tiles"],
                        "batched": st["batched"]}
        finally:
            for r in runners:
                r.close()
    best_seq = max(out["sequential_untiled"]["value"], out["sequential_auto"]["value"])
    out["speedup_batched_auto_vs_best_sequential"] = out["batched_auto"]["value"] / best_seq
    return out


def cpu_baseline(n_full, seconds=12.0):
    """The oracle (untiled, program order, FP64, all host cores) on a bounded
    sample: one step of the same chain on a grid with 1/4 of the points."""
    import oracle
    from synth import workloads as W
    n = n_full // 2
    chain = W.cloverleaf2d(n=n, steps=1)
    U, _ = workload_numbers(chain)
    oracle.build()
    dats = [d.init.copy() for d in chain.dats]
    t0 = time.perf_counter()
    nsteps = 0
    while True:
        oracle.run_loops(chain, dats, chain.loops, [oracle.red_identity(op) for op in chain.reductions])
        nsteps += 1
        if time.perf_counter() - t0 > seconds or nsteps >= 30:
            break
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": U * nsteps / t / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
           "sample": f"{nsteps} step(s) of the same chain at {n}^2 (1/4 of the points), untiled FP64 oracle",
           "seconds": t}
    # context: the paper's CPU scheme (Algorithms 1-2, OpenMP inside each tile) on the same cores,
    # tiles of whole rows sized so a tile's 25 dats fill about 32 MB
    rows = max(8, (32 << 20) // (8 * 25 * (n + 4)))
    tsteps = min(nsteps, 3)
    tchain = W.cloverleaf2d(n=n, steps=tsteps)
    t0 = time.perf_counter()
    oracle.run_chain_tiled(tchain, (n + 4, rows))
    tt = time.perf_counter() - t0
    out["skewed_tiled_cpu"] = {"value": U * tsteps / tt / 1e9, "unit": "GB/s", "tile": [n + 4, rows],
                               "steps": tsteps, "speedup_vs_untiled_cpu": (t / nsteps) / (tt / tsteps)}
    out["compiled_cpu"] = compiled_cpu_context(n)
    return out


def compiled_cpu_context(n, seconds=2.0, rows=(32, 64, 128, 256, 512)):
    """Context beside the oracle: the paper's CPU scheme with compiled loop
    bodies (oracle.cpu_compiled; C from the IR, gcc, OpenMP inside each
    tile) on the same sample, untiled and with Algorithm 1 tiles of whole
    rows, each timed over about `seconds`."""
    import numpy as np
    import oracle
    from oracle import cpu_compiled
    from synth import workloads as W
    chain = W.cloverleaf2d(n=n, steps=1)
    U, _ = workload_numbers(chain)
    comp = cpu_compiled.CompiledChain(chain)
    dats = [np.ascontiguousarray(d.init.astype(np.float64)) for d in chain.dats]
    ident = [oracle.red_identity(op) for op in chain.reductions]

    def timed(tile):
        comp.run(dats, ident, 1.0, tile)
        t0, k = time.perf_counter(), 0
        while True:
            comp.run(dats, ident, 1.0, tile)
            k += 1
            if time.perf_counter() - t0 > seconds:
                break
        return (time.perf_counter() - t0) / k

    tu = timed(None)
    out = {"sample": f"one step of the chain at {n}^2", "cores": comp.threads_used,
           "untiled": {"value": U / tu / 1e9, "unit": "GB/s", "ms_per_step": tu * 1e3}, "tiled": {}}
    for r in rows:
        tt = timed((n + 4, r))
        out["tiled"][str(r)] = {"value": U / tt / 1e9, "ms_per_step": tt * 1e3}
    best = min(out["tiled"], key=lambda k: out["tiled"][k]["ms_per_step"])
    out["best_tile_rows"] = int(best)
    out["speedup_tiled_vs_untiled"] = tu * 1e3 / out["tiled"][best]["ms_per_step"]
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from synth import workloads as W
    n = args.n // 2
    chain = W.cloverleaf2d(n=n, steps=1)
    U, _ = workload_numbers(chain)
    oracle.build()
    dats = [d.init.copy() for d in chain.dats]
    ident = [oracle.red_identity(op) for op in chain.reductions]
    for _ in range(args.warmup):
        oracle.run_loops(chain, dats, chain.loops, ident)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run_loops(chain, dats, chain.loops, ident)
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = U * args.steps / t / 1e9
    line = {"metric": "loop-chain effective GB/s", "value": v, "unit": "GB/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.n), "sample": f"each step: the chain at {n}^2 (1/4 of the points)"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step the same chain at {n}^2"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (sm_103a)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1704_00693_gb300 import _build
    _build.build()
    import paper_1704_00693_gb300 as ops
    from synth import workloads as W

    if args.only == "probe":
        with ClockSampler(local) as clk:
            res = ops.ops_probe_device(local)
        print(json.dumps({"only": "probe", "result": res, "clocks": clk.summary()}), flush=True)
        return
    probe = None
    if not args.no_probe:
        try:
            probe = ops.ops_probe_device(local)
        except ops.OpsError as e:
            probe = {"error": str(e)}

    chain = W.cloverleaf2d(n=args.n, steps=1)
    U, flops = workload_numbers(chain)
    tile = None
    if args.tile:
        tile = [int(x) for x in args.tile.split(",")] + [0]
    stream = torch.cuda.Stream()

    if args.only:
        n = args.n
        if args.only == "chain":
            f32 = args.real == "f32"
            ms, kms, kl, launches, st = time_mode(chain, args.mode, tile, args.steps, args.warmup, stream, torch,
                                                  fp32=f32)
            out = {"ms_per_step": ms / args.steps, "kernel_ms_per_step": kms / args.steps, "mode": args.mode,
                   "schedule": SCHEDULES.get(st["mode"]), "tile": st["tile"], "tiles": st["tiles"], "n": n,
                   "real": args.real, "gpu_launches": launches}
        elif args.only == "fp32":
            out = bench_fp32(stream, torch, n=n, steps=args.steps)
        elif args.only == "ppcg":
            out = bench_ppcg(stream, torch, n=n, steps=args.steps)
        elif args.only == "jacobi":
            out = bench_jacobi(stream, torch, n=n, steps=args.steps)
        elif args.only == "serve":
            out = bench_serving(args.serve_requests)
        else:
            out = bench_batch(torch, W.cloverleaf2d(n=n, steps=1), steps=args.steps, warmup=args.warmup)
        print(json.dumps({"only": args.only, "result": out}), flush=True)
        return

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    with ClockSampler(local) as clk:
        ms, kms, kl, launches, st = time_mode(chain, args.mode, tile, args.steps, args.warmup, stream, torch)
    barrier()
    ms = max_over_ranks(ms)
    value = whole_job_gbs(U, args.steps, world, ms)

    first = getattr(time_mode, "first", None) or {}
    untiled = None
    if not args.no_untiled and args.mode != "untiled":
        ums, ukms, ukl, _, _ = time_mode(chain, "untiled", None, args.steps, args.warmup, stream, torch)
        untiled = {"value": U * args.steps / (ums * 1e-3) / 1e9, "ms_per_step": ums / args.steps,
                   "kernel_ms_per_step": ukms / args.steps, "kernel_launches_per_step": ukl / args.steps}
    tilewave = None
    if not args.no_untiled and args.mode != "tilewave":
        tms, tkms, tkl, _, tst = time_mode(chain, "tilewave", None, args.steps, args.warmup, stream, torch)
        tfirst = getattr(time_mode, "first", None) or {}
        tilewave = {"value": U * args.steps / (tms * 1e-3) / 1e9, "ms_per_step": tms / args.steps,
                    "kernel_ms_per_step": tkms / args.steps, "tile": tst["tile"], "tiles": tst["tiles"],
                    "plan": {"plan_ms": tfirst.get("plan_ms"), "compile_ms": tfirst.get("compile_ms"),
                             "phases": tst["phases"], "steps": tst["barriers"], "skew": tst["skew"]},
                    "how": "OPS_MODE_TILEWAVE: Algorithm 1 tiles cut in x and y, each run whole by one CTA, "
                           "tiles concurrent with per-tile progress counters"}

    # the schedule the timed steps ran (the autotuner's pick in auto mode)
    chosen_mode = SCHEDULES.get(st["mode"], "skewed") if st else args.mode
    chosen_tile = list(st["tile"]) if st and chosen_mode != "untiled" else None
    e2e = None
    if not args.no_e2e:
        esteps = max(3, args.steps)
        ems, bi, bo = time_e2e(chain, chosen_mode, chosen_tile, esteps, stream, torch)
        sms = time_e2e_sequential(chain, chosen_mode, chosen_tile, 3, stream, torch)
        e2e = {"value": U * esteps / (ems * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": ems / esteps,
               "how": f"host wall clock; per step all {len(chain.dats)} dats uploaded from pinned memory and "
                      f"the {round(bo / bi * len(chain.dats))} the step writes fetched back; steps rotate over 3 "
                      "contexts so copies overlap compute",
               "sequential_one_context": {"value": U * 3 / (sms * 1e-3) / 1e9, "ms_per_step": sms / 3}}

    # roofline of the dominant kernel: the step's kernels (one per loop
    # untiled, one persistent launch tiled), per launch.  Per-kernel events
    # serialise launches that otherwise overlap (programmatic dependent
    # launch), so the kernel time is capped by the step's own time.
    step_ms = ms / args.steps
    kernel_ms_step = min(kms / max(1, args.steps), step_ms)
    launches_per_step = kl / max(1, args.steps)
    kernel_ms_per_launch = kernel_ms_step / max(1.0, launches_per_step)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if probe and probe.get("fp64_fma_tflops"):
        peak_tflops = probe["fp64_fma_tflops"]
        peak_source = ("FP64: measured by ops_probe_device on this GPU (every SM issuing independent DFMA "
                       "chains, 2 flop each)")
    else:
        peak_tflops = NUM_SMS * FP64_DFMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12
        peak_source = f"FP64: {NUM_SMS} SMs x {FP64_DFMA_PER_CLK_SM} DFMA/clk x 2 flop x {sm_max:.0f} MHz (no probe)"
    flops_per_launch = flops / max(1.0, launches_per_step)
    achieved = flops_per_launch / (kernel_ms_per_launch * 1e-3) / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = profile_traffic(chosen_mode, chosen_tile) if args.n == N_DEFAULT else None
    kernel_name = {"wavefront": "wf: the wavefront kernel, one launch per step",
                   "tilewave": "tw: the tile-wavefront kernel, one launch per step"}.get(
        chosen_mode, "u<i>: the loop bodies compiled from the IR, one kernel per loop, averaged over the step's "
                     "launches" if st and st.get("compiled") else "k_untiled")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic, "kernel": kernel_name,
                "peak_source": peak_source, "kernel_ms_per_launch": kernel_ms_per_launch,
                "kernel_time": "per-kernel CUDA events on the launching stream, capped by the step time",
                "algorithmic_flops_per_launch": flops_per_launch,
                "algorithmic_bytes_per_launch": U / max(1.0, launches_per_step),
                "effective_hbm_frac": (U / max(1.0, launches_per_step)) / (kernel_ms_per_launch * 1e-3) / 1e9 / hbm_peak,
                "hbm_peak_gbs": hbm_peak}
    if traffic is not None:
        roofline["dram_gbs"] = traffic / (kernel_ms_per_launch * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.n)
    cg = bench_cg() if rank == 0 and not args.no_cg else None
    chain3d = bench_opensbli3d(stream, torch) if rank == 0 and not args.no_3d else None
    hydro3d = bench_cloverleaf3d(stream, torch) if rank == 0 and not args.no_3d else None
    ppcg = bench_ppcg(stream, torch) if rank == 0 and not args.no_3d else None
    fp32 = bench_fp32(stream, torch) if rank == 0 and not args.no_3d else None
    jacobi = bench_jacobi(stream, torch) if rank == 0 and not args.no_3d else None
    serving = bench_serving(args.serve_requests) if rank == 0 and not args.no_serve else None
    batch = None
    if rank == 0 and not args.no_batch:
        batch = {"cloverleaf2d_256": bench_batch(torch, W.cloverleaf2d(n=256, steps=1)),
                 "small2d_256": bench_batch(torch, W.small2d(n=256, reps=10)),
                 "opensbli3d_32": bench_batch(torch, W.opensbli3d(n=32, steps=1))}

    line = {"metric": "loop-chain effective GB/s", "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.n), "mode": args.mode, "schedule": chosen_mode,
                       "tile": st["tile"] if st else None,
                       "tiles": st["tiles"] if st else None, "l2": "inputs larger than L2 (25 dats, 3.0 GB)",
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "untiled_bytes_per_step": U, "flops_per_step": flops},
            "speedup_vs_untiled": (untiled["ms_per_step"] / (ms / args.steps)) if untiled else None,
            "untiled": untiled, "tilewave": tilewave, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk.summary(),
            "cg_4000": cg, "serving": serving, "batch": batch, "opensbli3d_320": chain3d, "cloverleaf3d_330": hydro3d, "ppcg_4000": ppcg, "cloverleaf2d_3840_fp32": fp32, "jacobi2d_8192_fp32": jacobi,
            "plan": {"phases": st["phases"], "barriers": st["barriers"], "skew": st["skew"],
                     "plan_ms_first_flush": first.get("plan_ms"), "compile_ms_first_flush": first.get("compile_ms"),
                     "plan_cache_hits": st["plan_cache_hits"]} if st else None,
            "probe": probe}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
