#!/usr/bin/env python
"""Benchmark: noise-source solves per second at a true relative residual of
1e-10, and the HBM bandwidth of the clover dslash, on one GB300 per rank.

One step = the whole hot path on one batch of synthetic input: gauge-field
layout conversion (sq_load_gauge), FP64 clover build and inversion
(sq_build_clover), the batched mixed-precision even-odd BiCGStab solve of
all sources (sq_solve: FP32 dslash, FP64 reliable updates) with its fused
pion-contraction epilogue (the sq_contract_pion kernel, run by sq_solve
while its final FP64 residual check is in flight). Workload: 16^3 x 32 lattice, antiperiodic
time, eps = 0.25 SU(3) links, c_sw = 1.0, kappa = 0.120, 16 Z4 sources.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank solves its own sources (weak scaling, replicas:
the solve has no exchange step); value = all ranks' sources / max time.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "clover dslash HBM GB/s; noise-source solves/sec at 1e-10 rel. residual vs FP64"
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 (FMA = 2 flops); the FP64 operator is bound by it
WORKLOAD = "16x16x16x32"
TOL = 1e-10
UNIT = "sources/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="stochq", choices=["stochq", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--inner", default="f32", choices=["f16", "f32", "f64"])
    p.add_argument("--delta", type=float, default=0.0, help="<= 0: library default")
    p.add_argument("--extras", type=int, default=1, help="FP64/FP16 comparison solves")
    p.add_argument("--e2e", type=int, default=1, help="end-to-end host-buffer measurement")
    p.add_argument("--cpu", type=int, default=1, help="CPU oracle baseline")
    p.add_argument("--workloads", type=int, default=1,
                   help="also time the 24^3x48, 32^3x64 and batch workloads and their dslash rooflines")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    """Max of a per-rank scalar over all ranks (the slowest rank times the
    whole job). Uses a device tensor under NCCL and a host tensor under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_local: int, world: int, max_ms: float) -> float:
    """Whole-job sources/s: every rank solves n_local sources per step and
    the step takes as long as the slowest rank."""
    return n_local * world / (max_ms / 1000.0)


def tensor_peak():
    """Dense bf16 burst TFLOP/s of MEASURED_PEAKS.json (FP16 runs at the same
    nominal rate), else the fallback measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"])
    return 1900.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_sha():
    h = hashlib.sha256()
    for f in ["sq_dslash.cu", "sq_device.cuh", "sq_solver_dev.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_1405_4524_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, workload):
    """DRAM bytes per launch of the kernel from the committed ncu summary,
    or None if there is none or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel_class}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != source_sha():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampler during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.p = None
        self.path = os.path.join("/tmp", f"sq_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        # let the sampler finish starting up (its first query) before the
        # timed region begins
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.p.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != self.index:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        loaded = [x for x in sm if x > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


_ORACLE_CACHE = {}


def _oracle_sample(workload, seconds_budget, k=0):
    """Seconds per BiCGStab iteration of the FP64 oracle as it stands on
    source k of the workload, from about `seconds_budget` seconds of whole
    iterations; returns (seconds per iteration, iterations timed, seconds).
    The links and their field strength are built once per process."""
    import oracle
    from paper_1405_4524_gb300 import inputs

    if workload not in _ORACLE_CACHE:
        spec = dict(inputs.WORKLOADS[workload])
        U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
        _ORACLE_CACHE[workload] = (spec, U, oracle.field_strength(U))
    spec, U, F = _ORACLE_CACHE[workload]
    T = spec["dims"][3]
    # source k of the workload (source k draws from seed + k)
    eta = inputs.make_z4(spec["dims"], 1, spec["src_seed"] + k, [k % T] if spec["diluted"] else None)[0]
    apply = lambda v: oracle.apply_M(U, F, v, spec["kappa"], spec["csw"], -1.0)
    t0 = time.perf_counter()
    apply(eta)
    t_apply = time.perf_counter() - t0
    # bicgstab(maxiter=m) costs 2m operator applications plus one for the
    # initial and one for the final residual: m + 1 iteration equivalents
    m = int(max(1, min(40, seconds_budget / (2.0 * t_apply) - 1)))
    t0 = time.perf_counter()
    oracle.bicgstab(apply, eta, tol=1e-300, maxiter=m)
    el = time.perf_counter() - t0
    return el / (m + 1), m, el


def _oracle_worker(job):
    workload, budget, k = job
    return _oracle_sample(workload, budget, k)


class OraclePool:
    """One oracle process per host core (spawned, so none is forked from a
    process that has used the GPU). Each runs the oracle on its own source of
    the workload, sources k = 0 .. n-1 dealt round-robin to the cores."""

    def __init__(self):
        import concurrent.futures as cf
        import multiprocessing as mp

        self.cores = os.cpu_count() or 1
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        self.ex = cf.ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"))

    def sample(self, workload, n_src, budget):
        """Sources/s of the oracle over all cores: one source of the workload
        per core (sources 0 .. min(n_src, cores) - 1, a bounded sample of the
        n_src-source workload), each its measured seconds per iteration times
        the iterations the oracle needs for 1e-10
        (tests/golden/oracle_iterations.json); the cores run concurrently.
        Returns (sources/s, wall seconds, sources timed, iterations)."""
        gold = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")))[workload]
        m = min(n_src, self.cores)
        t0 = time.perf_counter()
        res = list(self.ex.map(_oracle_worker, [(workload, budget, k) for k in range(m)]))
        wall = time.perf_counter() - t0
        return sum(1.0 / (per_it * gold["iterations"]) for per_it, _, _ in res), wall, m, gold["iterations"]

    def close(self):
        self.ex.shutdown()


def cpu_baseline(workload, n_src, seconds_budget=10.0):
    """The FP64 oracle as it stands on the host cores: all cores, one source
    per core (the reported value); one core; and one full, non-extrapolated
    oracle solve of the small 4^3 x 8 workload (4 sources to 1e-12)."""
    import oracle
    from paper_1405_4524_gb300 import inputs

    pool = OraclePool()
    try:
        value, wall, m_src, iters = pool.sample(workload, n_src, seconds_budget)
    finally:
        pool.close()
    per_it, m, el = _oracle_sample(workload, seconds_budget, 0)
    spec, U, eta = inputs.workload("4x4x4x8")
    F = oracle.field_strength(U)
    t0 = time.perf_counter()
    for k in range(spec["n_rhs"]):
        oracle.solve(U, eta[k], spec["kappa"], spec["csw"], -1.0, tol=1e-12, F=F)
    full = time.perf_counter() - t0
    cpu = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                cpu = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": (f"{m_src} of the {n_src} sources of {workload}, one oracle process per host core "
                       f"({pool.cores} cores, {cpu or 'cpu model unknown'}): each times whole BiCGStab "
                       f"iterations of its own source for about {seconds_budget:.0f} s, scaled to the {iters} "
                       f"iterations the oracle needs for 1e-10 (tests/golden/oracle_iterations.json); "
                       f"{wall:.1f} s wall"),
            "one_core": {"value": 1.0 / (per_it * iters), "unit": UNIT, "cores": 1,
                         "sample": f"1 source, {m} iterations in {el:.1f} s, scaled to {iters}"},
            "full_solve_4x4x4x8": {"value": spec["n_rhs"] / full, "unit": UNIT, "cores": 1,
                                   "sample": f"4 sources of 4x4x4x8 solved to 1e-12 by the oracle, {full:.2f} s "
                                             f"(measured, not extrapolated)"}}


def dslash_roofline(sq, ctx, dims, prec, n, reps=10):
    """The clover dslash (hop + A^-1) on n sources of precision prec at the
    autotuned shape, timed alone with CUDA events on the caller's stream
    (the library orders its own stream between them). Algorithmic bytes per
    launch: links and clover blocks once, every source's input and output
    spinor once (FP32 96 + 96 B, FP16 52 + 52 B per site and source)."""
    import torch

    X, Y, Z, T = dims
    fb = sq.sq_field_bytes(ctx, prec, n)
    bi = torch.zeros(fb, dtype=torch.uint8, device="cuda")
    bo = torch.zeros(fb, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(5)
    psi = torch.randn((n, T, Z, Y, X, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
    sq.sq_pack_spinor(ctx, bi, psi, 1, prec, n)
    del psi
    flags = sq.SQ_DS_CLOVER_INV
    sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, n, flags | sq.SQ_DS_SYNC, 0.0)  # tunes the shape
    kind, shape = sq.sq_get_dslash_shape(ctx, prec, n)
    for _ in range(3):
        sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, n, flags, 0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        sq.sq_dslash_eo(ctx, bo, bi, None, 0, prec, n, flags, 0.0)
    e1.record()
    torch.cuda.synchronize()
    us = 1000.0 * e0.elapsed_time(e1) / reps
    vh = X * Y * Z * T // 2
    per_src = 192 if prec == sq.SQ_F32 else 104
    bytes_ = vh * (8 * 48 + 288 + n * per_src)
    hbm, how = peaks()
    gbs = bytes_ / (us * 1e-6) / 1e9
    del bi, bo
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
            "traffic": None, "kernel": f"dslash_clover ({'f32' if prec == sq.SQ_F32 else 'f16'}, recon-12, "
                                       f"{n} sources, {'tiled' if kind == 1 else 'per-site'} shape {list(shape)})",
            "bytes_per_launch": bytes_, "us_per_launch": round(us, 2),
            "peak_kind": f"{how} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}


def other_workloads(sq):
    """The large workloads, device-resident inputs, tol 1e-10: one timed
    solve each after a warm-up solve (24^3 x 48, 64 time-diluted sources,
    FP16 inner; 32^3 x 64, 24 sources, FP16 defect correction), the clover
    dslash timed alone at both sizes (FP16, and FP32 at 32^3 x 64), and the
    96-source batch over two lattices and three kappas."""
    import torch

    from paper_1405_4524_gb300 import inputs

    out = {}
    links = {}

    def timed_solve(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st

    for name, prm in [("24x24x24x48", sq.sq_default_params(inner_prec=sq.SQ_F16)),
                      ("32x32x32x64", sq.sq_default_params(inner_prec=sq.SQ_F16, outer=sq.SQ_OUTER_DEFECT))]:
        spec, U, eta = inputs.workload(name)
        links[name] = U
        ctx = sq.sq_create(spec["dims"], -1)
        sq.sq_load_gauge(ctx, U, 12)
        e = torch.from_numpy(eta).cuda()
        del eta
        x = torch.zeros_like(e)
        dt, (_, st) = timed_solve(lambda: sq.sq_solve(ctx, spec["kappa"], spec["csw"], e, x, spec["n_rhs"], TOL, prm))
        out[name] = {"sources_per_s": round(spec["n_rhs"] / dt, 2), "n_sources": spec["n_rhs"],
                     "iterations": int(np.mean([s["iterations"] for s in st])),
                     "max_true_residual": max(s["true_residual"] for s in st),
                     "solver": "FP16 inner, " + ("defect correction" if prm.outer else "reliable updates")}
        del e, x
        sq.sq_build_clover(ctx, spec["kappa"], spec["csw"])
        out[name]["roofline_dslash_f16"] = dslash_roofline(sq, ctx, spec["dims"], sq.SQ_F16, spec["n_rhs"])
        if name == "32x32x32x64":
            out[name]["roofline_dslash_f32"] = dslash_roofline(sq, ctx, spec["dims"], sq.SQ_F32, spec["n_rhs"])
        sq.sq_destroy(ctx)
    # 96 sources: 16^3x32 and 24^3x48 at kappa 0.118, 0.121, 0.124 in one batch
    ctxs, probs, bufs = [], [], []
    for gi, name in enumerate(["16x16x16x32", "24x24x24x48"]):
        spec = inputs.WORKLOADS[name]
        ctx = sq.sq_create(spec["dims"], -1)
        U = links.get(name)
        if U is None:
            U = inputs.make_links(spec["dims"], spec["eps"], spec["link_seed"])
        sq.sq_load_gauge(ctx, U, 12)
        ctxs.append(ctx)
        for ki, kappa in enumerate([0.118, 0.121, 0.124]):
            e = torch.from_numpy(inputs.make_z4(spec["dims"], 16, 3000 + 10 * gi + ki)).cuda()
            x = torch.zeros_like(e)
            bufs += [e, x]
            probs.append(dict(ctx=ctx, kappa=kappa, c_sw=1.0, sources=e, solutions=x, n_rhs=16, tol=TOL))
    prm = sq.sq_default_params(inner_prec=sq.SQ_F16)
    dt, (_, st) = timed_solve(lambda: sq.sq_solve_batch(probs, prm))
    out["batch_96_two_lattices_three_kappas"] = {
        "sources_per_s": round(96 / dt, 2), "max_true_residual": max(s["true_residual"] for s in st),
        "iterations_min_max": [int(min(s["iterations"] for s in st)), int(max(s["iterations"] for s in st))]}
    del bufs
    for ctx in ctxs:
        sq.sq_destroy(ctx)
    return out


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_1405_4524_gb300 import inputs

    steps, warm = args.steps, args.warmup
    n_src = inputs.WORKLOADS[args.workload]["n_rhs"]
    budget = max(1.0, 120.0 / max(1, steps + warm))
    pool = OraclePool()
    try:
        for _ in range(warm):
            pool.sample(args.workload, n_src, budget / 2)
        vals, walls = [], []
        t0 = time.perf_counter()
        for _ in range(steps):
            v, w, m_src, iters = pool.sample(args.workload, n_src, budget)
            vals.append(v)
            walls.append(w)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    value = statistics.median(vals)
    sample = (f"{m_src} of the {n_src} sources of {args.workload}, one oracle process per host core "
              f"({pool.cores} cores): each step times whole BiCGStab iterations of each core's source for "
              f"about {budget:.1f} s, scaled to the {iters} iterations the oracle needs for 1e-10")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warm, "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "n_sources": n_src, "tol": TOL,
                       "solver": "oracle: unpreconditioned FP64 BiCGStab (numpy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ms_per_source": 1000.0 / value,
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1405_4524_gb300 import inputs, stochq as sq

    spec = inputs.WORKLOADS[args.workload]
    dims, n = spec["dims"], spec["n_rhs"]
    kappa, csw = spec["kappa"], spec["csw"]
    U = inputs.make_links(dims, spec["eps"], spec["link_seed"])
    T = dims[3]
    ts = [k % T for k in range(n)] if spec["diluted"] else None
    eta = inputs.make_z4(dims, n, spec["src_seed"] + 100000 * rank, ts)
    inner = {"f64": sq.SQ_F64, "f32": sq.SQ_F32, "f16": sq.SQ_F16}[args.inner]

    stream = torch.cuda.Stream()
    ctx = sq.sq_create(dims, -1, stream)
    U_dev = torch.from_numpy(U).cuda()
    eta_dev = torch.from_numpy(eta).cuda()
    sol_dev = torch.zeros_like(eta_dev)
    pinned = [torch.from_numpy(U).pin_memory(), torch.from_numpy(eta).pin_memory(),
              torch.zeros(eta.shape, dtype=torch.complex128).pin_memory()]
    U_pin, eta_pin, sol_pin = (t.numpy() for t in pinned)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # timed steps carry event nodes around the two clover dslash launches of
    # every iteration only (the roofline kernel); the per-kernel breakdown
    # comes from separate, untimed steps with events around every kernel
    prm = sq.sq_default_params(inner_prec=inner, delta=args.delta, profile=2)
    prm_all = sq.sq_default_params(inner_prec=inner, delta=args.delta, profile=1)
    prm_e2e = sq.sq_default_params(inner_prec=inner, delta=args.delta)

    last = {}

    # the pion correlator is the solve's fused epilogue (sq_solve_params.pion)
    ts_np = np.array(ts if ts is not None else [0] * n, dtype=np.int32)
    ts_dev = torch.from_numpy(ts_np).cuda()
    C_dev = torch.zeros((n, T), dtype=torch.float64, device="cuda")
    C_pin = torch.zeros((n, T), dtype=torch.float64).pin_memory().numpy()

    def step_device(p=prm):
        sq.sq_load_gauge(ctx, U_dev, 12)
        sq.sq_build_clover(ctx, kappa, csw)
        _, st = sq.sq_solve(ctx, kappa, csw, eta_dev, sol_dev, n, TOL, p, pion=C_dev, pion_tslice=ts_dev)
        last["stats"] = st

    def step_e2e():
        sq.sq_load_gauge(ctx, U_pin, 12)
        sq.sq_build_clover(ctx, kappa, csw)
        _, st = sq.sq_solve(ctx, kappa, csw, eta_pin, sol_pin, n, TOL, prm_e2e, pion=C_pin, pion_tslice=ts_np)
        last["stats_e2e"] = st

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(step, k, prof=False):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        agg = {}
        barrier()
        torch.cuda.synchronize()
        l0 = sq.sq_kernel_launches(ctx)
        w0 = time.perf_counter()
        for i in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[i][0].record(stream)
            torch.cuda.nvtx.range_push("timed_step")
            step()
            torch.cuda.nvtx.range_pop()
            ev[i][1].record(stream)
            if prof:
                for row in sq.sq_get_profile(ctx):
                    a = agg.setdefault(row["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
                    for f in ("launches", "ms", "bytes", "flops"):
                        a[f] += row[f]
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier()
        launches = sq.sq_kernel_launches(ctx) - l0
        per = [a.elapsed_time(b) for a, b in ev]
        last["step_ms"] = per
        ms = reduce_max(sum(per) / k, world)
        return ms, wall, launches, agg

    for _ in range(max(3, args.warmup)):
        step_device()
    clocks = Clocks(local)
    clocks.start()
    ms, wall, launches, agg = timed(step_device, args.steps, prof=True)
    clk = clocks.stop()
    stats = last["stats"]
    step_ms = last["step_ms"]
    assert all(s["status"] == 0 and s["true_residual"] <= TOL for s in stats), stats
    value = job_throughput(n, world, ms)

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if args.e2e:
        for _ in range(2):
            step_e2e()
        ms_e2e, _, _, _ = timed(step_e2e, max(2, args.steps // 2))
        assert all(s["status"] == 0 and s["true_residual"] <= TOL for s in last["stats_e2e"])
        h2d = U.nbytes + eta.nbytes + ts_np.nbytes  # links, sources, source time slices
        d2h = eta.nbytes + C_pin.nbytes  # solutions, correlator
        e2e = {"value": round(job_throughput(n, world, ms_e2e), 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ms_e2e, 3)}

    # roofline kernel: the clover dslash D + A^-1 (two launches per iteration;
    # the fused-reduction variants differ only in their epilogue)
    top = "dslash_clover"
    d = agg[top]
    hbm, how = peaks()
    achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9
    traffic = ncu_traffic(f"{top}_{args.inner}", args.workload)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic,
                "kernel": f"{top} ({args.inner}, recon-12, {n} sources per launch)",
                "bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "us_per_launch": 1000.0 * d["ms"] / max(1, d["launches"]),
                "peak_kind": f"{how} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}
    for _ in range(2):
        step_device(prm_all)
    _, _, _, agg_all = timed(lambda: step_device(prm_all), 2, prof=True)
    tot_ms = sum(v["ms"] for v in agg_all.values())
    breakdown = {k: {"share": round(v["ms"] / tot_ms, 4),
                     "GB/s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                     "us_per_launch": round(1000.0 * v["ms"] / max(1, v["launches"]), 2)}
                 for k, v in agg_all.items()}

    extras = {}
    if args.extras and rank == 0:
        # the plain FP64 even-odd GPU solver and the FP16-inner solver on the same workload
        for name, p in [("fp64_solver", sq.sq_default_params(inner_prec=sq.SQ_F64)),
                        ("fp16_inner_solver", sq.sq_default_params(inner_prec=sq.SQ_F16, delta=args.delta))]:
            sol2 = torch.zeros_like(eta_dev)
            try:
                sq.sq_solve(ctx, kappa, csw, eta_dev, sol2, n, TOL, p)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st2 = sq.sq_solve(ctx, kappa, csw, eta_dev, sol2, n, TOL, p)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                extras[name] = {"sources_per_s": round(n / dt, 2),
                                "iterations": int(np.mean([s["iterations"] for s in st2])),
                                "fp64_updates": int(np.mean([s["updates"] for s in st2])),
                                "max_true_residual": max(s["true_residual"] for s in st2)}
            except sq.StochqError as e:
                extras[name] = {"error": str(e)}
            del sol2
        if "sources_per_s" in extras["fp64_solver"]:
            extras["speedup_vs_fp64_solver"] = round(value / world / extras["fp64_solver"]["sources_per_s"], 2)
        # the FP64 operator alone (hop + A^-1 + xpay on all sources): bound
        # by the FP64 pipe; CUDA events on the library's ordering stream
        fb = sq.sq_field_bytes(ctx, sq.SQ_F64, n)
        bi, bo, bx = (torch.zeros(fb, dtype=torch.uint8, device="cuda") for _ in range(3))
        flags = sq.SQ_DS_CLOVER_INV | sq.SQ_DS_XPAY
        for _ in range(2):
            sq.sq_dslash_eo(ctx, bo, bi, bx, 0, sq.SQ_F64, n, flags, -kappa * kappa)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            sq.sq_dslash_eo(ctx, bo, bi, bx, 0, sq.SQ_F64, n, flags, -kappa * kappa)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / reps
        vh = int(np.prod(dims)) // 2
        tflops = n * vh * (1320 + 504 + 48) / (ms64 / 1000.0) / 1e12
        extras["fp64_operator"] = {"bound": "alu", "achieved": round(tflops, 3), "peak": FP64_PEAK_TFLOPS,
                                   "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                                   "us_per_launch": round(1000.0 * ms64, 1),
                                   "flops_per_site_source": 1320 + 504 + 48,
                                   "peak_kind": "GB300 nominal FP64 rate (an FMA-loop probe measured the same)"}
        del bi, bo, bx
        # the stochastic operators O_ij(t) of all source pairs and their
        # correlator from the sources and the solutions (Eq. stoop): bound by
        # the FP64 pipe, three FMAs per complex term (t, i, j, row)
        O_dev = torch.zeros((T, n, n), dtype=torch.complex128, device="cuda")
        Cs_dev = torch.zeros(T, dtype=torch.complex128, device="cuda")
        for _ in range(2):
            sq.sq_contract_stoch_op(ctx, eta_dev, sol_dev, n, O_dev, Cs_dev)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_contract_stoch_op(ctx, eta_dev, sol_dev, n, O_dev, Cs_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_so = e0.elapsed_time(e1) / reps
        terms = float(n) * n * int(np.prod(dims)) * 12
        tflops = 6.0 * terms / (ms_so / 1000.0) / 1e12
        extras["stoch_op"] = {"bound": "alu", "achieved": round(tflops, 3), "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                              "us_per_call": round(1000.0 * ms_so, 1), "pairs": n * n,
                              "complex_terms_per_s": round(terms / (ms_so / 1000.0), 1),
                              "flops_per_term": 6,
                              "note": "device I/O, operators and correlator; 3 FP64 FMAs per complex term"}
        # the trace of the filled stochastic propagators (Eq. Sfill, Table Lcomp's
        # sum_x sum_z tr S S^dag for every source and sink timeslice) through
        # two Gram matrices per timeslice instead of the fill: FP64-pipe bound
        Cp_dev = torch.zeros((T, T), dtype=torch.complex128, device="cuda")
        for _ in range(2):
            sq.sq_contract_prop_trace(ctx, eta_dev, sol_dev, n, C=Cp_dev)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_contract_prop_trace(ctx, eta_dev, sol_dev, n, C=Cp_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_pt = e0.elapsed_time(e1) / reps
        tflops = 2 * 6.0 * terms / (ms_pt / 1000.0) / 1e12
        fill_cmul = 144.0 * (int(np.prod(dims[:3])) ** 2) * T * T * n  # complex multiplies of the fill route
        extras["prop_trace"] = {"bound": "alu", "achieved": round(tflops, 3), "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                                "us_per_call": round(1000.0 * ms_pt, 1), "source_sets": 1,
                                "fill_route_complex_multiplies": fill_cmul,
                                "note": "device I/O; C[t0][t] for all T^2 pairs from two Gram matrices per "
                                        "timeslice, 3 FP64 FMAs per complex term"}
        # the same operators on the tensor cores (exact digit split, sources
        # with components 0 or +-1) at the bench size, and at the paper's
        # N_r = 10^3 regime (Sec. "Stochastic propagators": 10^3 noise sources
        # on the L = 8 lattice): 8^3 x 16 with 1024 Z4 sources, Gaussian X
        # (the time does not depend on the values)
        O_dev = torch.zeros((T, n, n), dtype=torch.complex128, device="cuda")
        sq.sq_contract_stoch_op(ctx, eta_dev, sol_dev, n, O_dev, Cs_dev, tensor_cores=True)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_contract_stoch_op(ctx, eta_dev, sol_dev, n, O_dev, Cs_dev, tensor_cores=True)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["stoch_op"]["tensor_core_route_us_per_call"] = round(1000.0 * e0.elapsed_time(e1) / reps, 1)
        dims_tc, n_tc = (8, 8, 8, 16), 1024
        T_tc = dims_tc[3]
        ctx_tc = sq.sq_create(dims_tc, -1, stream)
        eta_tc = torch.from_numpy(inputs.make_z4(dims_tc, n_tc, 7001)).cuda()
        X_tc = torch.from_numpy(inputs.make_gaussian_spinors(dims_tc, n_tc, 8001)).cuda()
        O_tc = torch.zeros((T_tc, n_tc, n_tc), dtype=torch.complex128, device="cuda")
        C_tc = torch.zeros(T_tc, dtype=torch.complex128, device="cuda")
        sq.sq_contract_stoch_op(ctx_tc, eta_tc, X_tc, n_tc, O_tc, C_tc, tensor_cores=True)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_contract_stoch_op(ctx_tc, eta_tc, X_tc, n_tc, O_tc, C_tc, tensor_cores=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_tc = e0.elapsed_time(e1) / reps
        e0.record(stream)
        sq.sq_contract_stoch_op(ctx_tc, eta_tc, X_tc, n_tc, O_tc, C_tc)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_tc64 = e0.elapsed_time(e1)
        terms_tc = float(n_tc) * n_tc * int(np.prod(dims_tc)) * 12
        bf16_peak = tensor_peak()
        tflops = 40.0 * terms_tc / (ms_tc / 1000.0) / 1e12
        extras["stoch_op_tc"] = {"bound": "tensor", "achieved": round(tflops, 1), "peak": bf16_peak,
                                 "unit": "TFLOP/s", "frac": round(tflops / bf16_peak, 4),
                                 "workload": "8x8x8x16, 1024 Z4 sources, operators + correlator, device I/O",
                                 "ms_per_call": round(ms_tc, 3), "fp64_route_ms": round(ms_tc64, 2),
                                 "speedup_vs_fp64_route": round(ms_tc64 / ms_tc, 1),
                                 "complex_terms_per_s": round(terms_tc / (ms_tc / 1000.0), 1),
                                 "flops_per_term": 40,
                                 "method_flops_per_term": 8,
                                 "frac_method_flops": round(8.0 * terms_tc / (ms_tc / 1000.0) / 1e12 / bf16_peak, 4),
                                 "note": "FP16 x FP16 -> FP32 tcgen05 products of 5 exact 11-bit digits of "
                                         "gamma5 X (real and imaginary rows) against ternary sources; whole "
                                         "call (packing, products, FP64 digit sums, correlator) against the "
                                         "measured dense bf16 burst peak (FP16 has the same nominal rate)"}
        sq.sq_destroy(ctx_tc)
        del O_dev, Cs_dev, Cp_dev, eta_tc, X_tc, O_tc, C_tc
        # full (time-spin-colour) dilution of one Z4 noise vector on 8^3 x 16:
        # 192 sources made on the device and solved in one batch
        dims_d = (8, 8, 8, 16)
        ctx_d = sq.sq_create(dims_d, -1, stream)
        sq.sq_load_gauge(ctx_d, torch.from_numpy(inputs.make_links(dims_d, 0.25, 1005)).cuda(), 12)
        noise_d = torch.from_numpy(inputs.make_z4(dims_d, 1, 2005)).cuda()
        src_d = sq.sq_dilute(ctx_d, noise_d, 1, sq.SQ_DILUTE_FULL)
        n_d = src_d.shape[0]
        sol_d = torch.zeros_like(src_d)
        prm_d = sq.sq_default_params(inner_prec=inner)
        sq.sq_solve(ctx_d, 0.12, 1.0, src_d, sol_d, n_d, TOL, prm_d)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_dilute(ctx_d, noise_d, 1, sq.SQ_DILUTE_FULL, out=src_d)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_dil = e0.elapsed_time(e1) / reps
        sol_d.zero_()
        e0.record(stream)
        _, st_d = sq.sq_solve(ctx_d, 0.12, 1.0, src_d, sol_d, n_d, TOL, prm_d)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_sd = e0.elapsed_time(e1)
        extras["full_dilution"] = {"workload": "8x8x8x16, 1 Z4 noise vector -> 192 sources (time-spin-colour)",
                                   "dilute_us": round(1000.0 * ms_dil, 1),
                                   "dilute_gb_s": round(n_d * int(np.prod(dims_d)) * 12 * 16 / (ms_dil / 1000.0) / 1e9, 1),
                                   "solve_ms": round(ms_sd, 2), "sources_per_s": round(n_d / (ms_sd / 1000.0), 1),
                                   "iterations": int(np.mean([x["iterations"] for x in st_d])),
                                   "max_true_residual": max(x["true_residual"] for x in st_d)}
        sq.sq_destroy(ctx_d)
        del noise_d, src_d, sol_d
        # the four diagrams at zero momentum (Sec. "Stochastic propagators",
        # Sec. "Correlation function") on the bench lattice: the twelve
        # point solutions of the origin, set A = the bench's own 16 sources
        # and solutions, set B = 16 more sources; FP64-pipe bound (Gram
        # matrices of the two sets, of the point and noise solutions)
        one = torch.zeros((1,) + tuple(eta_dev.shape[1:]), dtype=torch.complex128, device="cuda")
        one[0, 0, 0, 0, 0] = 1.0
        src_p = sq.sq_dilute(ctx, one, 1, sq.SQ_DILUTE_SPIN_COLOUR)
        Xp = torch.zeros_like(src_p)
        sq.sq_solve(ctx, kappa, csw, src_p, Xp, 12, TOL, sq.sq_default_params(inner_prec=inner))
        eB = torch.from_numpy(inputs.make_z4(dims, n, spec["src_seed"] + 500000)).cuda()
        xB = torch.zeros_like(eB)
        sq.sq_solve(ctx, kappa, csw, eB, xB, n, TOL, sq.sq_default_params(inner_prec=inner))
        Dg = sq.sq_contract_diagrams(ctx, Xp, eta_dev, sol_dev, n, eB, xB)
        e0.record(stream)
        for _ in range(reps):
            sq.sq_contract_diagrams(ctx, Xp, eta_dev, sol_dev, n, eB, xB, out=Dg)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_dg = e0.elapsed_time(e1) / reps
        vol = float(np.prod(dims)) * 12
        terms_dg = 2.0 * n * n * vol + 2.0 * 12 * n * vol  # complex terms of the Gram matrices
        tflops = 6.0 * terms_dg / (ms_dg / 1000.0) / 1e12
        extras["diagrams"] = {"bound": "alu", "achieved": round(tflops, 3), "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                              "ms_per_call": round(ms_dg, 3),
                              "workload": f"{WORKLOAD}: 12 point solutions, two sets of {n} Z4 sources",
                              "C0_plus_C1_minus_C2_minus_C3_at_t1": float((Dg[3, 1] + Dg[4, 1] - Dg[5, 1]
                                                                            - Dg[6, 1]).real),
                              "note": "device I/O; P, Q0, Qtt, C0..C3 per sink timeslice; 3 FP64 FMAs per "
                                      "complex term of the Gram matrices (noise-noise and point-noise)"}
        del one, src_p, Xp, eB, xB, Dg

    if args.workloads and rank == 0:
        extras["workloads"] = other_workloads(sq)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms, 3),
        "step_ms_min_median_max": [round(min(step_ms), 3), round(statistics.median(step_ms), 3),
                                   round(max(step_ms), 3)],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16", "f64": "f64"}[args.inner], "data": "synthetic",
        "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "t_bc": "antiperiodic",
                   "kappa": kappa, "c_sw": csw, "link_eps": spec["eps"], "sources_per_gpu": n,
                   "noise": "Z4" + (" time-diluted" if spec["diluted"] else ""), "tol": TOL,
                   "solver": f"even-odd BiCGStab, {args.inner} inner, FP64 reliable updates (delta={args.delta or 'auto'})",
                   "step": "load_gauge + build_clover + solve (fused pion epilogue)",
                   "l2": "256 MB flush between timed steps; working set > L2",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clk,
        "iterations": int(np.mean([s["iterations"] for s in stats])),
        "fp64_updates": int(np.mean([s["updates"] for s in stats])),
        "max_true_residual": max(s["true_residual"] for s in stats),
        "kernel_breakdown": breakdown,
        "extras": extras,
    }
    if rank == 0 and world == 1 and args.cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload, n)
    sq.sq_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
