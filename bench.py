"""Benchmark of the exact Voronoi RayCast on its exhaustive-traversal workload.

Workload (one step): node preparation + exhaustive vertex traversal
(Algorithm 2) of N = 20,000 iid uniform nodes in [0,1]^5 (seed 0), cells
clipped to the unit cube, on the library's default path (tensor-core
screening of the rays grouped by reference node, binary32 rescreen,
binary64 recheck).  The metric is raycasts per second of that traversal; the
same workload on the binary32-screened path and on the plain binary64 path
is timed beside it, and their vertex tuples must equal the default path's bit
for bit.

Secondary lines in the same JSON object: "mc" (MC volumes + areas + adjoint,
d=4, N=100,000, 1024 rays per cell; binary32-screened, tensor-core screened
and binary64 paths), "highd" (the same at d=16, N=200,000 mixture nodes,
64 rays per cell; tensor-core walk vs binary32 tree walk), "mc.integrals"
(Algorithm 3's function integrals on the d=4 rays), "hmc" (heuristic MC
integrals, Section 3.3, and the exact integration of Section 3.2 on the
traversal workload's diagram), "walk" (random walks on the vertex graph),
"cells" (the per-cell sequential exploration of Section 2.3 beside the
whole-diagram traversal: time and table memory), "plain_fp64_d3" (the plain binary64 method at d=3, N=2,000: traversal + MC
with 64 rays per cell + adjoint) and "batch" (512 point sets of uneven N and
d, 256 rays per cell).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank runs an independent
replica of the workload (the traversal of one node set does not shard);
`value` is all ranks' raycasts over the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload's rays.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "raycasts/s and MC vol+grad cells/s: mixed vs FP64 path, same GB300, exact hits"
WORKLOAD = "exhaustive vertex traversal, d=5, N=20000 iid uniform in [0,1]^5 (seed 0), clipped to the cube"
NEIGHBOURS_D5 = 95  # neighbours per cell in d = 5 (the paper's table of vertices and neighbours per cell)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, ncu) of one traversal's RayCast on the default path,
# every launch of k_grp_count, k_grp_alloc, k_grp_scatter, k_ray_list_tc, k_grp_finish and the tree-walk and
# binary64 follow-ups: 8964.0 MB over the three traversals of `python bench.py --steps 1 --warmup 1 --no-fp64
# --no-binary32 --no-cpu --no-mc --no-highd --no-hmc --no-walk --no-small --no-batch --no-cells`, captured with
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none -k
# "regex:k_ray_list_tc|k_grp_|k_ray_mixed|k_ray_fp64"` (list scan at 8 blocks per SM, lists of 1024 nodes).
# k_grp_scatter and k_grp_finish changed after that capture (the box-face zero and sign tests moved to the
# binary32 copy of u_a: arithmetic only, no load or store added or removed), so the line reports it as
# `traffic_last_capture` and `traffic` stays null until the counters are taken again.
RAYCAST_DRAM_BYTES_PER_STEP = 2988.0e6
RAYCAST_TRAFFIC_CURRENT = False


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce_over_ranks(x, ws, dist.ReduceOp.MAX)


def _sum_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce_over_ranks(x, ws, dist.ReduceOp.SUM)


def replica_value(units, seconds, ws):
    """Whole-job throughput of N independent replicas: every rank's units
    over the slowest rank's time (the replicas start together after a
    barrier)."""
    return _sum_over_ranks(units, ws) / _max_over_ranks(seconds, ws)


def edge_rays_from_mesh(orc, X, tuples, coords, n, seed=0):
    """Rays of Algorithm 2 (vertex origin, edge direction, eta) for n random
    (vertex, edge) pairs of a traversal result, built with the oracle."""
    rng = np.random.default_rng(seed)
    d = X.shape[1]
    O, U, E = [], [], []
    while len(O) < n:
        v = int(rng.integers(0, len(tuples)))
        drop = int(rng.integers(0, d + 1))
        sig = tuples[v]
        eta = [int(g) for q, g in enumerate(sig) if q != drop]
        nodes = sorted(g for g in eta if g >= 0)
        if not nodes:
            continue
        u = orc.search_direction(X, sig, drop)
        if u is None:
            continue
        O.append(coords[v])
        U.append(u)
        E.append([nodes[0]] + [g for g in eta if g != nodes[0]])
    return np.array(O), np.array(U), np.array(E, np.int32)


def cpu_oracle_rate(X, tuples, coords, target_s=15.0):
    """Oracle raycasts/s on the host cores over a bounded sample of the
    traversal's edge rays (about target_s seconds of CPU work), with every
    core and with one core (a sample a sixteenth the size)."""
    import oracle
    oracle.build()
    O, U, E = edge_rays_from_mesh(oracle, X, tuples, coords, 256, seed=1)
    t0 = time.perf_counter()
    oracle.raycast(X, O, U, E)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(200000, max(512, 256 * target_s / dt)))
    O, U, E = edge_rays_from_mesh(oracle, X, tuples, coords, n, seed=2)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.raycast(X, O, U, E)
    dt = time.perf_counter() - t0
    n1 = max(64, n // 16)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.raycast(X, O[:n1], U[:n1], E[:n1])
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return n / dt, n, dt, cores, n1 / dt1, n1, dt1


def run_reference(args):
    """The FP64 CPU oracle on the host cores: each step times its brute-force
    RayCast on a bounded sample of the workload's edge rays (from vertices the
    oracle itself finds by a bounded Algorithm 2 walk from its Descent seed)."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2405_10050_gb300 import synth
    oracle.build()
    X = synth.uniform(args.N, args.d, seed=0)
    tuples, coords = _oracle_local_vertices(oracle, X, 300)
    rates, secs = [], []
    for s in range(args.warmup + args.steps):
        O, U, E = edge_rays_from_mesh(oracle, X, tuples, coords, args.ref_rays, seed=100 + s)
        t0 = time.perf_counter()
        oracle.raycast(X, O, U, E)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            rates.append(len(O) / dt)
            secs.append(dt)
    value = statistics.mean(rates)
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "raycasts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": args.N, "d": args.d, "sample_rays_per_step": args.ref_rays},
            "cpu_baseline": {"value": value, "unit": "raycasts/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_rays} edge rays per step of the workload's diagram "
                                       f"(FP64 brute force over all {args.N} nodes)"},
            "e2e": {"value": value, "unit": "raycasts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_local_vertices(orc, X, nmax):
    """Up to nmax vertices of the diagram of X found by the oracle: Descent
    from node 0, then a breadth-first walk of Algorithm 2."""
    import collections
    d = X.shape[1]
    sig0 = orc.descent(X, 0)
    seen = {tuple(int(g) for g in sig0)}
    q = collections.deque([tuple(int(g) for g in sig0)])
    out_t, out_c = [], []
    while q and len(out_t) < nmax:
        sig = q.popleft()
        sa = np.array(sig, np.int32)
        r = orc.vertex_coords(X, sa)
        out_t.append(sig)
        out_c.append(r)
        for drop in range(d + 1):
            eta = [g for k, g in enumerate(sig) if k != drop]
            nodes = sorted(g for g in eta if g >= 0)
            if not nodes:
                continue
            u = orc.search_direction(X, sa, drop)
            if u is None:
                continue
            er = [nodes[0]] + [g for g in eta if g != nodes[0]]
            h, _ = orc.raycast(X, r[None], u[None], np.array([er], np.int32))
            ns = tuple(sorted(eta + [int(h[0])]))
            if ns not in seen:
                seen.add(ns)
                q.append(ns)
    return np.array(out_t, np.int32), np.array(out_c)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2405_10050_gb300 import VD_AUTO, VD_FP32, VD_FP64, synth, vd
    vd.load()
    if args.only_mc:  # the MC secondary measurement alone (profiling)
        print(json.dumps({"mc": run_mc(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    if args.only_highd:
        print(json.dumps({"highd": run_highd(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    if args.only_hmc:
        print(json.dumps({"hmc": run_hmc(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    if args.only_walk:
        print(json.dumps({"walk": run_walk(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    if args.only_cells:
        print(json.dumps({"cells": run_cells(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    if args.only_batch:
        print(json.dumps({"batch": run_batch(args, vd, torch.cuda.current_stream())}), flush=True)
        return
    X = synth.uniform(args.N, args.d, seed=0)
    Xd = torch.tensor(X, device="cuda")
    stream = torch.cuda.current_stream()
    cfg = vd.vd_config_default()
    cfg.precision = VD_AUTO  # the library's default: the tensor-core list scan at 3 <= d <= 8
    cfg.knn_k = args.knn_k
    ctx = vd.vd_create(cfg, stream.cuda_stream)

    def step(c):
        vd.vd_set_nodes(c, Xd)
        m = vd.vd_vertices(c)
        st = vd.vd_mesh_stats(m)
        return m, st

    for _ in range(args.warmup):
        m, st = step(ctx)
        vd.vd_mesh_free(m)
    torch.cuda.synchronize()
    _barrier(ws)
    clock = ClockSampler(local)
    clock.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = vd.vd_kernel_launches()
    torch.cuda.synchronize()
    e0.record(stream)
    rays = 0
    rc_ms = 0.0
    last = None
    for k in range(args.steps):
        m, st = step(ctx)
        rays += st["rays"]
        rc_ms += st["raycast_ms"]
        last_stats = st
        if k == args.steps - 1:
            last = m
        else:
            vd.vd_mesh_free(m)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = vd.vd_kernel_launches() - launches0
    clocks = clock.stop()
    _barrier(ws)
    ms = e0.elapsed_time(e1)
    ms_max = _max_over_ranks(ms, ws)
    value = replica_value(rays, ms / 1000.0, ws)
    nv = vd.vd_mesh_count(last)
    tup = torch.empty((nv, args.d + 1), dtype=torch.int32, device="cuda")
    crd = torch.empty((nv, args.d), dtype=torch.float64, device="cuda")
    vd.vd_mesh_copy(last, tup, crd)
    vd.vd_mesh_free(last)

    def other_path(prec, reps=1):
        """The same traversal on another RayCast path: CUDA-event time of
        `reps` steps after one untimed step, and whether its vertex tuples
        equal the headline path's bit for bit."""
        c2 = vd.vd_config_default()
        c2.precision = prec
        c2.knn_k = args.knn_k
        ctx2 = vd.vd_create(c2, stream.cuda_stream)
        m, st = step(ctx2)
        vd.vd_mesh_free(m)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        rc, n = 0.0, 0
        for k in range(reps):
            m, st = step(ctx2)
            rc += st["raycast_ms"]
            n += st["rays"]
            if k < reps - 1:
                vd.vd_mesh_free(m)
        f1.record(stream)
        torch.cuda.synchronize()
        ms2 = f0.elapsed_time(f1) / reps
        tup2 = torch.empty((vd.vd_mesh_count(m), args.d + 1), dtype=torch.int32, device="cuda")
        vd.vd_mesh_copy(m, tup2, None)
        same = bool(tup2.shape == tup.shape and torch.equal(tup2, tup))
        vd.vd_mesh_free(m)
        vd.vd_destroy(ctx2)
        return {"value": n / reps / (ms2 / 1000.0), "ms_per_step": ms2, "raycast_ms": rc / reps,
                "pairs_per_ray": st["pairs_screened"] / max(st["rays"], 1), "tuples_identical_to_default": same}

    # ---- plain binary64 path and binary32 screening on the same workload ----
    fp64 = None if args.no_fp64 else other_path(VD_FP64)
    fp32 = None if args.no_binary32 else other_path(VD_FP32, reps=max(1, min(args.steps, 5)))

    # ---- end to end through the C ABI with host buffers ----
    Xh = np.ascontiguousarray(X)
    th = np.empty((nv, args.d + 1), np.int32)
    ch = np.empty((nv, args.d))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_rays = 0
    for _ in range(max(1, min(args.steps, 3))):
        vd.vd_set_nodes(ctx, Xh)
        m = vd.vd_vertices(ctx)
        e2e_rays += vd.vd_mesh_stats(m)["rays"]
        vd.vd_mesh_copy(m, th, ch)
        vd.vd_mesh_free(m)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = replica_value(e2e_rays, e2e_s, ws)
    h2d = Xh.nbytes
    d2h = th.nbytes + ch.nbytes

    # ---- roofline of the dominant kernel (the RayCast) ----
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    peak_tflops = nsm * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 lanes x FMA x clock
    pairs = NEIGHBOURS_D5 + 2 * args.d
    flops_per_ray = pairs * (2 * args.d + 6)
    achieved = rays * flops_per_ray / (rc_ms / 1000.0) / 1e12 if rc_ms > 0 else None
    # DRAM bytes of the RayCast per traversal of this workload (one ncu capture, above; `traffic` is null while a
    # kernel of the path has changed since); the ray I/O alone is ~573 MB
    captured = RAYCAST_DRAM_BYTES_PER_STEP if (args.N, args.d, args.knn_k) == (20000, 5, 0) else None
    traffic = captured if RAYCAST_TRAFFIC_CURRENT else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved / peak_tflops) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per step (every RayCast launch of one traversal)",
                "traffic_last_capture": captured,
                "traffic_last_capture_note": None if RAYCAST_TRAFFIC_CURRENT else
                "k_grp_scatter and k_grp_finish changed since (arithmetic of the face tests only)",
                "kernel": "k_ray_list_tc<5> with its prep/finish kernels and the tree-walk follow-up (tcgen05 fp16 screening of rays grouped by reference node, binary32 rescreen, binary64 recheck)",
                "peak_source": f"FP32 lanes x 2 x sm_max_mhz ({src} peaks file)",
                "algorithmic_flops_per_ray": flops_per_ray, "raycast_ms_per_step": rc_ms / args.steps}

    mc = None
    if not args.no_mc:
        mc = run_mc(args, vd, stream)
    highd = None
    if not args.no_highd:
        highd = run_highd(args, vd, stream)
    hmc = None
    if not args.no_hmc:
        hmc = run_hmc(args, vd, stream)
    walk = None
    if not args.no_walk:
        walk = run_walk(args, vd, stream)
    cells = None if args.no_cells else run_cells(args, vd, stream)
    small = None if args.no_small else run_small(args, vd, stream)
    batch = None if args.no_batch else run_batch(args, vd, stream)

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, n, dt, cores, rate1, n1, dt1 = cpu_oracle_rate(X, tup.cpu().numpy(), crd.cpu().numpy(),
                                                             target_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": "raycasts/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} random edge rays of the workload's diagram, FP64 brute force over all "
                         f"{args.N} nodes ({dt:.1f} s)",
               "one_core": {"value": rate1, "cores": 1, "sample": f"the first {n1} of those rays ({dt1:.1f} s)"}}
    vd.vd_destroy(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "raycasts/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": args.N, "d": args.d, "precision": "tcgen05 fp16 screen + fp32 rescreen + fp64 recheck",
                           "vertices": nv, "raycasts_per_step": rays / args.steps,
                           "levels": last_stats["levels"],
                           "pairs_per_ray": last_stats["pairs_screened"] / max(last_stats["rays"], 1),
                           "rechecked_per_ray": last_stats["rechecked"] / max(last_stats["rays"], 1),
                           "tree_walk_rays_per_step": last_stats["fallback_rays"],
                           "binary64_overflow_rays_per_step": last_stats["overflow_rays"],
                           "knn_k": args.knn_k,
                           "step_launches": last_stats["launches"],
                           "l2": "inputs larger than L2 (traversal tables ~1.5 GB per step)",
                           "parallelism": f"replicas x{ws}"},
                "fp64_path": fp64,
                "binary32_path": (dict(fp32, precision="binary32 screen, one thread per ray + fp64 recheck")
                                  if fp32 else None),
                "speedup_vs_fp64": (value / ws / fp64["value"]) if fp64 else None,
                "e2e": {"value": e2e_value, "unit": "raycasts/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "mc": mc, "highd": highd, "hmc": hmc, "walk": walk, "cells": cells, "plain_fp64_d3": small,
                "batch": batch}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


MC_WORKLOAD = ("MC volumes + interface areas + adjoint, d=4, N=100000 iid uniform in [0,1]^4 (seed 0), "
               "1024 rays per cell")


def time_integrals(vd, m, N, R, msamp, stream, reps=3):
    """Algorithm 3's function integrals F_V (msamp samples per ray) and F_d of
    f = sin(x_1^2) on the rays of a finished MC run: CUDA-event time of one
    vd_mc_integrals call (device outputs), mean of reps after one warm-up."""
    import torch
    nnz = vd.vd_mc_get(m)
    FV = torch.empty(N, dtype=torch.float64, device="cuda")
    Fd = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    f = vd.func_sin_sq(0)
    vd.vd_mc_integrals(m, f, msamp, FV, Fd[:nnz])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        vd.vd_mc_integrals(m, f, msamp, FV, Fd[:nnz])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"f": "sin(x_1^2)", "samples_per_ray": msamp, "ms": ms, "cells_per_s": N / (ms / 1000.0),
            "volume_samples_per_s": N * R * msamp / (ms / 1000.0)}


def run_mc(args, vd, stream):
    """Secondary line of the metric: MC vol+grad cells/s on the MC workload,
    binary32-screened path, tensor-core (fp16 tcgen05) screened path and
    plain binary64 path (same seeded directions, identical per-ray hits
    required)."""
    import torch
    from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, synth
    N, d, R = args.mc_n, 4, args.mc_rays
    X = torch.tensor(synth.uniform(N, d, seed=0), device="cuda")
    gV = torch.ones(N, dtype=torch.float64, device="cuda")
    out = {"workload": MC_WORKLOAD.replace("100000", str(N)).replace("1024 rays", f"{R} rays"),
           "unit": "cells/s"}
    hits = {}
    for name, prec in (("mixed", VD_FP32), ("tensor", VD_TC16), ("fp64", VD_FP64)):
        cfg = vd.vd_config_default()
        cfg.precision = prec
        ctx = vd.vd_create(cfg, stream.cuda_stream)
        gX = torch.empty((N, d), dtype=torch.float64, device="cuda")

        def step():
            vd.vd_set_nodes(ctx, X)
            m = vd.vd_mc_integrate(ctx, R, 7)
            nnz = vd.vd_mc_get(m)
            gA = torch.ones(max(nnz, 1), dtype=torch.float64, device="cuda")
            vd.vd_mc_adjoint(m, gV, gA[:nnz], gX)
            return m

        vd.vd_mc_free(step())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = vd.vd_mc_stats(m)
        h = torch.empty((N, R), dtype=torch.int32, device="cuda")
        vd.vd_mc_rays(m, h, None)
        hits[name] = h
        out[name] = {"cells_per_s": N / (ms / 1000.0), "rays_per_s": N * R / (ms / 1000.0), "ms_per_step": ms,
                     "raycast_ms": st["raycast_ms"], "tree_walk_rays": st["fallback_rays"],
                     "pairs_per_ray": st["pairs_screened"] / max(st["rays"], 1)}
        if name == "mixed":
            out["integrals"] = time_integrals(vd, m, N, R, args.mc_m, stream)
        vd.vd_mc_free(m)
        vd.vd_destroy(ctx)
    out["value"] = out["mixed"]["cells_per_s"]
    out["speedup_vs_fp64"] = out["mixed"]["cells_per_s"] / out["fp64"]["cells_per_s"]
    out["hits_identical_to_fp64"] = bool(torch.equal(hits["mixed"], hits["fp64"]) and
                                         torch.equal(hits["tensor"], hits["fp64"]))
    return out


HIGHD_WORKLOAD = ("MC volumes + interface areas + adjoint, d=16, N=200000 from a 32-component Gaussian mixture "
                  "(centres U[0,1]^16, sigma 0.1, redrawn outside the cube; seed 0), 64 rays per cell")


HMC_WORKLOAD = ("integrals of sin(x_1^2) over the cells and interfaces, d=5, N=20000 iid uniform in [0,1]^5 "
                "(seed 0): heuristic MC (Section 3.3) from the areas of 1024 rays per cell and the diagram's "
                "vertices, beside the MC integrals of Algorithm 3 (2 samples per ray) on the same rays and the "
                "exact integration of Section 3.2 (Algorithms 4-5) on the same vertices")


def run_hmc(args, vd, stream, reps=3):
    """Heuristic MC integration: CUDA-event time of one vd_hmc_integrals call
    (interface lists, sorted per interface, interface and cell integrals;
    device outputs), mean of reps after one warm-up, with the MC function
    integrals of the same rays timed the same way."""
    import torch
    from paper_2405_10050_gb300 import VD_FP32, synth
    N, d, R = args.N, args.d, 1024
    X = torch.tensor(synth.uniform(N, d, seed=0), device="cuda")
    cfg = vd.vd_config_default()
    cfg.precision = VD_FP32
    ctx = vd.vd_create(cfg, stream.cuda_stream)
    vd.vd_set_nodes(ctx, X)
    mesh = vd.vd_vertices(ctx)
    m = vd.vd_mc_integrate(ctx, R, 7)
    nnz = vd.vd_mc_get(m)
    VH = torch.empty(N, dtype=torch.float64, device="cuda")
    IH = torch.empty(N, dtype=torch.float64, device="cuda")
    FH = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    f = vd.func_sin_sq(0)

    def timed(fn, reps=reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: vd.vd_hmc_integrals(m, mesh, f, VH, FH[:nnz], IH))
    FV = torch.empty(N, dtype=torch.float64, device="cuda")
    ms_mc = timed(lambda: vd.vd_mc_integrals(m, f, 2, FV, FH[:nnz]))
    # the exact integration of Section 3.2 on the same vertices, and the
    # deviations of the MC volumes and of both integral estimates from it
    # (the comparisons of the paper's Section 4, here at this size)
    holder = []

    def poly_once():
        p = vd.vd_poly_integrate(ctx, mesh, f)
        holder.append(p)

    # one call, no warm-up: it takes seconds at this size (one thread per cell)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    poly_once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1)
    p = holder[-1]
    VP = torch.empty(N, dtype=torch.float64, device="cuda")
    FP = torch.empty(N, dtype=torch.float64, device="cuda")
    vd.vd_poly_get(p, VP, FP)
    vd.vd_poly_free(p)
    VM = torch.empty(N, dtype=torch.float64, device="cuda")
    vd.vd_mc_get(m, V=VM)
    rel = lambda a, b: float(((a - b) / b).abs().mean())
    out = {"workload": HMC_WORKLOAD.replace("N=20000", f"N={N}").replace("d=5", f"d={d}"), "unit": "cells/s",
           "value": N / (ms / 1000.0), "ms": ms, "vertices": vd.vd_mesh_count(mesh), "interfaces": nnz,
           "mc_integrals_ms": ms_mc, "exact_ms": ms_p, "exact_cells_per_s": N / (ms_p / 1000.0),
           "exact_volume_sum": float(VP.sum()),
           "mean_rel_dev_from_exact": {"mc_volume": rel(VM, VP), "mc_integral": rel(FV, FP),
                                       "hmc_integral": rel(IH, FP)}}
    vd.vd_mc_free(m)
    vd.vd_mesh_free(mesh)
    vd.vd_destroy(ctx)
    return out


WALK_WORKLOAD = ("random walks on the vertex graph (Section 2.3), d=5, N=20000 iid uniform in [0,1]^5 (seed 0): "
                 "1,000,000 walkers from distinct vertices of the diagram, 8 steps each")


def run_walk(args, vd, stream, W=1_000_000, S=8):
    """Random walks: CUDA-event time of one vd_random_walk call (device
    buffers), after one warm-up call; one RayCast per walker and step."""
    import torch
    from paper_2405_10050_gb300 import VD_FP32, synth
    N, d = args.N, args.d
    X = torch.tensor(synth.uniform(N, d, seed=0), device="cuda")
    cfg = vd.vd_config_default()
    cfg.precision = VD_FP32
    ctx = vd.vd_create(cfg, stream.cuda_stream)
    vd.vd_set_nodes(ctx, X)
    mesh = vd.vd_vertices(ctx)
    nv = vd.vd_mesh_count(mesh)
    T = torch.empty((nv, d + 1), dtype=torch.int32, device="cuda")
    vd.vd_mesh_copy(mesh, T, None)
    vd.vd_mesh_free(mesh)
    W = min(W, nv)
    g = torch.Generator(device="cpu").manual_seed(0)
    start = T[torch.randperm(nv, generator=g)[:W].sort().values.to("cuda")].contiguous()
    PT = torch.empty((W, S, d + 1), dtype=torch.int32, device="cuda")
    PC = torch.empty((W, S, d), dtype=torch.float64, device="cuda")
    vd.vd_random_walk(ctx, start, S, 1, PT, PC)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    vd.vd_random_walk(ctx, start, S, 2, PT, PC)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = vd.vd_last_stats(ctx)
    distinct = int(torch.unique(PT.view(-1, d + 1), dim=0).shape[0])
    vd.vd_destroy(ctx)
    return {"workload": WALK_WORKLOAD.replace("N=20000", f"N={N}").replace("d=5", f"d={d}"), "unit": "raycasts/s",
            "value": W * S / (ms / 1000.0), "ms": ms, "raycast_ms": st["raycast_ms"], "walkers": W, "steps": S,
            "distinct_vertices_visited": distinct, "vertices": nv}


CELLS_WORKLOAD = ("per-cell sequential exploration (Section 2.3: cells in index order, 1024 at a time, the edge "
                  "counters rebuilt per batch) beside the whole-diagram traversal, d=5, N=20000 iid uniform in [0,1]^5 "
                  "(seed 0)")


def run_cells(args, vd, stream, batch=1024, reps=2):
    """Per-cell exploration against the whole-diagram traversal: CUDA-event
    time of one call each (mean of reps after one warm-up), raycasts/s, the
    edge and vertex tables' sizes, and the device memory each context holds
    after its calls (the high-water mark of its workspace)."""
    import torch
    from paper_2405_10050_gb300 import synth
    N, d = args.N, args.d
    X = torch.tensor(synth.uniform(N, d, seed=0), device="cuda")
    out, tuples = {}, {}
    for name, b in (("by_cells", batch), ("whole", None)):
        torch.cuda.synchronize()
        ctx = vd.vd_create(None, stream.cuda_stream)
        vd.vd_set_nodes(ctx, X)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ms, st = 0.0, None
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mesh = vd.vd_vertices(ctx) if b is None else vd.vd_vertices_by_cells(ctx, b)
            e1.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                ms += e0.elapsed_time(e1) / reps
            st = vd.vd_mesh_stats(mesh)
            if r == reps:
                nv = vd.vd_mesh_count(mesh)
                T = torch.empty((nv, d + 1), dtype=torch.int32, device="cuda")
                vd.vd_mesh_copy(mesh, T, None)
                tuples[name] = T
            vd.vd_mesh_free(mesh)
        torch.cuda.synchronize()
        held = free0 - torch.cuda.mem_get_info()[0]
        vd.vd_destroy(ctx)
        out[name] = {"ms": ms, "raycasts_per_s": st["rays"] / (ms / 1000.0), "rays": st["rays"],
                     "levels": st["levels"], "vertices": st["vertices"], "edge_table_bytes": st["edge_table_bytes"],
                     "vertex_table_bytes": st["vertex_table_bytes"], "device_bytes_held": held}
    same = bool(torch.equal(tuples["by_cells"], tuples["whole"]))
    c, w = out["by_cells"], out["whole"]
    return {"workload": CELLS_WORKLOAD.replace("N=20000", f"N={N}").replace("d=5", f"d={d}")
            .replace("1024 at a time", f"{batch} at a time"), "unit": "raycasts/s", "value": c["raycasts_per_s"],
            "cells_per_batch": batch, "by_cells": c, "whole_diagram": w,
            "edge_table_ratio": w["edge_table_bytes"] / max(c["edge_table_bytes"], 1),
            "tuples_identical": same}


def run_highd(args, vd, stream):
    """MC vol+grad cells/s on the high-dimensional workload: tensor-core walk
    (tcgen05 ball tests and leaf screening) vs the binary32 tree walk, same
    seeded directions, identical per-ray hits required."""
    import torch
    from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, synth
    N, d, R = args.highd_n, 16, 64
    X = torch.tensor(synth.gaussian_mixture(N, d, K=32, sigma=0.1, seed=0), device="cuda")
    gV = torch.ones(N, dtype=torch.float64, device="cuda")
    out = {"workload": HIGHD_WORKLOAD.replace("200000", str(N)), "unit": "cells/s"}
    legs = [("tensor", VD_TC16), ("mixed", VD_FP32)] + ([("fp64", VD_FP64)] if args.highd_fp64 else [])
    hits = {}
    for name, prec in legs:
        cfg = vd.vd_config_default()
        cfg.precision = prec
        ctx = vd.vd_create(cfg, stream.cuda_stream)
        gX = torch.empty((N, d), dtype=torch.float64, device="cuda")

        def step():
            vd.vd_set_nodes(ctx, X)
            m = vd.vd_mc_integrate(ctx, R, 5)
            nnz = vd.vd_mc_get(m)
            gA = torch.ones(max(nnz, 1), dtype=torch.float64, device="cuda")
            vd.vd_mc_adjoint(m, gV, gA[:nnz], gX)
            return m

        vd.vd_mc_free(step())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = vd.vd_mc_stats(m)
        h = torch.empty((N, R), dtype=torch.int32, device="cuda")
        vd.vd_mc_rays(m, h, None)
        hits[name] = h
        vd.vd_mc_free(m)
        vd.vd_destroy(ctx)
        out[name] = {"cells_per_s": N / (ms / 1000.0), "rays_per_s": N * R / (ms / 1000.0), "ms_per_step": ms,
                     "raycast_ms": st["raycast_ms"], "tile_visits_per_ray": st["tiles_visited"] / max(st["rays"], 1),
                     "tree_walk_rays": st["fallback_rays"]}
    out["value"] = out["tensor"]["cells_per_s"]
    out["speedup_vs_mixed"] = out["tensor"]["cells_per_s"] / out["mixed"]["cells_per_s"]
    if "fp64" in out:
        out["speedup_vs_fp64"] = out["tensor"]["cells_per_s"] / out["fp64"]["cells_per_s"]
    out["hits_identical"] = all(bool(torch.equal(hits[a], hits["tensor"])) for a in hits)
    return out


BATCH_WORKLOAD = ("batched MC volumes + areas + adjoint: 512 sets, N log-uniform in [200, 20000], d uniform in "
                  "{2..8}, half uniform, half 8-component Gaussian mixtures (sigma 0.05), 256 rays per cell")


SMALL_WORKLOAD = ("plain method in binary64: exhaustive vertex traversal + MC volumes, areas and adjoint with 64 "
                  "rays per cell, d=3, N=2000 iid uniform in [0,1]^3 (seed 0), clipped to the cube")


def run_small(args, vd, stream, reps=5):
    """The plain binary64 method on the small workload: node preparation,
    the traversal, MC volumes + areas + adjoint (R = 64) per step, beside the
    same step on the default (screened) path; hits and tuples identical."""
    import torch
    from paper_2405_10050_gb300 import VD_AUTO, VD_FP64, synth
    X = synth.uniform(2000, 3, seed=0)
    Xd = torch.tensor(X, device="cuda")
    R = 64
    out = {"workload": SMALL_WORKLOAD, "unit": "raycasts/s"}
    ref = None
    for name, prec in (("fp64", VD_FP64), ("auto", VD_AUTO)):
        cfg = vd.vd_config_default()
        cfg.precision = prec
        ctx = vd.vd_create(cfg, stream.cuda_stream)

        def step():
            vd.vd_set_nodes(ctx, Xd)
            m = vd.vd_vertices(ctx)
            mst = vd.vd_mesh_stats(m)
            mc = vd.vd_mc_integrate(ctx, R, 1)
            N = X.shape[0]
            nnz = vd.vd_mc_get(mc)
            gX = torch.empty((N, 3), dtype=torch.float64, device="cuda")
            vd.vd_mc_adjoint(mc, torch.ones(N, dtype=torch.float64, device="cuda"),
                             torch.ones(max(nnz, 1), dtype=torch.float64, device="cuda")[:nnz], gX)
            return m, mc, mst

        m, mc, _ = step()
        vd.vd_mesh_free(m)
        vd.vd_mc_free(mc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            m, mc, mst = step()
            if k < reps - 1:
                vd.vd_mesh_free(m)
                vd.vd_mc_free(mc)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nv = vd.vd_mesh_count(m)
        tup = torch.empty((nv, 4), dtype=torch.int32, device="cuda")
        vd.vd_mesh_copy(m, tup, None)
        hit = torch.empty((2000, R), dtype=torch.int32, device="cuda")
        vd.vd_mc_rays(mc, hit, None)
        vd.vd_mesh_free(m)
        vd.vd_mc_free(mc)
        vd.vd_destroy(ctx)
        rays = mst["rays"] + 2000 * R
        out[name] = {"value": rays / (ms / 1000.0), "ms_per_step": ms, "vertices": nv, "traversal_rays": mst["rays"],
                     "mc_rays": 2000 * R, "mc_cells_per_s": 2000 / (ms / 1000.0)}
        if ref is None:
            ref = (tup, hit)
        else:
            out[name]["identical_to_fp64"] = bool(torch.equal(tup, ref[0]) and torch.equal(hit, ref[1]))
    out["value"] = out["fp64"]["value"]
    return out


def run_batch(args, vd, stream):
    """MC vol+grad cells/s on the batched workload (one persistent,
    graph-captured forward launch over all sets, then the adjoint of each)."""
    import torch
    from paper_2405_10050_gb300 import VD_FP32, synth
    sets = synth.batch_sets(args.batch_sets, seed=0)
    Xd = [torch.tensor(X, device="cuda") for X, _ in sets]
    ncell = sum(X.shape[0] for X, _ in sets)
    R = args.batch_rays
    cfg = vd.vd_config_default()
    cfg.precision = VD_FP32
    ctx = vd.vd_create(cfg, stream.cuda_stream)
    for mc in vd.vd_mc_integrate_batch(ctx, Xd, R, 3):  # first call: autotune
        vd.vd_mc_free(mc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mcs = vd.vd_mc_integrate_batch(ctx, Xd, R, 3)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st = vd.vd_last_stats(ctx)
    for mc, X in zip(mcs, Xd):
        N, d = X.shape
        nnz = vd.vd_mc_get(mc)
        gX = torch.empty((N, d), dtype=torch.float64, device="cuda")
        vd.vd_mc_adjoint(mc, torch.ones(N, dtype=torch.float64, device="cuda"),
                         torch.ones(max(nnz, 1), dtype=torch.float64, device="cuda")[:nnz], gX)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for mc in mcs:
        vd.vd_mc_free(mc)
    vd.vd_destroy(ctx)
    return {"workload": BATCH_WORKLOAD.replace("512", str(args.batch_sets)).replace("256 rays", f"{R} rays"),
            "cells": ncell, "rays": ncell * R, "unit": "cells/s",
            "value": ncell / (t2 - t0), "forward_graph_ms": st["ms"], "forward_call_s": t1 - t0,
            "adjoint_s": t2 - t1, "rays_per_s_forward_graph": ncell * R / (st["ms"] / 1000.0),
            "brute_force_rays": st["fallback_rays"], "launches_forward": st["launches"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=20000)
    ap.add_argument("--d", type=int, default=5)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-binary32", action="store_true", help="skip the binary32-screened traversal leg")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-rays", type=int, default=4000)
    ap.add_argument("--knn-k", type=int, default=0, help="candidate list length (0 automatic, -1 none)")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--only-mc", action="store_true")
    ap.add_argument("--only-batch", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-highd", action="store_true")
    ap.add_argument("--only-highd", action="store_true")
    ap.add_argument("--no-hmc", action="store_true")
    ap.add_argument("--no-walk", action="store_true")
    ap.add_argument("--only-walk", action="store_true")
    ap.add_argument("--no-cells", action="store_true")
    ap.add_argument("--only-cells", action="store_true")
    ap.add_argument("--only-hmc", action="store_true")
    ap.add_argument("--highd-fp64", action="store_true", help="also time the binary64 path (about 25 s)")
    ap.add_argument("--highd-n", type=int, default=200000)
    ap.add_argument("--batch-sets", type=int, default=512)
    ap.add_argument("--batch-rays", type=int, default=256)
    ap.add_argument("--mc-n", type=int, default=100000)
    ap.add_argument("--mc-rays", type=int, default=1024)
    ap.add_argument("--mc-m", type=int, default=2, help="samples per ray of the function-integral timing")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
