#!/usr/bin/env python
"""Benchmark: tet elements/s of the fused force + K*w map and the implicit
step, on the 64^3 mixed-precision neo-Hookean cube-grid workload.

Workload (stands in for the paper's FEM meshes, which are not available):
64 x 64 x 64 cubes, 5 tets per cube (274,625 vertices, 1,310,720 tets),
rest positions jittered by 1% of the edge, E log-uniform in [1e4, 1e6] per tet,
nu = 0.4, FP32 element math.  A timed step is one fused force + K*w map over
every tet (the metric's kernel) with inputs resident in HBM; L2 (129 MB) is
flushed by a 256 MB write before every timed step.  The implicit step (FP32
element maps + FP64 CG, 10 steps, rtol 1e-8) is timed in the same run next to
the plain FP64 form.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the baseline for this path: there is no reference code to run).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, each rank runs an independent replica of the
workload (the single-mesh path is not sharded), value = all ranks' tets / max
rank time.
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

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

METRIC = "tet elements/s for force+K·v (% of HBM roofline); implicit-step ms vs FP64 form"
UNIT = "tets/s"
N_SIDE = 64
SEED = 2
L2_FLUSH_BYTES = 256 << 20


# DRAM bytes (read + write) per launch of the bench kernel (interleaved
# fields) from one ncu capture on the 64^3 workload
# (profiles/tet_tile_kernel_fused_nh64.md).  Valid
# only while the kernel's sources are the ones captured; otherwise reported
# as null.
NCU_TRAFFIC = {"sources_sha256_16": "77a71dbb3d417ce1", "bytes_per_launch": 121.93e6}
# FP64 arithmetic of the FP64 kernels, counted by ncu (2 x DFMA + DADD + DMUL
# thread instructions per unit, sm__pipe_fp64_cycles_active) on the 64^3
# workload, valid while the map and spring sources hash to the same value.
NCU_FP64 = {"sources_sha256_16": "dc32b4c70d73aa62", "kv_map_nh_flops_per_tet": 454.8,
            "kv_map_nh_pipe_active": 0.882, "spring_flops_per_directed_spring": 32.15,
            "spring_pipe_active": 0.858}
# FP64 peak of the part, derived: 2 DFMA (4 flops) per clock per SM x 152 SMs
# x the maximum SM clock.
FP64_PEAK_TFLOPS = 4 * 152 * 2070e6 / 1e12
KERNEL_SOURCES = ["tet_maps.cu", "tile_map.cuh", "element.cuh", "tet_io.cuh", "tet_math.cuh", "tet_math_x2.cuh",
                  "async_copy.cuh", "ebb_internal.h", "layout.cu"]
FP64_SOURCES = KERNEL_SOURCES + ["springs.cu"]


def kernel_sources_hash(files=None):
    import hashlib
    h = hashlib.sha256()
    for f in files or KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1506_07577_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload():
    m = meshgen.cube_grid(N_SIDE, jitter=0.01, seed=SEED)
    mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, SEED)
    u = meshgen.random_displacement(m.X, N_SIDE, amp=0.05, seed=SEED, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=SEED)
    return m, mu, lam, u, w


def algorithmic_bytes_per_tet(n_verts, n_tets):
    """Bytes the fused FP32 map must move once per tet: keys (4 x int32),
    Dm^-1 (9 x f32), V (f32), per-tet (mu, lambda) (2 x f32), plus per vertex
    u and w read and f and K*w written (4 x 3 x f32) amortised over tets."""
    per_tet = 16 + 36 + 4 + 8
    per_vertex = 4 * 12
    return per_tet + per_vertex * n_verts / n_tets


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for name, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds, m, mu, lam, u, w, f_gpu, kw_gpu):
    """The CPU leg: the FP64 oracle's force + K*w on a contiguous sample of
    the same mesh's tets, timed on this host's cores (single thread); the
    same oracle then recomputes 32 sampled vertices exactly (from their
    incident tets only) and reports the GPU results' max-norm error there."""
    from oracle import fem
    sample = min(m.n_tets, 131072)
    tets = m.tets[:sample]
    B, V = fem.rest_shape(m.X, tets)
    mu_s, lam_s = mu[:sample], lam[:sample]
    x = m.X + u
    done = 0
    t0 = time.perf_counter()
    while True:
        fem.tet_forces(x, tets, B, V, mu_s, lam_s, fem.NEOHOOKEAN)
        fem.tet_Kv(x, w, tets, B, V, mu_s, lam_s, fem.NEOHOOKEAN)
        done += sample
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    rng = np.random.default_rng(0)
    vs = rng.choice(m.n_verts, size=32, replace=False)
    sel = np.isin(m.tets, vs).any(axis=1)
    sub = m.tets[sel]
    Bs, Vs = fem.rest_shape(m.X, sub)
    fo = fem.tet_forces(x, sub, Bs, Vs, mu[sel], lam[sel], fem.NEOHOOKEAN)[vs]
    ko = fem.tet_Kv(x, w, sub, Bs, Vs, mu[sel], lam[sel], fem.NEOHOOKEAN)[vs]
    err = max(float(np.max(np.abs(f_gpu[vs] - fo)) / np.max(np.abs(fo))),
              float(np.max(np.abs(kw_gpu[vs] - ko)) / np.max(np.abs(ko))))
    return {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle force+K*w over the first {sample} tets of the 64^3 mesh, "
                      f"repeated for {el:.1f} s ({done} tet evaluations), numpy single thread",
            "gpu_parity_max_rel_err_sampled": err}


def kern_avg_us(kern_ms):
    return 1e3 * sum(kern_ms) / len(kern_ms)


def max_over_ranks(seconds, dist, device):
    """The timing contract across replicas: the slowest rank's time (an
    all-reduce MAX when `dist` is torch.distributed, the value itself when
    it is None)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, seconds_max, world):
    """Whole-job throughput of `world` independent replicas that each did
    `units_per_rank` units, over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def run_reference(args, rank, world):
    if rank != 0:
        return
    m, mu, lam, u, w = workload()
    from oracle import fem
    sample = 65536
    tets = m.tets[:sample]
    B, V = fem.rest_shape(m.X, tets)
    x = m.X + u
    for _ in range(args.warmup):
        fem.tet_forces(x, tets, B, V, mu[:sample], lam[:sample], fem.NEOHOOKEAN)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fem.tet_forces(x, tets, B, V, mu[:sample], lam[:sample], fem.NEOHOOKEAN)
        fem.tet_Kv(x, w, tets, B, V, mu[:sample], lam[:sample], fem.NEOHOOKEAN)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "64^3 cube grid, 5 tets/cube, NH, E log-uniform [1e4,1e6], nu 0.4",
                       "n_tets": m.n_tets, "n_verts": m.n_verts, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: FP64 oracle force+K*w over the first {sample} tets"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1506_07577_gb300 import abi
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    m, mu, lam, u, w = workload()
    stream = torch.cuda.Stream(device=dev)
    dm = DeviceTetMesh(m.X, m.tets, mu, lam, device=local_rank, stream=stream, colour=True, edges=True)
    # Vector fields stored element by element (EBB_F32X4: x, y, z, padding), the
    # per-field contiguous vec3 storage of Section 6.1 padded to 16 bytes; the
    # same map on 3-plane fields is reported under "layouts".
    u32 = dm.vertex_field("u32", value=u, x4=True)
    w32 = dm.vertex_field("w32", value=w, x4=True)
    f = dm.vertex_field("f", x4=True)
    Kw = dm.vertex_field("Kw", x4=True)
    dm.vertex_field("u32p", torch.float32, value=u)
    dm.vertex_field("w32p", torch.float32, value=w)
    dm.vertex_field("fp", torch.float32)
    dm.vertex_field("Kwp", torch.float32)
    opts = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO)
    # The autotuner picks the tile size and reduction variant EBB_REDUCE_AUTO
    # resolves to (timing the K w map on these fields); untimed set-up.
    tune = tune_report(abi, abi.ebb_relation_autotune(dm.ctx, dm.tets, "u32", "w32",
                                                      abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32)))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nt = m.n_tets

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        f.zero_()
        Kw.zero_()
        if ev is not None:
            ev[1].record(stream)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32", "w32", "f", "Kw", opts)
        if ev is not None:
            ev[2].record(stream)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            flush.fill_(float(i))
            step()
        abi.ebb_ctx_sync(dm.ctx)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local_rank)
        clocks.start()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            step(evs[k])
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        abi.ebb_ctx_sync(dm.ctx)
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    kern_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = replica_throughput(nt * args.steps, total_s, world)

    # ---- end to end: one C-ABI call on pinned host buffers (copy u, w in,
    # zero f, K w, map, copy f, K w out, wait) -------------------------------
    uh = u32.cpu().pin_memory()
    wh = w32.cpu().pin_memory()
    fh = torch.empty_like(f, device="cpu").pin_memory()
    kh = torch.empty_like(Kw, device="cpu").pin_memory()
    opts_e2e = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO,
                            flags=abi.EBB_MAP_ZERO_OUT)
    with torch.cuda.stream(stream):
        e2e_ms = []
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u32", "w32", "f", "Kw", uh, wh, fh, kh, opts_e2e)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms) / 1e3, dist, dev)
    h2d = (uh.numel() + wh.numel()) * 4
    d2h = (fh.numel() + kh.numel()) * 4

    f_last = fh[:, :3].double().numpy().copy()
    kw_last = kh[:, :3].double().numpy().copy()

    # ---- reduction variants of the fused map (kernel time only) ----------
    variants = {}
    for name, red in (("atomic", abi.EBB_REDUCE_ATOMIC), ("colour", abi.EBB_REDUCE_COLOR),
                      ("gather", abi.EBB_REDUCE_GATHER), ("tiled_ordered", abi.EBB_REDUCE_TILED_ORDERED),
                      ("tiled", abi.EBB_REDUCE_TILED)):
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=red)
        ts = []
        with torch.cuda.stream(stream):
            for k in range(args.warmup + 5):
                flush.fill_(float(k))
                f.zero_()
                Kw.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32", "w32", "f", "Kw", o)
                b.record(stream)
                b.synchronize()
                if k >= args.warmup:
                    ts.append(a.elapsed_time(b) * 1e3)
        variants[name] = {"us": statistics.median(ts), "tets_per_s": nt / (statistics.median(ts) * 1e-6)}

    # ---- field layouts: the same tiled map on 3-plane fields --------------
    layouts = {"f32x4": {"us": kern_avg_us(kern_ms)}}
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    ts = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + 5):
            flush.fill_(float(k))
            dm._tensors["fp"].zero_()
            dm._tensors["Kwp"].zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32p", "w32p", "fp", "Kwp", o)
            b.record(stream)
            b.synchronize()
            if k >= args.warmup:
                ts.append(a.elapsed_time(b) * 1e3)
    layouts["planes"] = {"us": statistics.median(ts)}
    for v in layouts.values():
        v["tets_per_s"] = nt / (v["us"] * 1e-6)

    # ---- assembled K on the edge relation vs the matrix-free K w map ------
    asm = assembled_compare(dm, abi, torch, stream, args, flush)
    spr = springs_leg(dm, m, abi, torch, stream)
    f64map = fp64_map_leg(dm, u, w, abi, torch, stream, flush)

    # ---- implicit step: mixed form vs plain FP64 form -------------------
    imp = implicit_steps(dm, m, abi, torch, stream, args)
    bat = batched_steps(abi, torch, local_rank, args) if args.batch_meshes > 0 else None
    adj = adjoint_rollout(abi, torch, local_rank, args) if not args.no_adjoint else None
    perm = permuted_sweep(abi, torch, local_rank, args, _peaks()[0]) if args.permuted_n > 0 else None

    # ---- roofline of the dominant kernel ----------------------------------
    peak, peak_kind = _peaks()
    bpt = algorithmic_bytes_per_tet(m.n_verts, nt)
    kern_avg = sum(kern_ms) / len(kern_ms) / 1e3
    achieved = bpt * nt / kern_avg / 1e9
    traffic = NCU_TRAFFIC["bytes_per_launch"] if kernel_sources_hash() == NCU_TRAFFIC["sources_sha256_16"] else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read+write)",
            "kernel": {"tiled": "tet_tile_kernel<float, NEOHOOKEAN, FORCE|KV, interleaved>",
                       "atomic": "tet_map_kernel<float, NEOHOOKEAN, FORCE|KV, atomic, interleaved>",
                       "colour": "tet_map_kernel<float, NEOHOOKEAN, FORCE|KV, coloured, interleaved>",
                       "gather": "tet_corner_kernel<float, NEOHOOKEAN, FORCE|KV, interleaved> + "
                                 "vertex_sum_kernel<float, 2, interleaved>",
                       "tiled_ordered": "tet_tile_kernel<float, NEOHOOKEAN, FORCE|KV, interleaved> + "
                                        "partial_sum_kernel<float, 2, interleaved>"}[tune["reduce"]],
            "algorithmic_bytes_per_tet": bpt, "kernel_us": kern_avg * 1e6, "peak_kind": peak_kind}

    dm.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64^3 cube grid, 5 tets/cube (274,625 verts, 1,310,720 tets), NH, "
                                   "E log-uniform [1e4,1e6], nu 0.4, FP32 fused force+K*w map, reduction variant "
                                   "and tile size from the autotuner, vector fields stored as 4-float elements",
                       "n_tets": nt, "n_verts": m.n_verts, "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof,
            "autotune": tune,
            "reduction_variants": variants,
            "layouts": layouts,
            "assembled_K": asm,
            "spring_mass": spr,
            "fp64_kv_map": f64map,
            "e2e": {"value": replica_throughput(nt * args.steps, e2e_total, world), "unit": UNIT,
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "call": "ebb_map_tet_force_Kv_host on page-locked host buffers (EBB_MAP_ZERO_OUT)"},
            # library kernels per timed step: the map's launches for the
            # autotuned variant (the zeroing of f, K w is torch's fill)
            "gpu_launches": args.steps * {"tiled": 1, "atomic": 1, "gather": 2, "tiled_ordered": 2}.get(
                tune["reduce"], 1),
            "clocks": clk,
            "implicit_step": imp,
            "batched_step": bat,
            "adjoint_rollout": adj,
            "permuted_128": perm}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, m, mu, lam, u, w, f_last, kw_last)
    print(json.dumps(line), flush=True)


def assembled_compare(dm, abi, torch, stream, args, flush):
    """K(u) assembled on the edge relation (FP32 blocks) and its block-sparse
    product with w, against the matrix-free K w map (tiled), on the bench's
    4-float fields; L2 flushed before every timed launch."""
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32)
    o_kv = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    Kw = dm._tensors["Kw"]
    calls = {"assemble": lambda: abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u32", o),
             "spmv": lambda: abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w32", "Kw", o),
             "kv_map_tiled": lambda: abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u32", "w32", "Kw", o_kv)}
    res = {}
    with torch.cuda.stream(stream):
        for name, call in calls.items():
            ts = []
            for k in range(args.warmup + 5):
                flush.fill_(float(k))
                Kw.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                b.synchronize()
                if k >= args.warmup:
                    ts.append(a.elapsed_time(b) * 1e3)
            res[name + "_us"] = statistics.median(ts)
    return res


def springs_leg(dm, m, abi, torch, stream, steps=200):
    """The paper's spring-mass example (Section 4.1, Figure 1) on the 64^3
    mesh's edges: `steps` explicit steps per timed call, K = 1, dt = 1e-4,
    equal masses of density 1000 over the unit cube, from a perturbed rest
    state; FP32 (the figure's floats) and FP64.  Per-step time with CUDA
    events after warm-up."""
    rng = np.random.default_rng(7)
    q0 = m.X + 0.002 * rng.normal(size=m.X.shape)
    mass = np.full(m.n_verts, 1000.0 / m.n_verts)
    out = {"steps_per_call": steps, "k": 1.0, "dt": 1e-4}
    for name, dt_ in (("f32", torch.float32), ("f64", torch.float64)):
        dm.vertex_field("spos_" + name, dt_, value=m.X)
        dm.vertex_field("sq_" + name, dt_, value=q0)
        dm.vertex_field("sqd_" + name, dt_)
        dm.vertex_field("sm_" + name, dt_, ncomp=1, value=mass)
        with torch.cuda.stream(stream):
            abi.ebb_springs_init(dm.ctx, dm.tets, "spos_" + name)
            for _ in range(3):
                abi.ebb_springs_run(dm.ctx, dm.tets, "sq_" + name, "sqd_" + name, "sm_" + name, 1.0, 1e-4, 10)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            abi.ebb_springs_run(dm.ctx, dm.tets, "sq_" + name, "sqd_" + name, "sm_" + name, 1.0, 1e-4, steps)
            b.record(stream)
            b.synchronize()
            energy = abi.ebb_springs_run(dm.ctx, dm.tets, "sq_" + name, "sqd_" + name, "sm_" + name, 1.0, 1e-4, 0,
                                         energy=True)
        us = a.elapsed_time(b) * 1e3 / steps
        out[name + "_us_per_step"] = us
        out[name + "_kinetic_energy_after"] = energy
    nsprings = int(springs_directed_count(m))
    out["directed_springs"] = nsprings
    out["f32_springs_per_s"] = nsprings / (out["f32_us_per_step"] * 1e-6)
    if kernel_sources_hash(FP64_SOURCES) == NCU_FP64["sources_sha256_16"]:
        # FP64 steps are bound by the FP64 pipe: flops counted by ncu
        fl = NCU_FP64["spring_flops_per_directed_spring"] * nsprings
        out["f64_achieved_tflops"] = fl / (out["f64_us_per_step"] * 1e-6) / 1e12
        out["f64_frac_of_fp64_peak"] = out["f64_achieved_tflops"] / FP64_PEAK_TFLOPS
        out["f64_pipe_active_ncu"] = NCU_FP64["spring_pipe_active"]
    return out


def fp64_map_leg(dm, u, w, abi, torch, stream, flush):
    """The FP64 K w map (neo-Hookean, tiled, 3-plane FP64 fields) that the
    FP64 form of the implicit step runs once per CG iteration: CUDA-event
    median of 5 launches after 3 untimed ones, L2 flushed before each,
    against GB300's FP64 arithmetic peak (the kernel is bound by the FP64
    pipe, not by HBM)."""
    nt = dm.n_tets
    dm.vertex_field("u64", torch.float64, value=u)
    dm.vertex_field("w64", torch.float64, value=w)
    kk = dm.vertex_field("k64", torch.float64)
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64, reduce=abi.EBB_REDUCE_TILED)
    ts = []
    with torch.cuda.stream(stream):
        for it in range(3 + 5):
            flush.fill_(float(it))
            kk.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u64", "w64", "k64", o)
            b.record(stream)
            b.synchronize()
            if it >= 3:
                ts.append(a.elapsed_time(b) * 1e3)
    us = statistics.median(ts)
    out = {"kernel": "tet_tile_kernel<double, NEOHOOKEAN, KV>", "us": us, "tets_per_s": nt / (us * 1e-6),
           "bound": "alu", "peak_tflops": FP64_PEAK_TFLOPS, "peak_kind": "derived: 2 DFMA/clock/SM x 152 SMs x 2070 MHz"}
    if kernel_sources_hash(FP64_SOURCES) == NCU_FP64["sources_sha256_16"]:
        fl = NCU_FP64["kv_map_nh_flops_per_tet"]
        out.update({"fp64_flops_per_tet": fl, "achieved_tflops": fl * nt / (us * 1e-6) / 1e12,
                    "fp64_pipe_active_ncu": NCU_FP64["kv_map_nh_pipe_active"]})
        out["frac"] = out["achieved_tflops"] / FP64_PEAK_TFLOPS
    return out


def springs_directed_count(m):
    """Directed edges of the mesh (pairs of distinct vertices sharing a tet)."""
    t = m.tets.astype(np.int64)
    n = np.int64(m.n_verts)
    keys = [t[:, a] * n + t[:, b] for a in range(4) for b in range(4) if a != b]
    return np.unique(np.concatenate(keys)).size


def implicit_steps(dm, m, abi, torch, stream, args):
    """10 implicit steps from rest under gravity: the mixed form, the same with
    K assembled once per step (block-sparse CG products), the same with the
    ordered tiled reduction (the whole step bitwise reproducible), and the
    FP64 form.  One untimed step first (graph capture), then the state is
    reset."""
    uu = dm.vertex_field("u_state", torch.float64)
    vv = dm.vertex_field("v_state", torch.float64)
    dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(uu.device))
    out = {}
    res = {}
    for name, prec, flags, red in (("mixed", abi.EBB_PREC_F32, 0, abi.EBB_REDUCE_AUTO),
                                   ("mixed_assembled", abi.EBB_PREC_F32, abi.EBB_STEP_ASSEMBLED, abi.EBB_REDUCE_AUTO),
                                   ("mixed_ordered", abi.EBB_PREC_F32, 0, abi.EBB_REDUCE_TILED_ORDERED),
                                   ("fp64", abi.EBB_PREC_F64, 0, abi.EBB_REDUCE_AUTO)):
        prm = abi.step_params(abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, precision=prec, reduce=red, max_iters=1000,
                              rtol=1e-8, flags=flags)
        uu.zero_()
        vv.zero_()
        with torch.cuda.stream(stream):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u_state", "v_state", "pinned", prm)
        uu.zero_()
        vv.zero_()
        times, iters = [], []
        with torch.cuda.stream(stream):
            for s in range(args.implicit_steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u_state", "v_state", "pinned", prm)
                times.append(time.perf_counter() - t0)
                iters.append(rep.iters)
        res[name] = (uu.clone(), vv.clone())
        out[name] = {"ms_per_step": 1e3 * sum(times) / len(times), "cg_iters": iters}
    vmax = res["fp64"][1].abs().max().item()
    du = (res["mixed"][1] - res["fp64"][1]).abs().max().item() / vmax
    da = (res["mixed_assembled"][1] - res["fp64"][1]).abs().max().item() / vmax
    return {"steps": args.implicit_steps, "dt": 1e-3, "rtol": 1e-8,
            "mixed_ms_per_step": out["mixed"]["ms_per_step"], "fp64_ms_per_step": out["fp64"]["ms_per_step"],
            "speedup_vs_fp64_form": out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"],
            "cg_iters_mixed": out["mixed"]["cg_iters"], "cg_iters_fp64": out["fp64"]["cg_iters"],
            "v_rel_diff_mixed_vs_fp64_form": du,
            "mixed_assembled_ms_per_step": out["mixed_assembled"]["ms_per_step"],
            "cg_iters_mixed_assembled": out["mixed_assembled"]["cg_iters"],
            "v_rel_diff_mixed_assembled_vs_fp64_form": da,
            "mixed_ordered_ms_per_step": out["mixed_ordered"]["ms_per_step"],
            "cg_iters_mixed_ordered": out["mixed_ordered"]["cg_iters"],
            "v_rel_diff_mixed_ordered_vs_fp64_form":
                (res["mixed_ordered"][1] - res["fp64"][1]).abs().max().item() / vmax}


REDUCE_NAMES = {0: "atomic", 1: "colour", 3: "tiled", 4: "gather", 5: "tiled_ordered"}


def tune_report(abi, rep):
    return {"reduce": REDUCE_NAMES[rep.reduce], "tile_tets": rep.tile_tets, "interleaved": bool(rep.interleaved),
            "candidates_kw_map_us": [{"reduce": REDUCE_NAMES[rep.cand[i].reduce], "tile_tets": rep.cand[i].tile_tets,
                                      "interleaved": bool(rep.cand[i].interleaved), "us": rep.cand[i].us}
                                     for i in range(rep.ncand)]}


def batched_steps(abi, torch, local_rank, args):
    """256 independent cube grids, n log-uniform in [4, 24] (neo-Hookean,
    E = 1e5, nu = 0.45), one implicit step each: the batched call (mixed and
    FP64 forms) against one regular call per mesh (mixed)."""
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    sides = meshgen.batched_sizes(args.batch_meshes, 4, 24, seed=4)
    b = meshgen.cube_grid_batch(sides, jitter=0.01, seed=400)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    nt = int(b.tets.shape[0])
    out = {"meshes": int(len(sides)), "n_tets": nt, "n_verts": int(b.X.shape[0]),
           "sides_min": int(sides.min()), "sides_max": int(sides.max())}
    with DeviceTetMesh(b.X, b.tets, batch=b.batch, device=local_rank) as dm:
        uu = dm.vertex_field("u", torch.float64)
        vv = dm.vertex_field("v", torch.float64)
        dm.bind("pinned", torch.from_numpy(b.pinned.astype(np.uint8)).to(uu.device))
        # tile size and reduction variant of the batch picked by the autotuner
        dm.vertex_field("tu", torch.float32)
        dm.vertex_field("tw", torch.float32, value=meshgen.random_field(b.X.shape[0], seed=5))
        out["autotune"] = tune_report(abi, abi.ebb_relation_autotune(
            dm.ctx, dm.tets, "tu", "tw", abi.map_opts(abi.EBB_NEOHOOKEAN, mu, lam, precision=abi.EBB_PREC_F32)))
        vfinal = {}
        for name, prec in (("mixed", abi.EBB_PREC_F32), ("fp64", abi.EBB_PREC_F64)):
            prm = abi.step_params(abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, mu, lam, precision=prec, rtol=1e-8)
            ts = []
            for rep in range(3):
                uu.zero_()
                vv.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                reps = abi.ebb_cg_implicit_step_batched(dm.ctx, dm.tets, "u", "v", "pinned", "batch", len(sides),
                                                        prm)
                ts.append(time.perf_counter() - t0)
            out[f"{name}_ms"] = 1e3 * min(ts[1:])
            its = [r.iters for r in reps]
            out[f"{name}_cg_iters_min_max"] = [min(its), max(its)]
            vfinal[name] = vv.double().cpu().numpy()
        out["speedup_vs_fp64_form"] = out["fp64_ms"] / out["mixed_ms"]
        out["v_rel_diff_mixed_vs_fp64_form"] = float(np.max(np.abs(vfinal["mixed"] - vfinal["fp64"]))
                                                     / np.max(np.abs(vfinal["fp64"])))
    # one regular call per mesh (mixed), meshes resident, same workload
    meshes = []
    for m in range(len(sides)):
        X, tets, pinned = b.mesh(m)
        dm = DeviceTetMesh(X, tets, device=local_rank)
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64)
        dm.bind("pinned", torch.from_numpy(pinned.astype(np.uint8)).to(torch.device("cuda", local_rank)))
        meshes.append(dm)
    prm = abi.step_params(abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, mu, lam, precision=abi.EBB_PREC_F32, rtol=1e-8)
    for dm in meshes:   # warm-up (graph capture per mesh)
        abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
    for dm in meshes:
        dm._tensors["u"].zero_()
        dm._tensors["v"].zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for dm in meshes:
        abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm)
    out["per_mesh_calls_mixed_ms"] = 1e3 * (time.perf_counter() - t0)
    out["batched_speedup_vs_per_mesh_calls"] = out["per_mesh_calls_mixed_ms"] / out["mixed_ms"]
    for dm in meshes:
        dm.close()
    return out


def adjoint_rollout(abi, torch, local_rank, args):
    """32^3 StVK rollout (per-tet Lame parameters within +-20% of E = 1e5,
    nu = 0.45), 20 implicit steps, loss = sum of squared final displacements,
    gradient w.r.t. (u0, v0, mu, lambda) with checkpoints every 5 steps;
    timed against the plain FP64 forward rollout, and checked against a
    central difference (h = 1e-6) along one random direction."""
    from paper_1506_07577_gb300.autograd import rollout
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    n, steps, every, dt = 32, 20, 5, 1e-3
    m = meshgen.cube_grid(n, jitter=0.01, seed=3)
    mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed=3)
    dev = torch.device("cuda", local_rank)
    prm = abi.step_params(abi.EBB_STVK, dt, 1000.0, precision=abi.EBB_PREC_F64, max_iters=4000, rtol=1e-12)
    pin = torch.from_numpy(m.pinned.astype(np.uint8)).to(dev)
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=3)
    v0[m.pinned] = 0.0

    def make(mu_, lam_):
        dm = DeviceTetMesh(m.X, m.tets, mu_, lam_, device=local_rank)
        dm.bind("pinned", pin)
        return dm

    def forward_loss(dm, u0_, v0_):
        uu = dm.vertex_field("fu", torch.float64, value=u0_)
        dm.vertex_field("fv", torch.float64, value=v0_)
        for _ in range(steps):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "fu", "fv", "pinned", prm)
        return float((uu ** 2).sum())

    out = {"n_tets": m.n_tets, "n_verts": m.n_verts, "steps": steps, "checkpoint_every": every, "dt": dt}
    with make(mu, lam) as dm:
        u0 = np.zeros_like(m.X)
        forward_loss(dm, u0, v0)   # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        base = forward_loss(dm, u0, v0)
        torch.cuda.synchronize()
        out["fp64_forward_ms"] = 1e3 * (time.perf_counter() - t0)
        def leaves():
            return (torch.zeros((3, m.n_verts), dtype=torch.float64, device=dev, requires_grad=True),
                    torch.from_numpy(np.ascontiguousarray(v0.T)).to(dev).requires_grad_(True),
                    torch.from_numpy(mu).to(dev).requires_grad_(True),
                    torch.from_numpy(lam).to(dev).requires_grad_(True))

        # Warm-up rollout and backward (first use of the adjoint kernels and
        # of the solves on the recomputation fields), untimed.
        tu0, tv0, tmu, tlam = leaves()
        uT, _ = rollout(dm, tu0, tv0, tmu, tlam, steps, prm, checkpoint_every=every)
        (uT ** 2).sum().backward()
        tu0, tv0, tmu, tlam = leaves()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        uT, _ = rollout(dm, tu0, tv0, tmu, tlam, steps, prm, checkpoint_every=every)
        loss = (uT ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out["forward_with_checkpoints_ms"] = 1e3 * (t1 - t0)
        out["backward_ms"] = 1e3 * (t2 - t1)
        out["gradient_over_forward"] = (t2 - t0) / (out["fp64_forward_ms"] / 1e3)
        out["loss"] = float(loss.detach())
        out["loss_rel_diff_vs_plain_forward"] = abs(float(loss) - base) / base
        gu, gv = tu0.grad.cpu().numpy().T, tv0.grad.cpu().numpy().T
        gmu, glam = tmu.grad.cpu().numpy(), tlam.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    dv = rng.normal(size=v0.shape) * 1e-2
    dv[m.pinned] = 0.0
    dmu = rng.normal(size=mu.shape) * 1e3
    dlam = rng.normal(size=lam.shape) * 1e3
    h = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        with make(mu + sgn * h * dmu, lam + sgn * h * dlam) as dmp:
            vals.append(forward_loss(dmp, np.zeros_like(m.X), v0 + sgn * h * dv))
    fd = (vals[0] - vals[1]) / (2 * h)
    an = float(np.sum(gv * dv) + np.sum(gmu * dmu) + np.sum(glam * dlam))
    out["fd_directional_rel_err"] = abs(fd - an) / abs(an)
    return out


def permuted_sweep(abi, torch, local_rank, args, peak):
    """128^3 StVK (FP32 element math), vertex and tet ids randomly permuted
    (the library reorders tets internally): fused force + K*w per reduction
    variant, L2 flushed before each timed launch."""
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    n = args.permuted_n
    m = meshgen.cube_grid(n, jitter=0.01, seed=5, permute=True)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    u = meshgen.random_displacement(m.X, n, amp=0.05, seed=5, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=5)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    dm = DeviceTetMesh(m.X, m.tets, device=local_rank, colour=True)
    setup_s = time.perf_counter() - t0
    # 4-float vector elements (EBB_F32X4) as in the main line; "tiled_planes"
    # repeats the tiled map on 3-plane fields
    dm.vertex_field("u", value=u, x4=True)
    dm.vertex_field("w", value=w, x4=True)
    f = dm.vertex_field("f", x4=True)
    k = dm.vertex_field("k", x4=True)
    dm.vertex_field("up", torch.float32, value=u)
    dm.vertex_field("wp", torch.float32, value=w)
    fp = dm.vertex_field("fp", torch.float32)
    kp = dm.vertex_field("kp", torch.float32)
    bpt = 16 + 36 + 4 + 4 * 12 * m.n_verts / m.n_tets
    out = {"n_tets": m.n_tets, "n_verts": m.n_verts, "finalize_with_colouring_s": setup_s,
           "algorithmic_bytes_per_tet": bpt}
    t0 = time.perf_counter()
    dmr = DeviceTetMesh(m.X, m.tets, device=local_rank, reorder_verts=True)
    out["finalize_with_vertex_reorder_s"] = time.perf_counter() - t0
    dmr.vertex_field("u", value=u, x4=True)
    dmr.vertex_field("w", value=w, x4=True)
    fr = dmr.vertex_field("f", x4=True)
    kr = dmr.vertex_field("k", x4=True)
    names = ("u", "w", "f", "k")
    for name, red, mesh, ff, kk, nm in (("tiled", abi.EBB_REDUCE_TILED, dm, f, k, names),
                                        ("tiled_planes", abi.EBB_REDUCE_TILED, dm, fp, kp, ("up", "wp", "fp", "kp")),
                                        ("tiled_vertex_reordered", abi.EBB_REDUCE_TILED, dmr, fr, kr, names),
                                        ("atomic", abi.EBB_REDUCE_ATOMIC, dm, f, k, names),
                                        ("gather", abi.EBB_REDUCE_GATHER, dm, f, k, names),
                                        ("tiled_ordered", abi.EBB_REDUCE_TILED_ORDERED, dm, f, k, names),
                                        ("colour", abi.EBB_REDUCE_COLOR, dm, f, k, names)):
        o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=red)
        ts = []
        for it in range(3 + 5):
            flush.fill_(float(it))
            ff.zero_()
            kk.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.ebb_map_tet_force_Kv(mesh.ctx, mesh.tets, *nm, o)
            b.record()
            b.synchronize()
            if it >= 3:
                ts.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(ts)
        gbs = bpt * m.n_tets / t / 1e9
        out[name] = {"us": t * 1e6, "tets_per_s": m.n_tets / t, "algorithmic_GBps": gbs, "frac_of_peak": gbs / peak}
    out["tiled_vertex_reordered"]["note"] = ("includes permuting u, w into the internal vertex order and adding "
                                             "f, K*w back")
    dm.close()
    dmr.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--implicit-steps", type=int, default=10)
    ap.add_argument("--batch-meshes", type=int, default=256)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--permuted-n", type=int, default=128)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
