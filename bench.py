#!/usr/bin/env python
"""Benchmark: tet elements/s of the fused force + K*w map (fraction of the HBM
roofline) and implicit-step ms against the plain FP64 form.

Headline workload (stands in for the paper's large Vega meshes, Section 7.2,
which are not available): 128 x 128 x 128 cubes, 5 tets per cube (2,146,689
vertices, 10,485,760 tets), rest positions jittered by 1% of the edge, vertex
and tet ids randomly permuted by seed (poor locality: the library reorders
tets internally), St. Venant-Kirchhoff with E = 1e5, nu = 0.45, FP32 element
math.  A timed step zeroes f and K*w and runs one fused force + K*w map over
every tet with inputs resident in HBM; L2 (129 MB) is flushed by a 256 MB
write before every timed step (the map's inputs, about 1 GB, exceed L2 too).

Sub-records: the same map per reduction variant and field layout, warm; the
64^3 mixed-precision neo-Hookean workload (E log-uniform in [1e4, 1e6] per
tet, nu = 0.4): fused map, the assembled K, the spring-mass example, the FP64
K*w map, 10 implicit steps (mixed, assembled, ordered, FP64 form), the
batched step over 256 meshes and the 32^3 StVK adjoint rollout.

The CPU leg (`cpu_baseline`) times the FP64 oracle on the host and checks
every timed GPU result against it at sampled vertices (or whole meshes where
the oracle finishes in seconds).  --impl reference times the same oracle on
a bounded sample of the headline workload (the baseline for this path: there
is no reference code to run).  --profile runs one map or step a few times
for a profiler, and nothing else; --host-link measures the page-locked copy
bandwidth that bounds the end-to-end figure.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run each rank runs an independent replica of the workload
(the single-mesh path is not sharded), value = all ranks' tets / max rank
time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
L2_FLUSH_BYTES = 256 << 20
G = (0.0, 0.0, -9.81)

# DRAM bytes (read + write) per launch of the headline kernel (tiled, tiles
# of 128 tets) from one ncu capture of the full 128^3 headline workload per
# record layout (`--profile --n 128 --permute --renumber --model stvk
# --uniform --x4 [--planes]`).  They describe the kernel sources whose hash
# is given and are reported as null (with a note) once those sources change.
NCU_TRAFFIC = {"sources_sha256_16": "a1326421e942d5ff", "n": 128,
               "bytes_per_launch": {"rows": 989.13e6, "planes": 904.88e6}}
# FP64 arithmetic of the FP64 kernels, counted by ncu (2 x DFMA + DADD + DMUL
# thread instructions per unit) on the 64^3 workload, valid while the map and
# spring sources hash to the same value.
NCU_FP64 = {"sources_sha256_16": "e52dde8ea820429b", "kv_map_nh_flops_per_tet": 454.8,
            "kv_map_nh_pipe_active": 0.882, "spring_flops_per_directed_spring": 32.15,
            "spring_pipe_active": 0.858}
# FP64 peak of the part, derived: 2 DFMA (4 flops) per clock per SM x 152 SMs
# x the maximum SM clock.
FP64_PEAK_TFLOPS = 4 * 152 * 2070e6 / 1e12
KERNEL_SOURCES = ["tet_maps.cu", "tile_map.cuh", "element.cuh", "tet_io.cuh", "tet_math.cuh", "tet_math_x2.cuh",
                  "async_copy.cuh", "ebb_internal.h", "layout.cu"]
FP64_SOURCES = KERNEL_SOURCES + ["springs.cu"]
# Algorithmic bytes per free vertex and CG iteration of the mixed step's
# vector work (FP64 vectors, 24 B per vertex): p, A p's K p (FP32, 12 B),
# mass (8 B), 1/diag, r and y read; y, r and p written, and p's FP32 copy
# (12 B) for the next K p map.
CG_BYTES_PER_VERTEX = 24 + 12 + 8 + 24 + 24 + 24 + 24 + 24 + 24 + 12


def kernel_sources_hash(files=None):
    import hashlib
    h = hashlib.sha256()
    for f in files or KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1506_07577_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def host_info():
    """The host the CPU figures come from: logical CPUs and the CPU model."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model in ("", platform.machine()):
        try:  # Arm hosts name the model in lscpu, not in /proc/cpuinfo
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---- workloads --------------------------------------------------------------

def workload_permuted(n=128):
    """n^3 cube grid, ids permuted (seed 5), StVK E = 1e5, nu = 0.45 (uniform)."""
    m = meshgen.cube_grid(n, jitter=0.01, seed=5, permute=True)
    mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    u = meshgen.random_displacement(m.X, n, amp=0.05, seed=5, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=5)
    return m, mu, lam, u, w


def workload_nh64(n=64):
    """n^3 cube grid (seed 2), NH, E log-uniform [1e4, 1e6] per tet, nu = 0.4."""
    m = meshgen.cube_grid(n, jitter=0.01, seed=2)
    mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, 2)
    u = meshgen.random_displacement(m.X, n, amp=0.05, seed=2, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=2)
    return m, mu, lam, u, w


def algorithmic_bytes_per_tet(n_verts, n_tets, per_tet_material, fields=4):
    """Bytes an FP32 map must move once per tet: keys (4 x int32), Dm^-1
    (9 x f32), V (f32), per-tet (mu, lambda) (2 x f32) where bound, plus
    per vertex `fields` 3-vectors of f32 (u and w read, f and K*w written
    for the fused map) amortised over tets."""
    per_tet = 16 + 36 + 4 + (8 if per_tet_material else 0)
    return per_tet + fields * 12 * n_verts / n_tets


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


REDUCE_NAMES = {0: "atomic", 1: "colour", 3: "tiled", 4: "gather", 5: "tiled_ordered", 6: "coop"}


def tune_report(abi, rep):
    return {"reduce": REDUCE_NAMES[rep.reduce], "tile_tets": rep.tile_tets, "interleaved": bool(rep.interleaved),
            "records": "planes" if rep.record_planes else "rows",
            "candidates_kw_map_us": [{"reduce": REDUCE_NAMES[rep.cand[i].reduce], "tile_tets": rep.cand[i].tile_tets,
                                      "interleaved": bool(rep.cand[i].interleaved),
                                      "records": "planes" if rep.cand[i].record_planes else "rows",
                                      "us": rep.cand[i].us}
                                     for i in range(rep.ncand)]}


def map_launches(reduce_name, info, staged):
    """Library kernels one map call launches: the map itself (one launch per
    colour for the coloured variant, two passes for gather and ordered),
    plus the copy-in and add-back of staged operands."""
    n = {"tiled": 1, "atomic": 1, "coop": 1, "gather": 2, "tiled_ordered": 2,
         "colour": max(int(info.ncolours), 1)}[reduce_name]
    return n + (2 if staged else 0)


def time_calls(torch, stream, call, zero, flush, n, warm=3, flush_l2=True):
    """Median CUDA-event time (us) of `call` over n launches after `warm`
    untimed ones; `zero` (may be None) runs untimed before each; L2 flushed
    before each launch unless flush_l2 is false (warm-cache figure)."""
    ts = []
    with torch.cuda.stream(stream):
        for k in range(warm + n):
            if flush_l2:
                flush.fill_(float(k))
            if zero is not None:
                zero()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            b.synchronize()
            if k >= warm:
                ts.append(a.elapsed_time(b) * 1e3)
    return statistics.median(ts)


# ---- the headline: 128^3 permuted StVK, fused force + K*w -------------------

def run_headline(args, abi, torch, dev, local_rank, stream, flush, dist, world, barrier):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = workload_permuted(args.n)
    nt, nv = m.n_tets, m.n_verts
    # The relation renumbers its vertices at finalize (Morton order of the
    # rest positions; the runtime owns a relation's row order, Section 5.1),
    # and the vertex fields are loaded into that row order once, untimed.
    # The same map on fields kept in the scattered caller order is a
    # sub-record.
    t0 = time.perf_counter()
    dm = DeviceTetMesh(m.X, m.tets, device=local_rank, stream=stream, colour=True, renumber_verts=True)
    setup_s = time.perf_counter() - t0
    # Vector fields stored element by element (EBB_F32X4: x, y, z, padding),
    # the per-field contiguous vec3 storage of Section 6.1 padded to 16 bytes;
    # the same map on 3-plane fields is a sub-record.
    dm.vertex_field("u", value=u, x4=True)
    dm.vertex_field("w", value=w, x4=True)
    f = dm.vertex_field("f", x4=True)
    k = dm.vertex_field("k", x4=True)
    opts_t = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32)
    # The autotuner picks the tile size and reduction variant EBB_REDUCE_AUTO
    # resolves to (timing the K w map on these fields); untimed set-up.
    tune = tune_report(abi, abi.ebb_relation_autotune(dm.ctx, dm.tets, "u", "w", opts_t))
    info = abi.ebb_relation_info(dm.ctx, dm.tets)
    opts = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        f.zero_()
        k.zero_()
        if ev is not None:
            ev[1].record(stream)
        abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", opts)
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
        for s in range(args.steps):
            flush.fill_(float(s))
            step(evs[s])
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        abi.ebb_ctx_sync(dm.ctx)
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    kern_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    out = {"value": replica_throughput(nt * args.steps, total_s, world), "total_s": total_s,
           "kern_us": 1e3 * sum(kern_ms) / len(kern_ms), "clocks": clk, "tune": tune, "setup_s": setup_s,
           "n_tets": nt, "n_verts": nv, "ntiles": int(info.ntiles), "ncolours": int(info.ncolours),
           "launches_per_step": map_launches(tune["reduce"], info, False)}
    out["gpu_f"] = dm.caller(f[:, :3].double().cpu().numpy())
    out["gpu_k"] = dm.caller(k[:, :3].double().cpu().numpy())

    # ---- end to end: one C-ABI call on page-locked host buffers (copy u, w
    # in, zero f, K w, map, copy f, K w out, wait).  The host holds packed
    # (x, y, z) FP32 rows (EBB_MAP_HOST_XYZ: widened to the 4-float fields on
    # the device); the same call on 16-byte host elements is a sub-record.
    def e2e_calls(uh, wh, fh, kh, flags):
        o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO,
                         flags=abi.EBB_MAP_ZERO_OUT | flags)
        ms = []
        with torch.cuda.stream(stream):
            for s in range(args.warmup + args.steps):
                flush.fill_(float(s))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                abi.ebb_map_tet_force_Kv_host(dm.ctx, dm.tets, "u", "w", "f", "k", uh, wh, fh, kh, o)
                e1.record(stream)
                e1.synchronize()
                if s >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
        return ms

    uh = dm._tensors["u"][:, :3].contiguous().cpu().pin_memory()
    wh = dm._tensors["w"][:, :3].contiguous().cpu().pin_memory()
    fh = torch.empty((nv, 3), dtype=torch.float32).pin_memory()
    kh = torch.empty((nv, 3), dtype=torch.float32).pin_memory()
    e2e_ms = e2e_calls(uh, wh, fh, kh, abi.EBB_MAP_HOST_XYZ)
    # the host rows against the device-field map above (atomic order differs)
    e2e_diff = max(float(np.abs(dm.caller(fh.double().numpy()) - out["gpu_f"]).max() / np.abs(out["gpu_f"]).max()),
                   float(np.abs(dm.caller(kh.double().numpy()) - out["gpu_k"]).max() / np.abs(out["gpu_k"]).max()))
    e2e_total = max_over_ranks(sum(e2e_ms) / 1e3, dist, dev)
    out["e2e"] = {"value": replica_throughput(nt * args.steps, e2e_total, world), "unit": UNIT,
                  "h2d_bytes_per_step": (uh.numel() + wh.numel()) * 4,
                  "d2h_bytes_per_step": (fh.numel() + kh.numel()) * 4,
                  "ms_per_call": 1e3 * e2e_total / args.steps,
                  "call": "ebb_map_tet_force_Kv_host on page-locked packed (x, y, z) FP32 host rows "
                          "(EBB_MAP_HOST_XYZ | EBB_MAP_ZERO_OUT)",
                  "rel_diff_vs_device_map": e2e_diff}
    ux = dm._tensors["u"].cpu().pin_memory()
    wx = dm._tensors["w"].cpu().pin_memory()
    fx = torch.empty_like(f, device="cpu").pin_memory()
    kx = torch.empty_like(k, device="cpu").pin_memory()
    x4_ms = e2e_calls(ux, wx, fx, kx, 0)
    out["e2e"]["host_4float_elements"] = {
        "ms_per_call": statistics.mean(x4_ms), "tets_per_s": nt / (statistics.mean(x4_ms) * 1e-3),
        "h2d_bytes_per_step": (ux.numel() + wx.numel()) * 4, "d2h_bytes_per_step": (fx.numel() + kx.numel()) * 4}

    # ---- every reduction variant and field layout (kernel time), warm ------
    peak = _peaks()[0]
    bpt = algorithmic_bytes_per_tet(nv, nt, False)
    variants = {}

    def zero_xk():
        f.zero_()
        k.zero_()

    for name, red in (("tiled", abi.EBB_REDUCE_TILED), ("atomic", abi.EBB_REDUCE_ATOMIC),
                      ("tiled_ordered", abi.EBB_REDUCE_TILED_ORDERED), ("gather", abi.EBB_REDUCE_GATHER),
                      ("coop", abi.EBB_REDUCE_COOP), ("colour", abi.EBB_REDUCE_COLOR)):
        o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=red)
        us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o),
                        zero_xk, flush, 5)
        variants[name] = {"us": us, "tets_per_s": nt / (us * 1e-6),
                          "algorithmic_GBps": bpt * nt / (us * 1e-6) / 1e9,
                          "frac_of_peak": bpt * nt / (us * 1e-6) / 1e9 / peak}
    o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO)
    warm_us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o),
                         zero_xk, flush, 5, flush_l2=False)
    variants["autotuned_warm_l2"] = {"us": warm_us, "tets_per_s": nt / (warm_us * 1e-6),
                                     "note": "no L2 flush between launches (the map's ~1 GB of inputs exceed L2)"}
    dm.vertex_field("up", torch.float32, value=u)
    dm.vertex_field("wp", torch.float32, value=w)
    fp = dm.vertex_field("fp", torch.float32)
    kp = dm.vertex_field("kp", torch.float32)

    def zero_p():
        fp.zero_()
        kp.zero_()

    o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "up", "wp", "fp", "kp", o),
                    zero_p, flush, 5)
    variants["tiled_3plane_fields"] = {"us": us, "tets_per_s": nt / (us * 1e-6)}
    dm.close()
    # the vertex fields in the caller's scattered order (no renumbering): the
    # tiles gather and add each vertex where the caller's numbering puts it
    dmc = DeviceTetMesh(m.X, m.tets, device=local_rank, stream=stream)
    dmc.vertex_field("u", value=u, x4=True)
    dmc.vertex_field("w", value=w, x4=True)
    fc = dmc.vertex_field("f", x4=True)
    kc = dmc.vertex_field("k", x4=True)
    o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dmc.ctx, dmc.tets, "u", "w", "f", "k", o),
                    lambda: (fc.zero_(), kc.zero_()), flush, 5)
    variants["tiled_caller_order"] = {"us": us, "tets_per_s": nt / (us * 1e-6),
                                      "algorithmic_GBps": bpt * nt / (us * 1e-6) / 1e9,
                                      "frac_of_peak": bpt * nt / (us * 1e-6) / 1e9 / peak,
                                      "note": "fields in the caller's randomly permuted vertex order"}
    dmc.close()
    # vertex renumbering: the same map on a relation with internal Morton
    # vertex order (u, w permuted in and f, K w added back inside the call)
    t0 = time.perf_counter()
    dmr = DeviceTetMesh(m.X, m.tets, device=local_rank, stream=stream, reorder_verts=True)
    out["setup_vertex_reorder_s"] = time.perf_counter() - t0
    dmr.vertex_field("u", value=u, x4=True)
    dmr.vertex_field("w", value=w, x4=True)
    fr = dmr.vertex_field("f", x4=True)
    kr = dmr.vertex_field("k", x4=True)

    def zero_r():
        fr.zero_()
        kr.zero_()

    o = abi.map_opts(abi.EBB_STVK, mu, lam, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dmr.ctx, dmr.tets, "u", "w", "f", "k", o),
                    zero_r, flush, 5)
    variants["tiled_vertex_reordered"] = {"us": us, "tets_per_s": nt / (us * 1e-6),
                                          "note": "includes permuting u, w in and adding f, K*w back"}
    dmr.close()
    out["variants"] = variants
    out["workload"] = (m, mu, lam, u, w)
    return out


# ---- 64^3 mixed neo-Hookean sub-records -------------------------------------

def run_nh64(args, abi, torch, local_rank, stream, flush):
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, mu, lam, u, w = workload_nh64()
    nt = m.n_tets
    dm = DeviceTetMesh(m.X, m.tets, mu, lam, device=local_rank, stream=stream, colour=True, edges=True)
    dm.vertex_field("u32", value=u, x4=True)
    dm.vertex_field("w32", value=w, x4=True)
    f = dm.vertex_field("f", x4=True)
    Kw = dm.vertex_field("Kw", x4=True)
    tune = tune_report(abi, abi.ebb_relation_autotune(dm.ctx, dm.tets, "u32", "w32",
                                                      abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32)))
    peak = _peaks()[0]
    bpt = algorithmic_bytes_per_tet(m.n_verts, nt, True)

    def zero():
        f.zero_()
        Kw.zero_()

    variants = {}
    for name, red in (("autotuned", abi.EBB_REDUCE_AUTO), ("tiled", abi.EBB_REDUCE_TILED),
                      ("atomic", abi.EBB_REDUCE_ATOMIC), ("tiled_ordered", abi.EBB_REDUCE_TILED_ORDERED),
                      ("gather", abi.EBB_REDUCE_GATHER), ("coop", abi.EBB_REDUCE_COOP),
                      ("colour", abi.EBB_REDUCE_COLOR)):
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=red)
        us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32", "w32", "f", "Kw", o),
                        zero, flush, 5)
        variants[name] = {"us": us, "tets_per_s": nt / (us * 1e-6), "frac_of_peak": bpt * nt / (us * 1e-6) / 1e9 / peak}
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO)
    us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32", "w32", "f", "Kw", o),
                    zero, flush, 5, flush_l2=False)
    variants["autotuned_warm_l2"] = {"us": us, "tets_per_s": nt / (us * 1e-6),
                                     "frac_of_peak": bpt * nt / (us * 1e-6) / 1e9 / peak,
                                     "note": "no L2 flush: the map's 97 MB of algorithmic data fit in L2"}
    # the GPU result the CPU leg checks at sampled vertices
    abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32", "w32", "f", "Kw",
                             abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_AUTO,
                                          flags=abi.EBB_MAP_ZERO_OUT))
    abi.ebb_ctx_sync(dm.ctx)
    gpu_map = (f[:, :3].double().cpu().numpy(), Kw[:, :3].double().cpu().numpy())
    dm.vertex_field("u32p", torch.float32, value=u)
    dm.vertex_field("w32p", torch.float32, value=w)
    fp = dm.vertex_field("fp", torch.float32)
    kp = dm.vertex_field("Kwp", torch.float32)
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    us = time_calls(torch, stream, lambda: abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u32p", "w32p", "fp", "Kwp", o),
                    lambda: (fp.zero_(), kp.zero_()), flush, 5)
    variants["tiled_3plane_fields"] = {"us": us, "tets_per_s": nt / (us * 1e-6)}
    out = {"workload": "64^3 cube grid (274,625 verts, 1,310,720 tets), NH, E log-uniform [1e4,1e6] per tet, "
                       "nu 0.4, FP32 fused force+K*w map on 4-float vector elements, L2 flushed",
           "algorithmic_bytes_per_tet": bpt, "autotune": tune, "fused_map": variants}
    out["assembled_K"] = assembled_compare(dm, abi, torch, stream, flush)
    out["spring_mass"] = springs_leg(dm, m, abi, torch, stream)
    out["fp64_kv_map"] = fp64_map_leg(dm, u, w, abi, torch, stream, flush)
    imp, states = implicit_steps(dm, m, abi, torch, stream, args)
    out["implicit_step"] = imp
    dm.close()
    return out, {"mesh": (m, mu, lam, u, w), "map": gpu_map, "steps": states}


def assembled_compare(dm, abi, torch, stream, flush):
    """K(u) assembled on the edge relation (FP32 blocks) and its block-sparse
    product with w, against the matrix-free K w map (tiled), on 4-float
    fields; L2 flushed before every timed launch."""
    o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32)
    o_kv = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F32, reduce=abi.EBB_REDUCE_TILED)
    Kw = dm._tensors["Kw"]
    calls = {"assemble": lambda: abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u32", o),
             "spmv": lambda: abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w32", "Kw", o),
             "kv_map_tiled": lambda: abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u32", "w32", "Kw", o_kv)}
    return {name + "_us": time_calls(torch, stream, call, Kw.zero_, flush, 5) for name, call in calls.items()}


def springs_leg(dm, m, abi, torch, stream, steps=200):
    """The paper's spring-mass example (Section 4.1, Figure 1) on the 64^3
    mesh's edges: `steps` explicit steps per timed call, K = 1, dt = 1e-4,
    equal masses of density 1000 over the unit cube, from a perturbed rest
    state; FP32 (the figure's floats) and FP64."""
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
        out[name + "_us_per_step"] = a.elapsed_time(b) * 1e3 / steps
        out[name + "_kinetic_energy_after"] = energy
    nsprings = int(springs_directed_count(m))
    out["directed_springs"] = nsprings
    out["f32_springs_per_s"] = nsprings / (out["f32_us_per_step"] * 1e-6)
    if kernel_sources_hash(FP64_SOURCES) == NCU_FP64["sources_sha256_16"]:
        fl = NCU_FP64["spring_flops_per_directed_spring"] * nsprings
        out["f64_achieved_tflops"] = fl / (out["f64_us_per_step"] * 1e-6) / 1e12
        out["f64_frac_of_fp64_peak"] = out["f64_achieved_tflops"] / FP64_PEAK_TFLOPS
        out["f64_pipe_active_ncu"] = NCU_FP64["spring_pipe_active"]
    return out


def springs_directed_count(m):
    """Directed edges of the mesh (pairs of distinct vertices sharing a tet)."""
    t = m.tets.astype(np.int64)
    n = np.int64(m.n_verts)
    keys = [t[:, a] * n + t[:, b] for a in range(4) for b in range(4) if a != b]
    return np.unique(np.concatenate(keys)).size


def fp64_map_leg(dm, u, w, abi, torch, stream, flush):
    """The FP64 K w map (neo-Hookean, 3-plane FP64 fields) that the FP64
    form of the implicit step runs once per CG iteration, against GB300's
    FP64 arithmetic peak (the kernel is bound by the FP64 pipe): the tiled
    map with row records and with field-plane records, and the cooperative
    map (three threads per tet); the fastest is the winner."""
    nt = dm.n_tets
    dm.vertex_field("u64", torch.float64, value=u)
    dm.vertex_field("w64", torch.float64, value=w)
    kk = dm.vertex_field("k64", torch.float64)
    forms = {}
    for name, red, flags in (("tiled_row_records", abi.EBB_REDUCE_TILED, 0),
                             ("tiled_plane_records", abi.EBB_REDUCE_TILED, abi.EBB_TUNE_RECORD_PLANES),
                             ("coop", abi.EBB_REDUCE_COOP, 0)):
        abi.ebb_relation_set_tuning(dm.ctx, dm.tets, abi.EBB_NEOHOOKEAN, abi.EBB_PREC_F64, red, 128, flags)
        o = abi.map_opts(abi.EBB_NEOHOOKEAN, precision=abi.EBB_PREC_F64, reduce=abi.EBB_REDUCE_AUTO)
        forms[name] = time_calls(torch, stream, lambda: abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u64", "w64", "k64", o),
                                 kk.zero_, flush, 5)
    abi.ebb_relation_set_tuning(dm.ctx, dm.tets, abi.EBB_NEOHOOKEAN, abi.EBB_PREC_F64, abi.EBB_REDUCE_TILED, 128, 0)
    us = forms["tiled_row_records"]
    out = {"kernel": "tet_tile_kernel<double, NEOHOOKEAN, KV>", "us": us, "tets_per_s": nt / (us * 1e-6),
           "forms_us": forms, "winner": min(forms, key=forms.get),
           "bound": "alu", "peak_tflops": FP64_PEAK_TFLOPS, "peak_kind": "derived: 2 DFMA/clock/SM x 152 SMs x 2070 MHz"}
    if kernel_sources_hash(FP64_SOURCES) == NCU_FP64["sources_sha256_16"]:
        fl = NCU_FP64["kv_map_nh_flops_per_tet"]
        out.update({"fp64_flops_per_tet": fl, "achieved_tflops": fl * nt / (us * 1e-6) / 1e12,
                    "fp64_pipe_active_ncu": NCU_FP64["kv_map_nh_pipe_active"]})
        out["frac"] = out["achieved_tflops"] / FP64_PEAK_TFLOPS
    return out


def implicit_steps(dm, m, abi, torch, stream, args):
    """10 implicit steps from rest under gravity: the mixed form, the same with
    K assembled once per step (block-sparse CG products), the same with the
    ordered tiled reduction (the whole step bitwise reproducible), and the
    FP64 form.  One untimed step first (graph capture), then the state is
    reset.  Each form keeps the state before its last step for the CPU
    leg's check against the oracle's linear system."""
    uu = dm.vertex_field("u_state", torch.float64)
    vv = dm.vertex_field("v_state", torch.float64)
    dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(uu.device))
    res, out, states = {}, {}, {}
    nsteps = args.implicit_steps
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
            for s in range(nsteps):
                if s == nsteps - 1:
                    before = (uu.cpu().numpy().T.copy(), vv.cpu().numpy().T.copy())
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u_state", "v_state", "pinned", prm)
                times.append(time.perf_counter() - t0)
                iters.append(rep.iters)
        res[name] = (uu.clone(), vv.clone())
        states[name] = before + (vv.cpu().numpy().T.copy(),)
        out[name] = {"ms_per_step": 1e3 * sum(times) / len(times), "cg_iters": iters}
    vmax = res["fp64"][1].abs().max().item()
    peak = _peaks()[0]
    nt, nv = m.n_tets, m.n_verts
    free = int((~m.pinned).sum())
    # bytes moved per step by the mixed form: per CG iteration the K p map
    # (64 B per tet of keys, Dm^-1, V, mu, lambda and 3 x 12 B per vertex of
    # u, p read and K p written) and the CG vector work; once per step the
    # fused force + K v + diag map (60 B per vertex) and the set-up vectors.
    kp_map = 64 * nt + 36 * nv
    cg_vec = CG_BYTES_PER_VERTEX * free
    once = 64 * nt + 60 * nv + 8 * 24 * nv
    step_bytes = [it * (kp_map + cg_vec) + once for it in out["mixed"]["cg_iters"]]
    ms = out["mixed"]["ms_per_step"]
    gbs = statistics.mean(step_bytes) / (ms * 1e-3) / 1e9
    r = {"steps": nsteps, "dt": 1e-3, "rtol": 1e-8,
         "mixed_ms_per_step": ms, "fp64_ms_per_step": out["fp64"]["ms_per_step"],
         "speedup_vs_fp64_form": out["fp64"]["ms_per_step"] / ms,
         "cg_iters_mixed": out["mixed"]["cg_iters"], "cg_iters_fp64": out["fp64"]["cg_iters"],
         "mixed_us_per_cg_iteration": 1e3 * ms / statistics.mean(out["mixed"]["cg_iters"]),
         "mixed_roofline": {"bound": "hbm", "bytes_per_step": statistics.mean(step_bytes), "achieved_GBps": gbs,
                            "peak": peak, "frac": gbs / peak,
                            "bytes_model": f"iterations x (K p map {kp_map} B + CG vectors "
                                           f"{CG_BYTES_PER_VERTEX} B per free vertex) + {once} B once"},
         "v_rel_diff_mixed_vs_fp64_form": (res["mixed"][1] - res["fp64"][1]).abs().max().item() / vmax,
         "mixed_assembled_ms_per_step": out["mixed_assembled"]["ms_per_step"],
         "cg_iters_mixed_assembled": out["mixed_assembled"]["cg_iters"],
         "v_rel_diff_mixed_assembled_vs_fp64_form":
             (res["mixed_assembled"][1] - res["fp64"][1]).abs().max().item() / vmax,
         "mixed_ordered_ms_per_step": out["mixed_ordered"]["ms_per_step"],
         "cg_iters_mixed_ordered": out["mixed_ordered"]["cg_iters"],
         "v_rel_diff_mixed_ordered_vs_fp64_form":
             (res["mixed_ordered"][1] - res["fp64"][1]).abs().max().item() / vmax}
    return r, states


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
    vfinal = {}
    with DeviceTetMesh(b.X, b.tets, batch=b.batch, device=local_rank) as dm:
        uu = dm.vertex_field("u", torch.float64)
        vv = dm.vertex_field("v", torch.float64)
        dm.bind("pinned", torch.from_numpy(b.pinned.astype(np.uint8)).to(uu.device))
        dm.vertex_field("tu", torch.float32)
        dm.vertex_field("tw", torch.float32, value=meshgen.random_field(b.X.shape[0], seed=5))
        out["autotune"] = tune_report(abi, abi.ebb_relation_autotune(
            dm.ctx, dm.tets, "tu", "tw", abi.map_opts(abi.EBB_NEOHOOKEAN, mu, lam, precision=abi.EBB_PREC_F32)))
        for name, prec in (("mixed", abi.EBB_PREC_F32), ("fp64", abi.EBB_PREC_F64)):
            prm = abi.step_params(abi.EBB_NEOHOOKEAN, 1e-3, 1000.0, mu, lam, precision=prec, rtol=1e-8)
            ts = []
            for _ in range(3):
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
            vfinal[name] = (uu.double().cpu().numpy().T.copy(), vv.double().cpu().numpy().T.copy())
        out["speedup_vs_fp64_form"] = out["fp64_ms"] / out["mixed_ms"]
        out["v_rel_diff_mixed_vs_fp64_form"] = float(np.max(np.abs(vfinal["mixed"][1] - vfinal["fp64"][1]))
                                                     / np.max(np.abs(vfinal["fp64"][1])))
    meshes = []
    for mi in range(len(sides)):
        X, tets, pinned = b.mesh(mi)
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
    return out, {"batch": b, "mu": mu, "lam": lam, "final": vfinal}


ADJ = dict(n=32, steps=20, every=5, dt=1e-3, small_n=4)


def adjoint_rollout(abi, torch, local_rank, args):
    """32^3 StVK rollout (per-tet Lame parameters within +-20% of E = 1e5,
    nu = 0.45), 20 implicit steps, loss = sum of squared final displacements,
    gradient w.r.t. (u0, v0, mu, lambda) with checkpoints every 5 steps;
    timed against the plain FP64 forward rollout, and checked against a
    central difference (h = 1e-6) along one random direction.  The same
    rollout gradient on a 4^3 mesh is handed to the CPU leg, which checks it
    against the oracle's adjoint."""
    from paper_1506_07577_gb300.autograd import rollout
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    steps, every, dt = ADJ["steps"], ADJ["every"], ADJ["dt"]
    dev = torch.device("cuda", local_rank)
    prm = abi.step_params(abi.EBB_STVK, dt, 1000.0, precision=abi.EBB_PREC_F64, max_iters=4000, rtol=1e-12)

    def problem(n):
        m = meshgen.cube_grid(n, jitter=0.01, seed=3)
        mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed=3)
        v0 = 0.05 * meshgen.random_field(m.n_verts, seed=3)
        v0[m.pinned] = 0.0
        return m, mu, lam, v0

    def make(m, mu_, lam_):
        dm = DeviceTetMesh(m.X, m.tets, mu_, lam_, device=local_rank)
        dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dev))
        return dm

    def forward_loss(dm, u0_, v0_):
        uu = dm.vertex_field("fu", torch.float64, value=u0_)
        dm.vertex_field("fv", torch.float64, value=v0_)
        for _ in range(steps):
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "fu", "fv", "pinned", prm)
        return float((uu ** 2).sum())

    def grads(dm, m, mu, lam, v0, timed=None):
        def leaves():
            return (torch.zeros((3, m.n_verts), dtype=torch.float64, device=dev, requires_grad=True),
                    torch.from_numpy(np.ascontiguousarray(v0.T)).to(dev).requires_grad_(True),
                    torch.from_numpy(mu).to(dev).requires_grad_(True),
                    torch.from_numpy(lam).to(dev).requires_grad_(True))
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
        if timed is not None:
            timed["forward_with_checkpoints_ms"] = 1e3 * (t1 - t0)
            timed["backward_ms"] = 1e3 * (t2 - t1)
        return (float(loss.detach()), tu0.grad.cpu().numpy().T, tv0.grad.cpu().numpy().T, tmu.grad.cpu().numpy(),
                tlam.grad.cpu().numpy())

    m, mu, lam, v0 = problem(ADJ["n"])
    out = {"n_tets": m.n_tets, "n_verts": m.n_verts, "steps": steps, "checkpoint_every": every, "dt": dt}
    with make(m, mu, lam) as dm:
        u0 = np.zeros_like(m.X)
        forward_loss(dm, u0, v0)   # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        base = forward_loss(dm, u0, v0)
        torch.cuda.synchronize()
        out["fp64_forward_ms"] = 1e3 * (time.perf_counter() - t0)
        grads(dm, m, mu, lam, v0)  # warm-up of the adjoint kernels, untimed
        loss, gu, gv, gmu, glam = grads(dm, m, mu, lam, v0, timed=out)
        out["gradient_over_forward"] = (out["forward_with_checkpoints_ms"] + out["backward_ms"]) / out["fp64_forward_ms"]
        out["backward_over_forward"] = out["backward_ms"] / out["forward_with_checkpoints_ms"]
        out["loss"] = loss
        out["loss_rel_diff_vs_plain_forward"] = abs(loss - base) / base
    rng = np.random.default_rng(0)
    dv = rng.normal(size=v0.shape) * 1e-2
    dv[m.pinned] = 0.0
    dmu = rng.normal(size=mu.shape) * 1e3
    dlam = rng.normal(size=lam.shape) * 1e3
    h = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        with make(m, mu + sgn * h * dmu, lam + sgn * h * dlam) as dmp:
            vals.append(forward_loss(dmp, np.zeros_like(m.X), v0 + sgn * h * dv))
    fd = (vals[0] - vals[1]) / (2 * h)
    an = float(np.sum(gv * dv) + np.sum(gmu * dmu) + np.sum(glam * dlam))
    out["fd_directional_rel_err"] = abs(fd - an) / abs(an)
    # the same gradient on a small mesh for the CPU leg's oracle check
    ms, mus, lams, v0s = problem(ADJ["small_n"])
    with make(ms, mus, lams) as dm:
        small = grads(dm, ms, mus, lams, v0s)
    return out, {"mesh": (ms, mus, lams, v0s), "grads": small}


def small_configs(abi, torch, local_rank, stream):
    """The launch-bound configurations, reported as us per step and per map
    (their data fit in L2, so no roofline fraction):
      C1: 8^3 grid, StVK E = 1e5, nu = 0.45, FP64, one implicit step from rest
          (dt 1e-3, rho 1000, 50 CG iterations, early stop at 1e-14);
      C3: 32^3 grid, StVK with per-tet Lame parameters within +-20%, FP64,
          one implicit step from a random velocity (rtol 1e-12).
    Each also times the FP64 fused force + K*w map on a random state.  The C1
    step's result goes to the CPU leg for the oracle's check."""
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    dev = torch.device("cuda", local_rank)
    out, c1_check = {}, None
    cases = (("C1_8cubed", 8, False, 50, 1e-14, 0.0), ("C3_32cubed", 32, True, 4000, 1e-12, 0.05))
    for name, n, per_tet, iters, rtol, vscale in cases:
        m = meshgen.cube_grid(n, jitter=0.01, seed=1 if n == 8 else 3)
        if per_tet:
            mu, lam = meshgen.material_perturbed_lame(m.n_tets, 1e5, 0.45, 0.2, seed=3)
            mu0, lam0 = 0.0, 0.0
        else:
            mu0, lam0 = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
        v0 = vscale * meshgen.random_field(m.n_verts, seed=3)
        v0[m.pinned] = 0.0
        u = meshgen.random_displacement(m.X, n, amp=0.05, seed=4, smooth=0.01)
        w = meshgen.random_field(m.n_verts, seed=5)
        with DeviceTetMesh(m.X, m.tets, mu if per_tet else None, lam if per_tet else None, device=local_rank,
                           stream=stream) as dm:
            dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dev))
            us = dm.vertex_field("u", torch.float64)
            vs = dm.vertex_field("v", torch.float64, value=v0)
            v_init = vs.clone()
            prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu0, lam0, precision=abi.EBB_PREC_F64,
                                  max_iters=iters, rtol=rtol)
            ts, reps = [], []
            with torch.cuda.stream(stream):
                for k in range(8):
                    us.zero_()
                    vs.copy_(v_init)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    reps.append(abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm))
                    b.record(stream)
                    b.synchronize()
                    if k >= 3:
                        ts.append(a.elapsed_time(b) * 1e3)
            rec = {"n_tets": m.n_tets, "n_verts": m.n_verts, "fp64_step_us": statistics.median(ts),
                   "cg_iters": int(reps[-1].iters)}
            if n == 8:
                c1_check = {"mesh": m, "mu": mu0, "lam": lam0, "v0": v0,
                            "u": dm._tensors["u"].cpu().numpy().T.copy(), "v": dm._tensors["v"].cpu().numpy().T.copy()}
            dm.vertex_field("mu_", torch.float64, value=u)
            dm.vertex_field("mw_", torch.float64, value=w)
            dm.vertex_field("mf_", torch.float64)
            dm.vertex_field("mk_", torch.float64)
            o = abi.map_opts(abi.EBB_STVK, mu0, lam0, precision=abi.EBB_PREC_F64, flags=abi.EBB_MAP_ZERO_OUT)
            ms = []
            with torch.cuda.stream(stream):
                for k in range(23):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "mu_", "mw_", "mf_", "mk_", o)
                    b.record(stream)
                    b.synchronize()
                    if k >= 3:
                        ms.append(a.elapsed_time(b) * 1e3)
            rec["fp64_fused_map_us"] = statistics.median(ms)
            rec["note"] = "launch-bound (data fit in L2): warm, no roofline fraction"
            out[name] = rec
    return out, c1_check


# ---- the CPU leg: oracle timing and every result's error vs the oracle -----

def cpu_baseline(seconds, head, nh64, bat, adj, c1=None):
    """Times the FP64 oracle's force + K*w (single thread, numpy) on a
    contiguous sample of the headline mesh's tets, then checks the timed GPU
    results against the oracle: the maps at sampled vertices (each recomputed
    exactly from its incident tets), each implicit-step form's last step
    through the oracle's linear system at sampled free vertices (b and A dv
    from the tets around each vertex, dv the GPU's velocity change), the
    batched step on its smallest, a middle and its largest mesh (whole
    oracle steps), the rollout gradient on the small mesh (the oracle's
    adjoint) and the C1 step (a whole oracle step)."""
    from oracle import adjoint, fem, implicit
    m, mu, lam, u, w = head["workload"]
    sample = min(m.n_tets, 131072)
    tets = m.tets[:sample]
    B, V = fem.rest_shape(m.X, tets)
    x = m.X + u
    done = 0
    t0 = time.perf_counter()
    while True:
        fem.tet_forces(x, tets, B, V, mu, lam, fem.STVK)
        fem.tet_Kv(x, w, tets, B, V, mu, lam, fem.STVK)
        done += sample
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    out = {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
           "sample": f"FP64 oracle force+K*w over the first {sample} (randomly numbered) tets of the permuted "
                     f"128^3 StVK mesh, repeated for {el:.1f} s ({done} tet evaluations), numpy single thread"}
    rng = np.random.default_rng(0)
    errs = {}

    def map_err(mesh, mu_, lam_, u_, w_, model, f_gpu, k_gpu, nsample=32):
        vs = rng.choice(mesh.n_verts, size=nsample, replace=False)
        sel = np.isin(mesh.tets, vs).any(axis=1)
        sub = mesh.tets[sel]
        Bs, Vs = fem.rest_shape(mesh.X, sub)
        mu_s = mu_[sel] if np.ndim(mu_) else mu_
        lam_s = lam_[sel] if np.ndim(lam_) else lam_
        xs = mesh.X + u_
        fo = fem.tet_forces(xs, sub, Bs, Vs, mu_s, lam_s, model, mesh.n_verts)[vs]
        ko = fem.tet_Kv(xs, w_, sub, Bs, Vs, mu_s, lam_s, model, mesh.n_verts)[vs]
        return max(float(np.max(np.abs(f_gpu[vs] - fo)) / np.max(np.abs(fo))),
                   float(np.max(np.abs(k_gpu[vs] - ko)) / np.max(np.abs(ko))))

    errs["headline_fused_map_sampled"] = map_err(m, mu, lam, u, w, fem.STVK, head["gpu_f"], head["gpu_k"])
    if nh64 is not None:
        mn, mun, lamn, un, wn = nh64["mesh"]
        errs["nh64_fused_map_sampled"] = map_err(mn, mun, lamn, un, wn, fem.NEOHOOKEAN, *nh64["map"])
        free = np.flatnonzero(~mn.pinned)
        vs = rng.choice(free, size=64, replace=False)
        sel = np.isin(mn.tets, vs).any(axis=1)
        sub = mn.tets[sel]
        Bs, Vs = fem.rest_shape(mn.X, sub)
        mass = fem.lumped_mass(Vs, sub, 1000.0, mn.n_verts)[vs][:, None]
        dt = 1e-3
        for name, (u_n, v_n, v_np1) in nh64["steps"].items():
            xs = mn.X + u_n
            dvel = v_np1 - v_n
            f = fem.tet_forces(xs, sub, Bs, Vs, mun[sel], lamn[sel], fem.NEOHOOKEAN, mn.n_verts)[vs]
            kv = fem.tet_Kv(xs, v_n, sub, Bs, Vs, mun[sel], lamn[sel], fem.NEOHOOKEAN, mn.n_verts)[vs]
            kdv = fem.tet_Kv(xs, dvel, sub, Bs, Vs, mun[sel], lamn[sel], fem.NEOHOOKEAN, mn.n_verts)[vs]
            b = dt * (f + mass * np.array(G) - dt * kv)
            adv = mass * dvel[vs] + dt * dt * kdv
            errs[f"nh64_step_{name}_residual_sampled"] = float(np.max(np.abs(adv - b)) / np.max(np.abs(b)))
    if bat is not None:
        b = bat["batch"]
        order = np.argsort(b.sides, kind="stable")
        worst = 0.0
        for mi in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
            X, tets, pinned = b.mesh(mi)
            Bm, Vm = fem.rest_shape(X, tets)
            mass = fem.lumped_mass(Vm, tets, 1000.0, X.shape[0])
            uo, vo, _ = implicit.implicit_step(X, np.zeros_like(X), np.zeros_like(X), tets, Bm, Vm, mass, bat["mu"],
                                               bat["lam"], fem.NEOHOOKEAN, 1e-3, np.array(G), pinned, 1000, 1e-8)
            a, e = b.vert_off[mi], b.vert_off[mi + 1]
            worst = max(worst, float(np.max(np.abs(bat["final"]["mixed"][1][a:e] - vo)) / np.max(np.abs(vo))))
        errs["batched_mixed_v_rel_err_3_meshes"] = worst
    if adj is not None:
        ms, mus, lams, v0s = adj["mesh"]
        Bm, Vm = fem.rest_shape(ms.X, ms.tets)
        mass = fem.lumped_mass(Vm, ms.tets, 1000.0, ms.n_verts)
        states = adjoint.rollout(ms.X, np.zeros_like(ms.X), v0s, ms.tets, Bm, Vm, mass, mus, lams, ADJ["dt"],
                                 np.array(G), ms.pinned, ADJ["steps"])
        uT = states[-1][0]
        gu, gv, gmu, glam, _ = adjoint.rollout_grad(ms.X, np.zeros_like(ms.X), v0s, ms.tets, Bm, Vm, mass, mus, lams,
                                                    ADJ["dt"], np.array(G), ms.pinned, ADJ["steps"], 2 * uT,
                                                    np.zeros_like(uT))
        _, tgu, tgv, tgmu, tglam = adj["grads"]
        errs["adjoint_rollout_grad_4cubed"] = max(
            float(np.max(np.abs(a - b_)) / np.max(np.abs(b_))) for a, b_ in ((tgu, gu), (tgv, gv), (tgmu, gmu),
                                                                             (tglam, glam)))
    if c1 is not None:
        # the C1 FP64 step against the oracle's step (the whole field)
        m = c1["mesh"]
        B, V = fem.rest_shape(m.X, m.tets)
        mass = fem.lumped_mass(V, m.tets, 1000.0, m.n_verts)
        uo, vo, _ = implicit.implicit_step(m.X, np.zeros_like(m.X), c1["v0"], m.tets, B, V, mass, c1["mu"],
                                           c1["lam"], fem.STVK, 1e-3, np.array(G), m.pinned, 50, 1e-14)
        errs["c1_fp64_step_v"] = float(np.max(np.abs(c1["v"] - vo)) / np.max(np.abs(vo)))
        errs["c1_fp64_step_u"] = float(np.max(np.abs(c1["u"] - uo)) / np.max(np.abs(uo)))
    out["gpu_errors_vs_oracle"] = errs
    return out


# ---- reference arm and profiling mode ---------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    m, mu, lam, u, w = workload_permuted(args.n)
    from oracle import fem
    sample = min(65536, m.n_tets)
    tets = m.tets[:sample]
    B, V = fem.rest_shape(m.X, tets)
    x = m.X + u
    for _ in range(args.warmup):
        fem.tet_forces(x, tets, B, V, mu, lam, fem.STVK)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fem.tet_forces(x, tets, B, V, mu, lam, fem.STVK)
        fem.tet_Kv(x, w, tets, B, V, mu, lam, fem.STVK)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.n}^3 cube grid, 5 tets/cube, vertex and tet ids permuted, StVK E 1e5 "
                                   "nu 0.45, force+K*w", "n_tets": m.n_tets, "n_verts": m.n_verts,
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
                             "sample": f"each step: FP64 oracle force+K*w over the first {sample} tets"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(argv):
    """Run one element map (or step, assembled product, spring-mass steps) a
    few times on a cube-grid workload, for profilers; prints one line.

        python bench.py --profile --n 80 --permute --model stvk --uniform --x4

    Meshes: the n^3 cube grid (1% jitter, seed 2 or, with --permute, seed 5
    and permuted ids); neo-Hookean/StVK with E log-uniform in [1e4, 1e6],
    nu = 0.4 per tet, or with --uniform E = 1e5, nu = 0.45."""
    import torch

    from paper_1506_07577_gb300 import abi
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh

    ap = argparse.ArgumentParser(prog="bench.py --profile")
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--variant", choices=["auto", "atomic", "tiled", "colour", "gather", "ordered", "coop"],
                    default="tiled")
    ap.add_argument("--planes", action="store_true", help="tile blobs with per-tet data as field planes")
    ap.add_argument("--ops", choices=["fused", "kv", "force", "diag", "step", "spmv", "springs", "vjp"],
                    default="fused")
    ap.add_argument("--prec", choices=["f32", "f64"], default="f32")
    ap.add_argument("--model", choices=["nh", "stvk"], default="nh")
    ap.add_argument("--permute", action="store_true")
    ap.add_argument("--uniform", action="store_true", help="uniform material (no per-tet Lame fields)")
    ap.add_argument("--x4", action="store_true", help="FP32 vector fields as EBB_F32X4 elements")
    ap.add_argument("--renumber", action="store_true", help="the relation renumbers its vertices at finalize")
    ap.add_argument("--iters", type=int, default=3)
    a = ap.parse_args(argv)

    seed = 5 if a.permute else 2
    m = meshgen.cube_grid(a.n, jitter=0.01, seed=seed, permute=a.permute)
    if a.uniform:
        mu, lam = (float(x) for x in meshgen.lame_from_young(1e5, 0.45))
    else:
        mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, 2)
    u = meshgen.random_displacement(m.X, a.n, amp=0.05, seed=seed, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=seed)
    dt = torch.float32 if a.prec == "f32" else torch.float64
    mdl = abi.EBB_NEOHOOKEAN if a.model == "nh" else abi.EBB_STVK
    red = {"auto": abi.EBB_REDUCE_AUTO, "atomic": abi.EBB_REDUCE_ATOMIC, "tiled": abi.EBB_REDUCE_TILED,
           "colour": abi.EBB_REDUCE_COLOR, "gather": abi.EBB_REDUCE_GATHER,
           "ordered": abi.EBB_REDUCE_TILED_ORDERED, "coop": abi.EBB_REDUCE_COOP}[a.variant]
    mu0, lam0 = (mu, lam) if a.uniform else (0.0, 0.0)
    prec = abi.EBB_PREC_F32 if a.prec == "f32" else abi.EBB_PREC_F64
    with DeviceTetMesh(m.X, m.tets, None if a.uniform else mu, None if a.uniform else lam,
                       colour=(a.variant == "colour"), edges=a.ops in ("spmv", "springs"),
                       renumber_verts=a.renumber) as dm:
        x4 = a.x4 and a.prec == "f32"
        dm.vertex_field("u", dt, value=u, x4=x4)
        dm.vertex_field("w", dt, value=w, x4=x4)
        dm.vertex_field("f", dt, x4=x4)
        dm.vertex_field("k", dt, x4=x4)
        o = abi.map_opts(mdl, mu0, lam0, precision=prec, reduce=red, flags=abi.EBB_MAP_ZERO_OUT)
        if a.variant == "auto":
            abi.ebb_relation_autotune(dm.ctx, dm.tets, "u", "w", abi.map_opts(mdl, mu0, lam0, precision=prec))
        elif a.planes:
            abi.ebb_relation_set_tuning(dm.ctx, dm.tets, mdl, prec, red, 128, abi.EBB_TUNE_RECORD_PLANES)
        if a.ops == "step":
            # implicit steps (dt 1e-3, rho 1000, rtol 1e-8) from rest, pinned bottom face
            dm.vertex_field("uu", torch.float64)
            dm.vertex_field("vv", torch.float64)
            dm.bind("pinned", torch.from_numpy(dm.rows(m.pinned).astype(np.uint8)).to(dm.device))
            prm = abi.step_params(mdl, 1e-3, 1000.0, mu0, lam0, precision=prec, reduce=red, rtol=1e-8)
            for _ in range(a.iters):
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "uu", "vv", "pinned", prm)
        elif a.ops == "vjp":
            # StVK FP64 (C3's solver settings): one implicit step from rest
            # with a random initial velocity, then the step's VJP at the new
            # velocity (adjoint solve + per-tet VJP map), a few times
            prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu0, lam0, precision=abi.EBB_PREC_F64,
                                  max_iters=4000, rtol=1e-12)
            pin = dm.bind("pinned", torch.from_numpy(dm.rows(m.pinned).astype(np.uint8)).to(dm.device))
            v0 = 0.05 * meshgen.random_field(m.n_verts, seed=seed)
            v0[m.pinned] = 0.0
            dm.vertex_field("uu", torch.float64)
            dm.vertex_field("vv", torch.float64, value=v0)
            dm.vertex_field("u0", torch.float64)
            dm.vertex_field("v0", torch.float64, value=v0)
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "uu", "vv", "pinned", prm)
            gu = dm.vertex_field("gu", torch.float64)
            gv = dm.vertex_field("gv", torch.float64)
            gmu = dm.bind_tets("gmu", torch.zeros(m.n_tets, dtype=torch.float64, device=pin.device))
            glam = dm.bind_tets("glam", torch.zeros(m.n_tets, dtype=torch.float64, device=pin.device))
            for _ in range(a.iters):
                gu.copy_(dm._tensors["uu"])
                gv.zero_()
                abi.ebb_cg_implicit_step_vjp_at(dm.ctx, dm.tets, "u0", "v0", "vv", "pinned", "gu", "gv", "gmu",
                                                "glam", prm)
        elif a.ops == "spmv":
            # K(u) assembled once, then the block-sparse product K w
            abi.ebb_assemble_tet_K(dm.ctx, dm.tets, "u", o)
            for _ in range(a.iters):
                abi.ebb_spmv_tet_K(dm.ctx, dm.tets, "w", "k", o)
        elif a.ops == "springs":
            # spring-mass steps (K = 1, dt = 1e-4, equal masses) from a perturbed rest state
            dm.vertex_field("pos", dt, value=m.X)
            dm.vertex_field("q", dt, value=m.X + 0.002 * np.asarray(w))
            dm.vertex_field("qd", dt)
            dm.vertex_field("mass", dt, ncomp=1, value=np.full(m.n_verts, 1000.0 / m.n_verts))
            abi.ebb_springs_init(dm.ctx, dm.tets, "pos")
            abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "mass", 1.0, 1e-4, a.iters)
        else:
            for _ in range(a.iters):
                if a.ops == "fused":
                    abi.ebb_map_tet_force_Kv(dm.ctx, dm.tets, "u", "w", "f", "k", o)
                elif a.ops == "kv":
                    abi.ebb_map_tet_Kv(dm.ctx, dm.tets, "u", "w", "k", o)
                elif a.ops == "force":
                    abi.ebb_map_tet_forces(dm.ctx, dm.tets, "u", "f", o)
                else:
                    abi.ebb_map_tet_diagK(dm.ctx, dm.tets, "u", "k", o)
        abi.ebb_ctx_sync(dm.ctx)
    print("ok", m.n_tets)


# ---- main line ----------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1506_07577_gb300 import abi

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    head = run_headline(args, abi, torch, dev, local_rank, stream, flush, dist, world, barrier)
    nt, nv = head["n_tets"], head["n_verts"]
    sub = {}
    nh64 = bat = adj = c1 = None
    if not args.headline_only:
        sub["nh64"], nh64 = run_nh64(args, abi, torch, local_rank, stream, flush)
        if args.batch_meshes > 0:
            sub["batched_step"], bat = batched_steps(abi, torch, local_rank, args)
        if not args.no_adjoint:
            sub["adjoint_rollout"], adj = adjoint_rollout(abi, torch, local_rank, args)
        sub["small_configs"], c1 = small_configs(abi, torch, local_rank, stream)

    peak, peak_kind = _peaks()
    bpt = algorithmic_bytes_per_tet(nv, nt, False)
    kern_s = head["kern_us"] * 1e-6
    achieved = bpt * nt / kern_s / 1e9
    tune = head["tune"]
    fresh = NCU_TRAFFIC["sources_sha256_16"] == kernel_sources_hash()
    captured = fresh and args.n == NCU_TRAFFIC["n"] and tune["reduce"] == "tiled" and tune["tile_tets"] == 128
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": NCU_TRAFFIC["bytes_per_launch"][tune["records"]] if captured else None,
            "traffic_unit": "bytes per launch (ncu dram read+write)",
            "kernel": {"tiled": "tet_tile_kernel<float, STVK, FORCE|KV, interleaved>",
                       "atomic": "tet_map_kernel<float, STVK, FORCE|KV, atomic, interleaved>",
                       "colour": "tet_map_kernel<float, STVK, FORCE|KV, coloured, interleaved>",
                       "gather": "tet_corner_kernel + vertex_sum_kernel",
                       "tiled_ordered": "tet_tile_kernel (partial rows) + partial_sum_kernel",
                       "coop": "tet_coop_kernel<float, STVK, FORCE|KV, interleaved>"}[tune["reduce"]],
            "algorithmic_bytes_per_tet": bpt, "kernel_us": head["kern_us"], "peak_kind": peak_kind}
    if not fresh:
        roof["traffic_note"] = "no ncu capture of the current kernel sources"
    elif not captured:
        roof["traffic_note"] = "ncu traffic was captured for the tiled kernel with 128-tet tiles on the 128^3 mesh only"
    else:
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of the same kernel "
                                  "and record layout on the same mesh")
    if rank != 0:
        return
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * head["total_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.n}^3 cube grid, 5 tets/cube ({nv:,} verts, {nt:,} tets), vertex and tet "
                                   "ids randomly permuted (seed 5) and renumbered by the library at finalize "
                                   "(Morton order; fields loaded into that row order once, untimed), StVK E 1e5 "
                                   "nu 0.45, FP32 fused force+K*w map, reduction variant and tile size from the "
                                   "autotuner, vector fields stored as 4-float elements",
                       "n_tets": nt, "n_verts": nv, "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof,
            "e2e": head["e2e"],
            "gpu_launches": args.steps * head["launches_per_step"],
            "clocks": head["clocks"],
            "autotune": tune,
            "layout": {"tiles": head["ntiles"], "colours": head["ncolours"],
                       "finalize_renumbered_with_colouring_s": head["setup_s"],
                       "finalize_with_vertex_reorder_s": head["setup_vertex_reorder_s"]},
            "reduction_variants": head["variants"]}
    line.update(sub)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, head, nh64, bat, adj, c1)
    print(json.dumps(line), flush=True)


def run_host_link(argv):
    """Page-locked host <-> device copy bandwidth for copies of the headline
    end-to-end call's size (the 4-float u and w of the 128^3 mesh, 34.3 MB
    each) and of 4x that: host to device alone, device to host alone, and
    both directions at once on two streams.  CUDA events, median of 10 after
    3 warm-up copies; prints one line.

        python bench.py --host-link"""
    import torch

    out = {"metric": "page-locked host link bandwidth", "unit": "GB/s", "sizes": {}}
    dev = torch.device("cuda", 0)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    for nbytes in (2146689 * 16, 4 * 2146689 * 16):
        n = nbytes // 4
        h_in = torch.empty(n, dtype=torch.float32).pin_memory()
        h_out = torch.empty(n, dtype=torch.float32).pin_memory()
        d_in = torch.empty(n, dtype=torch.float32, device=dev)
        d_out = torch.zeros(n, dtype=torch.float32, device=dev)

        def timed(fn):
            ts = []
            for it in range(13):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s1)
                fn()
                s1.wait_stream(s2)
                b.record(s1)
                b.synchronize()
                if it >= 3:
                    ts.append(a.elapsed_time(b) * 1e-3)
            return statistics.median(ts)

        def h2d():
            with torch.cuda.stream(s1):
                d_in.copy_(h_in, non_blocking=True)

        def d2h():
            with torch.cuda.stream(s1):
                h_out.copy_(d_out, non_blocking=True)

        def both():
            s2.wait_stream(s1)
            with torch.cuda.stream(s1):
                d_in.copy_(h_in, non_blocking=True)
            with torch.cuda.stream(s2):
                h_out.copy_(d_out, non_blocking=True)

        t_h2d, t_d2h, t_both = timed(h2d), timed(d2h), timed(both)
        out["sizes"][str(nbytes)] = {"h2d_GBps": nbytes / t_h2d / 1e9, "d2h_GBps": nbytes / t_d2h / 1e9,
                                     "both_directions_GBps_each": nbytes / t_both / 1e9}
    print(json.dumps(out), flush=True)


def main():
    if "--profile" in sys.argv[1:]:
        run_profile([a for a in sys.argv[1:]])
        return
    if "--host-link" in sys.argv[1:]:
        run_host_link(sys.argv[1:])
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=128, help="cube-grid side of the headline workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="skip the 64^3, batched and adjoint sub-records")
    ap.add_argument("--implicit-steps", type=int, default=10)
    ap.add_argument("--batch-meshes", type=int, default=256)
    ap.add_argument("--no-adjoint", action="store_true")
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
