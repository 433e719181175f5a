"""Run one element map (or the assembled K, or the spring-mass steps) a few
times on a cube-grid workload (for profilers).

    python -m paper_1506_07577_gb300.profile_maps --n 64 --variant tiled --ops fused

Builds the n^3 cube grid (5 tets per cube, 1% jitter, neo-Hookean with E
log-uniform in [1e4, 1e6], nu = 0.4 by default), binds it, and calls the
chosen map `--iters` times through the C ABI.  It prints nothing but a final
line with the tet count; use it under ncu to capture the map kernel alone.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import numpy as np
    import torch

    import meshgen
    from paper_1506_07577_gb300 import abi
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--variant", choices=["atomic", "tiled", "colour", "gather", "ordered"], default="tiled")
    ap.add_argument("--ops", choices=["fused", "kv", "force", "diag", "step", "spmv", "springs"], default="fused")
    ap.add_argument("--prec", choices=["f32", "f64"], default="f32")
    ap.add_argument("--model", choices=["nh", "stvk"], default="nh")
    ap.add_argument("--permute", action="store_true")
    ap.add_argument("--x4", action="store_true", help="FP32 vector fields as EBB_F32X4 elements")
    ap.add_argument("--iters", type=int, default=3)
    a = ap.parse_args(argv)

    m = meshgen.cube_grid(a.n, jitter=0.01, seed=2, permute=a.permute)
    mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, 2)
    u = meshgen.random_displacement(m.X, a.n, amp=0.05, seed=2, smooth=0.01)
    w = meshgen.random_field(m.n_verts, seed=2)
    dt = torch.float32 if a.prec == "f32" else torch.float64
    mdl = abi.EBB_NEOHOOKEAN if a.model == "nh" else abi.EBB_STVK
    red = {"atomic": abi.EBB_REDUCE_ATOMIC, "tiled": abi.EBB_REDUCE_TILED, "colour": abi.EBB_REDUCE_COLOR,
           "gather": abi.EBB_REDUCE_GATHER, "ordered": abi.EBB_REDUCE_TILED_ORDERED}[a.variant]
    with DeviceTetMesh(m.X, m.tets, mu, lam, colour=(a.variant == "colour"),
                       edges=a.ops in ("spmv", "springs")) as dm:
        x4 = a.x4 and a.prec == "f32"
        dm.vertex_field("u", dt, value=u, x4=x4)
        dm.vertex_field("w", dt, value=w, x4=x4)
        dm.vertex_field("f", dt, x4=x4)
        dm.vertex_field("k", dt, x4=x4)
        o = abi.map_opts(mdl, precision=abi.EBB_PREC_F32 if a.prec == "f32" else abi.EBB_PREC_F64, reduce=red,
                         flags=abi.EBB_MAP_ZERO_OUT)
        if a.ops == "step":
            # implicit steps (dt 1e-3, rho 1000, rtol 1e-8) from rest, pinned bottom face
            dm.vertex_field("uu", torch.float64)
            dm.vertex_field("vv", torch.float64)
            dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dm.device))
            prm = abi.step_params(mdl, 1e-3, 1000.0, precision=abi.EBB_PREC_F32 if a.prec == "f32" else abi.EBB_PREC_F64,
                                  reduce=red, rtol=1e-8)
            for _ in range(a.iters):
                abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "uu", "vv", "pinned", prm)
        if a.ops == "spmv":
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
        for _ in range(a.iters if a.ops not in ("step", "spmv", "springs") else 0):
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


if __name__ == "__main__":
    main()
