"""Differentiable implicit-step rollouts (St. Venant-Kirchhoff, FP64).

``rollout(mesh, u0, v0, mu, lam, steps, params)`` runs ``steps`` implicit
backward-Euler steps through ``ebb_cg_implicit_step`` and returns the final
displacement and velocity as tensors that autograd can differentiate with
respect to the initial state (u0, v0) and the per-tet Lame parameters
(mu, lam).  The backward pass calls the library's step VJP once per step,
newest first.  Only every ``checkpoint_every``-th state is kept in the
forward pass; the states inside a segment are recomputed from its checkpoint
during the backward pass, so memory grows with steps / checkpoint_every
rather than with steps.  Each step's new velocity comes from that replay
(or from the next checkpoint, or the final state), so the VJP is called in
its form that takes it (``ebb_cg_implicit_step_vjp_at``) and solves only the
adjoint system.

The library computes with the per-tet ``mu``/``lambda`` fields that the mesh
was finalized with; the ``mu``, ``lam`` tensors passed here must be those
same values (they are the autograd leaves the gradients are returned for).
"""
from __future__ import annotations

import torch

from . import abi


class _ImplicitRollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, mesh, params, steps, every, pinned, u0, v0, mu, lam):
        u = mesh.bind("_ad_u", u0.detach().clone().contiguous())
        v = mesh.bind("_ad_v", v0.detach().clone().contiguous())
        ckpts = []
        for k in range(steps):
            if k % every == 0:
                ckpts.append((u.clone(), v.clone()))
            abi.ebb_cg_implicit_step(mesh.ctx, mesh.tets, "_ad_u", "_ad_v", pinned, params)
        fctx.mesh, fctx.params, fctx.steps, fctx.every, fctx.pinned = mesh, params, steps, every, pinned
        fctx.ckpts = ckpts
        fctx.vT = v.clone()
        fctx.n_tets = mu.shape[0]
        return u.clone(), v.clone()

    @staticmethod
    def backward(fctx, guT, gvT):
        mesh, params, steps, every, pinned = fctx.mesh, fctx.params, fctx.steps, fctx.every, fctx.pinned
        ref = fctx.ckpts[0][0]
        gu = mesh.bind("_ad_gu", (guT if guT is not None else torch.zeros_like(ref)).detach().clone().contiguous())
        gv = mesh.bind("_ad_gv", (gvT if gvT is not None else torch.zeros_like(ref)).detach().clone().contiguous())
        gmu = mesh.bind_tets("_ad_gmu", torch.zeros(fctx.n_tets, dtype=torch.float64, device=ref.device))
        glam = mesh.bind_tets("_ad_glam", torch.zeros(fctx.n_tets, dtype=torch.float64, device=ref.device))
        su = mesh.bind("_ad_su", torch.empty_like(ref))
        sv = mesh.bind("_ad_sv", torch.empty_like(ref))
        vn = mesh.bind("_ad_vn", torch.empty_like(ref))
        for seg in range(len(fctx.ckpts) - 1, -1, -1):
            start = seg * every
            end = min(start + every, steps)
            su.copy_(fctx.ckpts[seg][0])
            sv.copy_(fctx.ckpts[seg][1])
            states = []
            for k in range(start, end):
                states.append((su.clone(), sv.clone()))
                if k < end - 1:
                    abi.ebb_cg_implicit_step(mesh.ctx, mesh.tets, "_ad_su", "_ad_sv", pinned, params)
            # velocity at the segment's end: the next checkpoint's, or the final one
            v_end = fctx.ckpts[seg + 1][1] if seg + 1 < len(fctx.ckpts) else fctx.vT
            for k in range(end - 1, start - 1, -1):
                su.copy_(states[k - start][0])
                sv.copy_(states[k - start][1])
                vn.copy_(states[k + 1 - start][1] if k < end - 1 else v_end)
                abi.ebb_cg_implicit_step_vjp_at(mesh.ctx, mesh.tets, "_ad_su", "_ad_sv", "_ad_vn", pinned, "_ad_gu",
                                                "_ad_gv", "_ad_gmu", "_ad_glam", params)
        return None, None, None, None, None, gu.clone(), gv.clone(), gmu.clone(), glam.clone()


def rollout(mesh, u0, v0, mu, lam, steps, params, checkpoint_every=5, pinned="pinned"):
    """Run `steps` implicit steps from (u0, v0); returns (u_T, v_T).
    u0, v0: (3, N_v) float64 CUDA tensors; mu, lam: (N_t,) float64 CUDA
    tensors equal to the per-tet values the mesh was finalized with.
    `params` must be an FP64 StVK ebb_step_params_t."""
    if params.model != abi.EBB_STVK or params.precision != abi.EBB_PREC_F64:
        raise ValueError("differentiable rollouts support StVK in FP64")
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    return _ImplicitRollout.apply(mesh, params, int(steps), int(checkpoint_every), pinned, u0, v0, mu, lam)
