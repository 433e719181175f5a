"""Device-resident tet mesh: torch-owned field storage bound to the C ABI.

PyTorch supplies device memory and the stream; every computation runs in
``libebb_gb300.so`` through the calls in ``abi``.  Vertex fields are stored
as column stores shaped (3, N_v) (one contiguous plane per component,
Section 6.1), the tet key-field ``v`` as (4, N_t) int32.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi


class DeviceTetMesh:
    """Relations ``verts``/``tets`` on one CUDA device with the rest shape,
    keys, optional per-tet Lame fields and optional per-vertex batch ids
    bound, finalized on construction."""

    def __init__(self, X, tets, mu=None, lam=None, device=0, stream=None, colour=False, batch=None,
                 reorder_verts=False, edges=False, renumber_verts=False):
        self.device = torch.device("cuda", device)
        self.ctx = abi.ebb_ctx_create(device, stream)
        self.n_verts = int(X.shape[0])
        self.n_tets = int(tets.shape[0])
        self.verts = abi.ebb_relation_create(self.ctx, "verts", self.n_verts)
        self.tets = abi.ebb_relation_create(self.ctx, "tets", self.n_tets)
        self._tensors = {}
        self.X = self._put("X", np.ascontiguousarray(np.asarray(X, np.float64).T), self.verts)
        keys = np.ascontiguousarray(np.asarray(tets, np.int32).T)
        self.keys = torch.from_numpy(keys).to(self.device)
        abi.ebb_field_bind(self.ctx, self.tets, "v", self.keys, key_target=self.verts)
        if (mu is None) != (lam is None):
            raise ValueError("give both per-tet mu and lam, or neither")
        if mu is not None and np.ndim(mu) > 0:
            self._put("mu", np.asarray(mu, np.float64), self.tets)
            self._put("lambda", np.asarray(lam, np.float64), self.tets)
        if batch is not None:
            self.batch = self._put("batch", np.asarray(batch, np.int32), self.verts)
        # uploads ran on torch's current stream; the library may use another
        torch.cuda.synchronize(self.device)
        flags = ((abi.EBB_FINALIZE_COLOR if colour else 0) | (abi.EBB_FINALIZE_REORDER_VERTS if reorder_verts else 0) |
                 (abi.EBB_FINALIZE_EDGES if edges else 0) | (abi.EBB_FINALIZE_RENUMBER_VERTS if renumber_verts else 0))
        abi.ebb_relation_finalize(self.ctx, self.tets, flags)
        # Row order of vertex fields: identity unless the relation renumbered
        # its vertices (then row i holds the caller's vertex order[i]).
        self.renumbered = bool(renumber_verts)
        self.order = abi.ebb_relation_vertex_order(self.ctx, self.tets, self.n_verts)

    def rows(self, arr):
        """A per-vertex array (N_v, ...) in the caller's vertex order, put in
        the relation's row order."""
        return np.asarray(arr)[self.order] if self.renumbered else np.asarray(arr)

    def caller(self, arr):
        """A per-vertex array (N_v, ...) in the relation's row order, put
        back in the caller's vertex order."""
        arr = np.asarray(arr)
        if not self.renumbered:
            return arr
        out = np.empty_like(arr)
        out[self.order] = arr
        return out

    def _put(self, name, arr, rel):
        t = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device)
        abi.ebb_field_bind(self.ctx, rel, name, t)
        self._tensors[name] = t
        return t

    def vertex_field(self, name, dtype=torch.float64, ncomp=3, value=None, x4=False):
        """Allocate (or upload) a vertex field of shape (ncomp, N_v), bind it
        under ``name`` and return the tensor.  ``value`` may be an (N_v, ncomp)
        numpy array.  With ``x4`` the field is an EBB_F32X4 field: a float32
        tensor of shape (N_v, 4) whose first three columns hold the vectors.
        ``value`` is given in the caller's vertex order; on a relation that
        renumbered its vertices it is stored in the relation's row order."""
        if value is not None:
            value = self.rows(value)
        if x4:
            t = torch.zeros((self.n_verts, 4), dtype=torch.float32, device=self.device)
            if value is not None:
                t[:, :3] = torch.from_numpy(np.ascontiguousarray(np.asarray(value, dtype=np.float32))).to(self.device)
            torch.cuda.synchronize(self.device)
            abi.ebb_field_bind(self.ctx, self.verts, name, t, x4=True)
            self._tensors[name] = t
            return t
        if value is not None:
            arr = np.asarray(value)
            arr = arr.T if arr.ndim == 2 else arr
            t = torch.from_numpy(np.ascontiguousarray(arr)).to(self.device, dtype)
        else:
            shape = (ncomp, self.n_verts) if ncomp > 1 else (self.n_verts,)
            t = torch.zeros(shape, dtype=dtype, device=self.device)
        torch.cuda.synchronize(self.device)
        abi.ebb_field_bind(self.ctx, self.verts, name, t)
        self._tensors[name] = t
        return t

    def bind(self, name, tensor):
        """Bind an existing CUDA tensor as a vertex field."""
        abi.ebb_field_bind(self.ctx, self.verts, name, tensor)
        self._tensors[name] = tensor
        return tensor

    def bind_tets(self, name, tensor):
        """Bind an existing CUDA tensor as a field of the tets relation."""
        abi.ebb_field_bind(self.ctx, self.tets, name, tensor)
        self._tensors[name] = tensor
        return tensor

    def close(self):
        if self.ctx is not None:
            abi.ebb_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
