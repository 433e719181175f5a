"""Thin ctypes binding of the C ABI in ``include/ebb.h`` (same names).

Argument marshalling only: every step of the tet path runs in the CUDA
library ``libebb_gb300.so``.  There is no fallback: importing this module
without the built library raises ``ImportError``.  Device memory comes from
PyTorch tensors (their ``data_ptr()`` is handed to the library, which borrows
it); the stream is a ``torch.cuda.Stream`` or ``None`` (legacy default).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libebb_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the tet FEM path has no CPU fallback)")

_lib = C.CDLL(LIB_PATH)

# ---- constants (mirror include/ebb.h) ------------------------------------
EBB_OK = 0
EBB_ERR_ARG = 1
EBB_ERR_KEY = 2
EBB_ERR_PHASE = 3
EBB_ERR_INVERTED = 4
EBB_ERR_CG_BREAKDOWN = 5
EBB_ERR_NOT_CONVERGED = 6
EBB_ERR_TIMEOUT = 7
EBB_ERR_CUDA = 8
EBB_ERR_STATE = 9
EBB_ERR_NOMEM = 10
STATUS_NAMES = {v: k for k, v in dict(globals()).items() if k.startswith("EBB_ERR_") or k == "EBB_OK"}

EBB_F32, EBB_F64, EBB_I32, EBB_U8, EBB_F32X4 = 1, 2, 3, 4, 5
EBB_STVK, EBB_NEOHOOKEAN = 0, 1
EBB_PREC_F64, EBB_PREC_F32 = 0, 1
EBB_REDUCE_ATOMIC, EBB_REDUCE_COLOR, EBB_REDUCE_AUTO, EBB_REDUCE_TILED, EBB_REDUCE_GATHER = 0, 1, 2, 3, 4
EBB_REDUCE_TILED_ORDERED = 5
EBB_REDUCE_COOP = 6
EBB_FINALIZE_COLOR = 1
EBB_FINALIZE_REORDER_VERTS = 2
EBB_FINALIZE_EDGES = 4
EBB_FINALIZE_RENUMBER_VERTS = 8
EBB_STEP_ASSEMBLED = 1
EBB_MAP_ZERO_OUT = 1
EBB_MAP_HOST_XYZ = 2
EBB_MAP_TEST_DROP_TILE = 0x80000000
EBB_NOALLOC_MAX_VERTS = 4096
EBB_NOALLOC_MAX_TETS = 24576

ebb_ctx_t = C.c_void_p
ebb_rel_t = C.c_void_p
ebb_status_t = C.c_int32


class ebb_map_opts_t(C.Structure):
    _fields_ = [("model", C.c_int), ("mu", C.c_double), ("lambda_", C.c_double),
                ("precision", C.c_int), ("reduce", C.c_int), ("flags", C.c_uint32)]


class ebb_step_params_t(C.Structure):
    _fields_ = [("model", C.c_int), ("mu", C.c_double), ("lambda_", C.c_double),
                ("precision", C.c_int), ("reduce", C.c_int), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("rho", C.c_double), ("max_iters", C.c_int32),
                ("rtol", C.c_double), ("fail_on_max_iters", C.c_int32), ("flags", C.c_uint32)]


EBB_AUTOTUNE_MAX_CAND = 12
EBB_TUNE_INTERLEAVED = 1
EBB_TUNE_RECORD_PLANES = 2


class ebb_autotune_cand_t(C.Structure):
    _fields_ = [("reduce", C.c_int32), ("tile_tets", C.c_int32), ("interleaved", C.c_int32),
                ("record_planes", C.c_int32), ("us", C.c_double)]


class ebb_autotune_report_t(C.Structure):
    _fields_ = [("reduce", C.c_int32), ("tile_tets", C.c_int32), ("interleaved", C.c_int32),
                ("record_planes", C.c_int32), ("ncand", C.c_int32),
                ("cand", ebb_autotune_cand_t * EBB_AUTOTUNE_MAX_CAND)]


class ebb_cg_report_t(C.Structure):
    _fields_ = [("iters", C.c_int32), ("rel_residual", C.c_double), ("status", C.c_int32)]


class ebb_relation_info_t(C.Structure):
    _fields_ = [("n_tets", C.c_int64), ("n_verts", C.c_int64), ("ntiles", C.c_int32), ("tile_tets", C.c_int32),
                ("ncolours", C.c_int32), ("interleaved", C.c_int32), ("reordered", C.c_int32),
                ("record_planes", C.c_int32), ("tuned", (C.c_int32 * 2) * 2)]


_P = C.c_char_p
_SIGS = {
    "ebb_ctx_create": ([C.POINTER(ebb_ctx_t), C.c_int, C.c_void_p], ebb_status_t),
    "ebb_ctx_set_stream": ([ebb_ctx_t, C.c_void_p], ebb_status_t),
    "ebb_ctx_destroy": ([ebb_ctx_t], ebb_status_t),
    "ebb_ctx_sync": ([ebb_ctx_t], ebb_status_t),
    "ebb_last_error": ([ebb_ctx_t], C.c_char_p),
    "ebb_relation_create": ([ebb_ctx_t, _P, C.c_int64, C.POINTER(ebb_rel_t)], ebb_status_t),
    "ebb_field_bind": ([ebb_rel_t, _P, C.c_int, C.c_int32, C.c_void_p, ebb_rel_t], ebb_status_t),
    "ebb_relation_finalize": ([ebb_rel_t, C.c_uint32], ebb_status_t),
    "ebb_map_tet_forces": ([ebb_ctx_t, ebb_rel_t, _P, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_map_tet_Kv": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_map_tet_force_Kv": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_map_tet_force_Kv_host": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, _P, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_map_tet_diagK": ([ebb_ctx_t, ebb_rel_t, _P, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_assemble_tet_K": ([ebb_ctx_t, ebb_rel_t, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_spmv_tet_K": ([ebb_ctx_t, ebb_rel_t, _P, _P, C.POINTER(ebb_map_opts_t)], ebb_status_t),
    "ebb_springs_init": ([ebb_ctx_t, ebb_rel_t, _P], ebb_status_t),
    "ebb_springs_run": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, C.c_double, C.c_double, C.c_int32,
                         C.POINTER(C.c_double)], ebb_status_t),
    "ebb_relation_autotune": ([ebb_ctx_t, ebb_rel_t, _P, _P, C.POINTER(ebb_map_opts_t),
                               C.POINTER(ebb_autotune_report_t)], ebb_status_t),
    "ebb_relation_set_tuning": ([ebb_ctx_t, ebb_rel_t, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
                                ebb_status_t),
    "ebb_relation_info": ([ebb_ctx_t, ebb_rel_t, C.POINTER(ebb_relation_info_t)], ebb_status_t),
    "ebb_relation_vertex_order": ([ebb_ctx_t, ebb_rel_t, C.c_void_p, C.c_int64], ebb_status_t),
    "ebb_cg_implicit_step": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, C.POINTER(ebb_step_params_t),
                              C.POINTER(ebb_cg_report_t)], ebb_status_t),
    "ebb_cg_implicit_step_vjp": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, _P, _P, _P, _P, C.POINTER(ebb_step_params_t),
                                  C.POINTER(ebb_cg_report_t)], ebb_status_t),
    "ebb_cg_implicit_step_vjp_at": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, _P, _P, _P, _P, _P,
                                     C.POINTER(ebb_step_params_t), C.POINTER(ebb_cg_report_t)], ebb_status_t),
    "ebb_cg_implicit_step_batched": ([ebb_ctx_t, ebb_rel_t, _P, _P, _P, _P, C.c_int32,
                                      C.POINTER(ebb_step_params_t), C.POINTER(ebb_cg_report_t)], ebb_status_t),
    "ebb_cg_implicit_step_noalloc": ([C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(ebb_step_params_t),
                                      C.POINTER(ebb_cg_report_t)], ebb_status_t),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

EXPORTED = tuple(_SIGS)


class EbbError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


def _b(s):
    return None if s is None else s.encode()


def _check(ctx, status):
    if status != EBB_OK:
        msg = _lib.ebb_last_error(ctx).decode() if ctx else ""
        raise EbbError(status, msg)
    return status


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ---- same-name wrappers ----------------------------------------------------
def ebb_ctx_create(device=0, stream=None):
    h = ebb_ctx_t()
    st = _lib.ebb_ctx_create(C.byref(h), int(device), _stream_handle(stream))
    if st != EBB_OK:
        raise EbbError(st, "ebb_ctx_create failed")
    return h


def ebb_ctx_set_stream(ctx, stream):
    return _check(ctx, _lib.ebb_ctx_set_stream(ctx, _stream_handle(stream)))


def ebb_ctx_destroy(ctx):
    return _lib.ebb_ctx_destroy(ctx)


def ebb_ctx_sync(ctx):
    return _check(ctx, _lib.ebb_ctx_sync(ctx))


def ebb_last_error(ctx):
    return _lib.ebb_last_error(ctx).decode()


def ebb_relation_create(ctx, name, size):
    h = ebb_rel_t()
    _check(ctx, _lib.ebb_relation_create(ctx, _b(name), int(size), C.byref(h)))
    return h


_DT = {"torch.float32": EBB_F32, "torch.float64": EBB_F64, "torch.int32": EBB_I32, "torch.uint8": EBB_U8}


def ebb_field_bind(ctx, rel, name, tensor, key_target=None, x4=False):
    """Bind a CUDA tensor shaped (ncomp, rows) or (rows,) as a column-store
    field (ncomp contiguous planes), or with ``x4`` a float32 tensor shaped
    (rows, 4) as an EBB_F32X4 field of 3-vectors (x, y, z, padding).  The
    tensor must stay alive while bound."""
    if not tensor.is_cuda or not tensor.is_contiguous():
        raise ValueError("fields must be contiguous CUDA tensors")
    if x4:
        if str(tensor.dtype) != "torch.float32" or tensor.dim() != 2 or int(tensor.shape[1]) != 4:
            raise ValueError("EBB_F32X4 fields are float32 tensors shaped (rows, 4)")
        return _check(ctx, _lib.ebb_field_bind(rel, _b(name), EBB_F32X4, 3, C.c_void_p(tensor.data_ptr()),
                                               key_target))
    dt = _DT.get(str(tensor.dtype))
    if dt is None:
        raise ValueError(f"unsupported dtype {tensor.dtype}")
    ncomp = 1 if tensor.dim() == 1 else int(tensor.shape[0])
    return _check(ctx, _lib.ebb_field_bind(rel, _b(name), dt, ncomp, C.c_void_p(tensor.data_ptr()), key_target))


def ebb_relation_finalize(ctx, rel, flags=0):
    return _check(ctx, _lib.ebb_relation_finalize(rel, int(flags)))


def map_opts(model, mu=0.0, lam=0.0, precision=EBB_PREC_F64, reduce=EBB_REDUCE_AUTO, flags=0):
    return ebb_map_opts_t(int(model), float(mu), float(lam), int(precision), int(reduce), int(flags))


def ebb_map_tet_forces(ctx, tets, u, f_out, opts):
    return _check(ctx, _lib.ebb_map_tet_forces(ctx, tets, _b(u), _b(f_out), C.byref(opts)))


def ebb_map_tet_Kv(ctx, tets, u, w, Kw_out, opts):
    return _check(ctx, _lib.ebb_map_tet_Kv(ctx, tets, _b(u), _b(w), _b(Kw_out), C.byref(opts)))


def ebb_map_tet_force_Kv(ctx, tets, u, w, f_out, Kw_out, opts):
    return _check(ctx, _lib.ebb_map_tet_force_Kv(ctx, tets, _b(u), _b(w), _b(f_out), _b(Kw_out), C.byref(opts)))


def _host_ptr(buf):
    """Address of a contiguous host buffer: a CPU torch tensor or a numpy array
    (None passes a null pointer)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if buf.is_cuda or not buf.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        return buf.data_ptr()
    if not buf.flags["C_CONTIGUOUS"]:
        raise ValueError("host buffers must be C-contiguous arrays")
    return buf.ctypes.data


def ebb_map_tet_force_Kv_host(ctx, tets, u, w, f_out, Kw_out, u_host, w_host, f_host, Kw_host, opts):
    """The fused map on host buffers (each the exact bytes of its field)."""
    return _check(ctx, _lib.ebb_map_tet_force_Kv_host(ctx, tets, _b(u), _b(w), _b(f_out), _b(Kw_out),
                                                       _host_ptr(u_host), _host_ptr(w_host), _host_ptr(f_host),
                                                       _host_ptr(Kw_host), C.byref(opts)))


def ebb_map_tet_diagK(ctx, tets, u, d_out, opts):
    return _check(ctx, _lib.ebb_map_tet_diagK(ctx, tets, _b(u), _b(d_out), C.byref(opts)))


def ebb_assemble_tet_K(ctx, tets, u, opts):
    return _check(ctx, _lib.ebb_assemble_tet_K(ctx, tets, _b(u), C.byref(opts)))


def ebb_spmv_tet_K(ctx, tets, w, Kw_out, opts):
    return _check(ctx, _lib.ebb_spmv_tet_K(ctx, tets, _b(w), _b(Kw_out), C.byref(opts)))


def ebb_springs_init(ctx, tets, pos):
    return _check(ctx, _lib.ebb_springs_init(ctx, tets, _b(pos)))


def ebb_springs_run(ctx, tets, q, qd, mass, k, dt, steps, energy=False):
    """`steps` spring-mass steps in place; returns the kinetic energy after
    them when `energy` is true (synchronous), else None."""
    e = C.c_double(0.0)
    _check(ctx, _lib.ebb_springs_run(ctx, tets, _b(q), _b(qd), _b(mass), float(k), float(dt), int(steps),
                                     C.byref(e) if energy else None))
    return e.value if energy else None


def ebb_relation_autotune(ctx, tets, u, w, opts):
    """Pick the tile size and reduction variant of `tets` by timing the K w
    map; returns the report (chosen variant, tile size, timed candidates)."""
    rep = ebb_autotune_report_t()
    _check(ctx, _lib.ebb_relation_autotune(ctx, tets, _b(u), _b(w), C.byref(opts), C.byref(rep)))
    return rep


def ebb_relation_set_tuning(ctx, tets, model, precision, reduce, tile_tets, flags=0):
    """`flags`: EBB_TUNE_INTERLEAVED | EBB_TUNE_RECORD_PLANES (a bool is
    taken as EBB_TUNE_INTERLEAVED)."""
    return _check(ctx, _lib.ebb_relation_set_tuning(ctx, tets, int(model), int(precision), int(reduce),
                                                    int(tile_tets), int(flags)))


def ebb_relation_info(ctx, tets):
    """Layout of a finalized tets relation (tiles, colours, staging, tuning)."""
    info = ebb_relation_info_t()
    _check(ctx, _lib.ebb_relation_info(ctx, tets, C.byref(info)))
    return info


def ebb_relation_vertex_order(ctx, tets, n_verts):
    """Row order of the verts relation: numpy int32 array, entry i = the
    caller's vertex held in row i of every vertex field."""
    import numpy as np
    order = np.empty(int(n_verts), dtype=np.int32)
    _check(ctx, _lib.ebb_relation_vertex_order(ctx, tets, C.c_void_p(order.ctypes.data), int(n_verts)))
    return order


def step_params(model, dt, rho, mu=0.0, lam=0.0, gravity=(0.0, 0.0, -9.81), precision=EBB_PREC_F64,
                reduce=EBB_REDUCE_AUTO, max_iters=1000, rtol=1e-8, fail_on_max_iters=False, flags=0):
    g = (C.c_double * 3)(*[float(x) for x in gravity])
    return ebb_step_params_t(int(model), float(mu), float(lam), int(precision), int(reduce), float(dt), g,
                             float(rho), int(max_iters), float(rtol), int(bool(fail_on_max_iters)), int(flags))


def ebb_cg_implicit_step(ctx, tets, u, v, pinned, params):
    rep = ebb_cg_report_t()
    _check(ctx, _lib.ebb_cg_implicit_step(ctx, tets, _b(u), _b(v), _b(pinned), C.byref(params), C.byref(rep)))
    return rep


def ebb_cg_implicit_step_vjp(ctx, tets, u, v, pinned, gu, gv, gmu, glam, params):
    """Adjoint of one step: gu, gv (in dL/du', dL/dv'; out dL/du, dL/dv),
    per-tet dL/dmu, dL/dlambda added into the tets fields gmu, glam."""
    rep = ebb_cg_report_t()
    _check(ctx, _lib.ebb_cg_implicit_step_vjp(ctx, tets, _b(u), _b(v), _b(pinned), _b(gu), _b(gv), _b(gmu),
                                              _b(glam), C.byref(params), C.byref(rep)))
    return rep


def ebb_cg_implicit_step_vjp_at(ctx, tets, u, v, v_next, pinned, gu, gv, gmu, glam, params):
    """The step VJP with the step's new velocity v_next given (no forward
    solve)."""
    rep = ebb_cg_report_t()
    _check(ctx, _lib.ebb_cg_implicit_step_vjp_at(ctx, tets, _b(u), _b(v), _b(v_next), _b(pinned), _b(gu), _b(gv),
                                                 _b(gmu), _b(glam), C.byref(params), C.byref(rep)))
    return rep


def ebb_cg_implicit_step_batched(ctx, tets, u, v, pinned, batch, nbatch, params):
    """One implicit step per mesh of a batch; returns the list of reports."""
    reps = (ebb_cg_report_t * int(nbatch))()
    _check(ctx, _lib.ebb_cg_implicit_step_batched(ctx, tets, _b(u), _b(v), _b(pinned), _b(batch), int(nbatch),
                                                  C.byref(params), reps))
    return list(reps)


def ebb_cg_implicit_step_noalloc(stream, n_verts, n_tets, keys, X, u, v, pinned, params):
    """The allocation-free implicit step.  ``keys`` (4, n_tets) int32, ``X``,
    ``u``, ``v`` (3, n_verts) float64 and ``pinned`` (n_verts,) uint8 or None
    are CUDA tensors; u and v are updated in place.  Raises EbbError on a
    non-zero status (this call has no context, so no message)."""
    def ptr(t):
        return None if t is None else C.c_void_p(t.data_ptr())
    rep = ebb_cg_report_t()
    st = _lib.ebb_cg_implicit_step_noalloc(_stream_handle(stream), int(n_verts), int(n_tets), ptr(keys), ptr(X),
                                           ptr(u), ptr(v), ptr(pinned), C.byref(params), C.byref(rep))
    if st != EBB_OK:
        raise EbbError(st, "ebb_cg_implicit_step_noalloc failed")
    return rep
