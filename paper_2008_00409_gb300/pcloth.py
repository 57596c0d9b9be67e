"""Thin Python binding of libpcloth (include/pcloth.h), same entry-point names.

Argument marshalling only: every step of the hot path runs in the CUDA library. PyTorch
supplies device memory and the current stream. Importing this module loads the library
and raises if it has not been built (``paper_2008_00409_gb300.build.build()``); there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

c_int32, c_int64, c_float, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_void_p

PC_OK, PC_ERR_ARG, PC_ERR_CAPACITY, PC_ERR_NOT_CONVERGED, PC_ERR_NONFINITE, PC_ERR_TIMEOUT, PC_ERR_CUDA, PC_ERR_MESH = range(8)
PC_PREC_FP32, PC_PREC_MIXED = 0, 1
PC_PRECOND_JACOBI, PC_PRECOND_BLOCK = 0, 1
PC_STORAGE_SYM, PC_STORAGE_FULL, PC_STORAGE_SELL, PC_STORAGE_OFFDIAG = 0, 1, 2, 3
PC_SCHED_AUTO, PC_SCHED_GRID, PC_SCHED_CLUSTER = 0, 1, 2
PC_WARM_ZERO, PC_WARM_PREV, PC_WARM_GIVEN, PC_WARM_MLP, PC_WARM_COMBINED = 0, 1, 2, 3, 4
PC_MLP_IN, PC_MLP_HIDDEN, PC_MLP_OUT, PC_MLP_NPARAMS, PC_MLP_NSTATS = 12, 64, 3, 5187, 30


class pc_material(ctypes.Structure):
    _fields_ = [("rho", c_float), ("young", c_float), ("poisson", c_float), ("k_bend", c_float),
                ("k_contact", c_float), ("gravity", c_float * 3), ("damp_mass", c_float), ("damp_stiff", c_float),
                ("contact_thickness", c_float)]


class pc_contacts(ctypes.Structure):
    _fields_ = [("n", c_int32), ("pairs", c_void_p), ("w", c_void_p)]


class pc_bsr(ctypes.Structure):
    _fields_ = [("row_ptr", c_void_p), ("col_idx", c_void_p), ("cap", c_int64), ("nnzb", c_int64)]


class pc_solve_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int32), ("precision", c_int32), ("refresh", c_double),
                ("refresh_every", c_int32), ("check_every", c_int32), ("precond", c_int32), ("storage", c_int32),
                ("fuse", c_int32), ("schedule", c_int32)]


class pc_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("outer", c_int32), ("rel_res", c_double), ("bnorm", c_double)]

    def as_dict(self):
        return {"iters": self.iters, "outer": self.outer, "rel_res": self.rel_res, "bnorm": self.bnorm}


class pc_step_opts(ctypes.Structure):
    _fields_ = [("h", c_float), ("solve", pc_solve_opts), ("warm_start", c_int32), ("feat_out", c_void_p)]


class pc_step_info(ctypes.Structure):
    _fields_ = [("nnzb", c_int64), ("solve", pc_solve_info), ("guess", c_int32), ("pad", c_int32),
                ("guess_res", c_double * 3), ("guess_energy", c_double * 3), ("guess_coef", c_double * 2),
                ("combo_energy", c_double)]


class pc_adam_opts(ctypes.Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float)]


class PcError(RuntimeError):
    def __init__(self, status: int, what: str, required: int | None = None):
        self.status = status
        self.required = required
        msg = f"{what}: {_lib.pc_status_string(status).decode()} (status {status})"
        if status == PC_ERR_CUDA:
            msg += f" [{_lib.pc_last_cuda_error().decode()}]"
        super().__init__(msg)


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libpcloth.so is not built ({path}); run paper_2008_00409_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.pc_status_string.restype = ctypes.c_char_p
    L.pc_status_string.argtypes = [c_int32]
    L.pc_last_cuda_error.restype = ctypes.c_char_p
    L.pc_last_cuda_error.argtypes = []
    L.pc_default_solve_opts.argtypes = [P(pc_solve_opts)]
    L.pc_default_solve_opts.restype = None
    L.pc_create.argtypes = [P(c_void_p), c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_int32, P(pc_material),
                            c_int32, c_void_p]
    L.pc_destroy.argtypes = [c_void_p]
    L.pc_get_sizes.argtypes = [c_void_p, P(c_int32), P(c_int32), P(c_int32), P(c_int64)]
    L.pc_get_rest.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.pc_assemble_pattern.argtypes = [c_void_p, P(pc_contacts), P(pc_bsr), c_void_p]
    L.pc_assemble_values.argtypes = [c_void_p, P(pc_bsr), c_void_p, c_void_p, P(pc_contacts), c_float, c_void_p,
                                     c_void_p, c_void_p, c_void_p]
    L.pc_bsr_spmv.argtypes = [c_void_p, P(pc_bsr), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.pc_pcg_solve.argtypes = [c_void_p, P(pc_bsr), c_void_p, c_void_p, c_void_p, c_void_p, P(pc_solve_opts),
                               P(pc_solve_info), c_void_p]
    L.pc_pcg_solve_static.argtypes = [c_int32, P(pc_bsr), c_void_p, c_void_p, c_void_p, c_void_p,
                                      P(pc_solve_opts), P(pc_solve_info), c_void_p]
    L.pc_step.argtypes = [c_void_p, c_void_p, c_void_p, P(pc_contacts), P(pc_step_opts), c_void_p, P(pc_step_info),
                          c_void_p]
    L.pc_pcg_solve_batched.argtypes = [c_void_p, P(pc_bsr), c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                       c_void_p, P(pc_solve_opts), c_void_p, c_void_p]
    L.pc_step_batched.argtypes = [c_void_p, c_void_p, c_void_p, P(pc_contacts), c_int32, c_void_p, P(pc_step_opts),
                                  c_void_p, c_void_p]
    L.pc_batched_config.argtypes = [c_void_p, P(c_int32), P(c_int32), P(c_int32), c_void_p, c_void_p]
    L.pc_set_barrier_wait.argtypes = [c_void_p, c_int64]
    L.pc_get_prev_dv.argtypes = [c_void_p, c_void_p, P(c_int32), c_void_p]
    L.pc_set_prev_dv.argtypes = [c_void_p, c_void_p, c_void_p]
    L.pc_mlp_get_state.argtypes = [c_void_p, c_void_p, c_void_p, P(c_int64), c_void_p]
    L.pc_mlp_set_state.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]
    L.pc_proximity_query.argtypes = [c_void_p, c_void_p, c_float, c_int32, c_void_p, c_void_p, P(c_int32), c_void_p]
    L.pc_step_host.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, P(pc_step_opts),
                               P(pc_step_info), c_void_p]
    L.pc_mlp_features.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p, c_void_p]
    L.pc_mlp_create.argtypes = [P(c_void_p)]
    L.pc_mlp_destroy.argtypes = [c_void_p]
    L.pc_mlp_reset.argtypes = [c_void_p, c_void_p]
    L.pc_mlp_stats.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]
    L.pc_mlp_infer.argtypes = [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.pc_mlp_grad.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              P(c_double), c_void_p]
    L.pc_mlp_train_step.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    P(pc_adam_opts), P(c_double), c_void_p]
    L.pc_mlp_adam_apply.argtypes = [c_void_p, c_void_p, c_void_p, P(pc_adam_opts), c_void_p]
    L.pc_set_warm_mlp.argtypes = [c_void_p, c_void_p, c_void_p]
    L.pc_launch_count.restype = c_int64
    L.pc_launch_count.argtypes = [c_void_p]
    L.pc_set_profiling.argtypes = [c_void_p, c_int32]
    L.pc_spmv_stats.argtypes = [c_void_p, P(c_int64), P(c_double), P(c_int64)]
    L.pc_assembly_stats.argtypes = [c_void_p, P(c_int64), P(c_double)]
    L.pc_cluster_stats.argtypes = [c_void_p, P(c_int64), P(c_int64), P(c_double)]
    L.pc_get_solution64.argtypes = [c_void_p, c_void_p, c_void_p]
    for name in ("pc_create", "pc_destroy", "pc_get_sizes", "pc_get_rest", "pc_assemble_pattern",
                 "pc_assemble_values", "pc_bsr_spmv", "pc_pcg_solve", "pc_pcg_solve_static", "pc_step", "pc_step_host",
                 "pc_pcg_solve_batched", "pc_step_batched", "pc_batched_config", "pc_set_barrier_wait", "pc_proximity_query", "pc_get_prev_dv", "pc_set_prev_dv",
                 "pc_mlp_get_state", "pc_mlp_set_state", "pc_mlp_features", "pc_mlp_create",
                 "pc_mlp_destroy", "pc_mlp_reset", "pc_mlp_stats", "pc_mlp_infer", "pc_mlp_grad", "pc_mlp_train_step",
                 "pc_mlp_adam_apply", "pc_set_warm_mlp",
                 "pc_set_profiling", "pc_spmv_stats", "pc_assembly_stats", "pc_cluster_stats", "pc_get_solution64"):
        getattr(L, name).restype = c_int32
    return L


_lib = _load()


def lib():
    return _lib


# --------------------------------------------------------------------------- marshalling


def _stream(stream=None) -> c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def _ptr(t) -> c_void_p:
    if t is None:
        return c_void_p(None)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return c_void_p(t.data_ptr())


def _check(status: int, what: str, required: int | None = None):
    if status != PC_OK:
        raise PcError(status, what, required)


def material_struct(m) -> pc_material:
    """pc_material from a workloads.Material (or anything with the same fields)."""
    s = pc_material()
    s.rho, s.young, s.poisson, s.k_bend, s.k_contact = m.rho, m.young, m.poisson, m.k_bend, m.k_contact
    for i in range(3):
        s.gravity[i] = m.gravity[i]
    s.damp_mass = getattr(m, "damp_mass", 0.0)
    s.damp_stiff = getattr(m, "damp_stiff", 0.0)
    s.contact_thickness = getattr(m, "contact_thickness", 0.0)
    return s


def contacts_struct(pairs=None, w=None) -> pc_contacts:
    c = pc_contacts()
    if pairs is None or pairs.shape[0] == 0:
        c.n, c.pairs, c.w = 0, None, None
    else:
        c.n = int(pairs.shape[0])
        c.pairs = pairs.data_ptr()
        c.w = w.data_ptr()
    return c


def bsr_struct(row_ptr, col_idx, nnzb: int = 0) -> pc_bsr:
    A = pc_bsr()
    A.row_ptr = row_ptr.data_ptr()
    A.col_idx = col_idx.data_ptr()
    A.cap = (col_idx.numel() // 4) * 4
    A.nnzb = nnzb
    return A


def solve_opts(tol=1e-6, max_iter=20000, precision=PC_PREC_FP32, refresh=1e-2, refresh_every=1000, check_every=32,
               precond=PC_PRECOND_JACOBI, storage=None, fuse=True, schedule=PC_SCHED_AUTO):
    o = pc_solve_opts()
    o.tol, o.max_iter, o.precision, o.refresh, o.refresh_every, o.check_every, o.precond = (
        tol, max_iter, precision, refresh, refresh_every, check_every, precond)
    o.storage = PC_STORAGE_OFFDIAG if storage is None else storage
    o.fuse = 1 if fuse else 0
    o.schedule = schedule
    return o


# --------------------------------------------------------------------------- entry points


def pc_create(V, T, tris, rest, pins, material, max_contacts, stream=None):
    h = c_void_p()
    npin = 0 if pins is None else int(pins.numel())
    m = material if isinstance(material, pc_material) else material_struct(material)
    st = _lib.pc_create(ctypes.byref(h), int(V), int(T), _ptr(tris), _ptr(rest), _ptr(pins) if npin else c_void_p(None),
                        npin, ctypes.byref(m), int(max_contacts), _stream(stream))
    _check(st, "pc_create")
    return h


def pc_destroy(ctx):
    _check(_lib.pc_destroy(ctx), "pc_destroy")


def pc_get_sizes(ctx):
    V, T, H, S = c_int32(), c_int32(), c_int32(), c_int64()
    _check(_lib.pc_get_sizes(ctx, ctypes.byref(V), ctypes.byref(T), ctypes.byref(H), ctypes.byref(S)), "pc_get_sizes")
    return V.value, T.value, H.value, S.value


def pc_get_rest(ctx, hinges=None, mass=None, stream=None):
    _check(_lib.pc_get_rest(ctx, _ptr(hinges), _ptr(mass), _stream(stream)), "pc_get_rest")


def pc_assemble_pattern(ctx, pairs, w, row_ptr, col_idx, stream=None) -> int:
    A = bsr_struct(row_ptr, col_idx)
    c = contacts_struct(pairs, w)
    st = _lib.pc_assemble_pattern(ctx, ctypes.byref(c), ctypes.byref(A), _stream(stream))
    _check(st, "pc_assemble_pattern", int(A.nnzb) if st == PC_ERR_CAPACITY else None)
    return int(A.nnzb)


def pc_assemble_values(ctx, row_ptr, col_idx, nnzb, x, v, pairs, w, h, vals, b, dres=None, stream=None):
    A = bsr_struct(row_ptr, col_idx, nnzb)
    c = contacts_struct(pairs, w)
    st = _lib.pc_assemble_values(ctx, ctypes.byref(A), _ptr(x), _ptr(v), ctypes.byref(c), float(h), _ptr(vals),
                                 _ptr(b), _ptr(dres), _stream(stream))
    _check(st, "pc_assemble_values")


def pc_bsr_spmv(ctx, row_ptr, col_idx, nnzb, vals, dres, x, y, stream=None):
    A = bsr_struct(row_ptr, col_idx, nnzb)
    _check(_lib.pc_bsr_spmv(ctx, ctypes.byref(A), _ptr(vals), _ptr(dres), _ptr(x), _ptr(y), _stream(stream)),
           "pc_bsr_spmv")


def pc_pcg_solve(ctx, row_ptr, col_idx, nnzb, vals, dres, b, dv, opts=None, stream=None, allow_not_converged=False):
    A = bsr_struct(row_ptr, col_idx, nnzb)
    info = pc_solve_info()
    o = opts if opts is not None else solve_opts()
    st = _lib.pc_pcg_solve(ctx, ctypes.byref(A), _ptr(vals), _ptr(dres), _ptr(b), _ptr(dv), ctypes.byref(o),
                           ctypes.byref(info), _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_pcg_solve")
    return info, st


def pc_pcg_solve_static(V, row_ptr, col_idx, nnzb, vals, dres, b, dv, opts=None, stream=None,
                        allow_not_converged=False):
    """pc_pcg_solve without a context: all scratch in the library's static device array."""
    A = bsr_struct(row_ptr, col_idx, nnzb)
    info = pc_solve_info()
    o = opts if opts is not None else solve_opts()
    st = _lib.pc_pcg_solve_static(int(V), ctypes.byref(A), _ptr(vals), _ptr(dres), _ptr(b), _ptr(dv),
                                  ctypes.byref(o), ctypes.byref(info), _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_pcg_solve_static")
    return info, st


def _inst_array(inst_rows):
    arr = np.ascontiguousarray(np.asarray(inst_rows, dtype=np.int32))
    return arr, arr.ctypes.data_as(c_void_p)


def pc_pcg_solve_batched(ctx, row_ptr, col_idx, nnzb, vals, dres, b, dv, inst_rows, opts=None, stream=None,
                         allow_not_converged=False):
    """Batched solve; returns (list of per-instance pc_solve_info, status)."""
    A = bsr_struct(row_ptr, col_idx, nnzb)
    arr, ptr = _inst_array(inst_rows)
    n = len(arr) - 1
    infos = (pc_solve_info * n)()
    o = opts if opts is not None else solve_opts()
    st = _lib.pc_pcg_solve_batched(ctx, ctypes.byref(A), _ptr(vals), _ptr(dres), _ptr(b), _ptr(dv), n, ptr,
                                   ctypes.byref(o), ctypes.cast(infos, c_void_p), _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_pcg_solve_batched")
    return list(infos), st


def pc_step_batched(ctx, x, v, pairs, w, inst_rows, opts: pc_step_opts, stream=None, allow_not_converged=False):
    arr, ptr = _inst_array(inst_rows)
    n = len(arr) - 1
    infos = (pc_solve_info * n)()
    c = contacts_struct(pairs, w)
    st = _lib.pc_step_batched(ctx, _ptr(x), _ptr(v), ctypes.byref(c), n, ptr, ctypes.byref(opts),
                              ctypes.cast(infos, c_void_p), _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_step_batched")
    return list(infos), st


def pc_batched_config(ctx):
    """(grid in CTAs, SpMV entry order 0 strided / 1 chunked, stage width in blocks per row,
    candidate grid sizes [7], timings {width: [order][grid index]} in ms)."""
    grid, order, width = c_int32(), c_int32(), c_int32()
    sizes = (c_int32 * 7)()
    ms = (c_float * 28)()
    _check(_lib.pc_batched_config(ctx, ctypes.byref(grid), ctypes.byref(order), ctypes.byref(width),
                                  ctypes.cast(sizes, c_void_p), ctypes.cast(ms, c_void_p)), "pc_batched_config")
    return grid.value, order.value, width.value, list(sizes), {14: [list(ms[0:7]), list(ms[7:14])],
                                                               18: [list(ms[14:21]), list(ms[21:28])]}


def pc_proximity_query(ctx, x, delta, pairs, w, stream=None):
    """Contact pairs within `delta` of the positions x into the device buffers pairs
    (int32[cap, 4]) and w (float32[cap, 3]); returns the pair count."""
    cap = pairs.shape[0] if pairs is not None else 0
    if w is not None and w.shape[0] < cap:
        raise ValueError("w holds fewer rows than pairs")
    n = c_int32()
    _check(_lib.pc_proximity_query(ctx, _ptr(x), float(delta), int(cap), _ptr(pairs), _ptr(w), ctypes.byref(n),
                                   _stream(stream)), "pc_proximity_query", required=n.value)
    return n.value


def pc_get_prev_dv(ctx, dv, stream=None):
    """Copy the previous step's dv into dv (device float[V*3]); returns whether one exists."""
    valid = c_int32()
    _check(_lib.pc_get_prev_dv(ctx, _ptr(dv), ctypes.byref(valid), _stream(stream)), "pc_get_prev_dv")
    return bool(valid.value)


def pc_set_prev_dv(ctx, dv, stream=None):
    _check(_lib.pc_set_prev_dv(ctx, _ptr(dv), _stream(stream)), "pc_set_prev_dv")


def pc_mlp_get_state(m, m1, m2, stream=None):
    t = c_int64()
    _check(_lib.pc_mlp_get_state(m, _ptr(m1), _ptr(m2), ctypes.byref(t), _stream(stream)), "pc_mlp_get_state")
    return t.value


def pc_mlp_set_state(m, m1, m2, t, stream=None):
    _check(_lib.pc_mlp_set_state(m, _ptr(m1), _ptr(m2), int(t), _stream(stream)), "pc_mlp_set_state")


def pc_set_barrier_wait(ctx, cycles):
    """Grid-barrier wait budget (SM cycles) of the persistent batched solver; <= 0 restores
    the default."""
    _check(_lib.pc_set_barrier_wait(ctx, int(cycles)), "pc_set_barrier_wait")


def pc_step(ctx, x, v, pairs, w, opts: pc_step_opts, dv_out=None, stream=None, allow_not_converged=False):
    info = pc_step_info()
    c = contacts_struct(pairs, w)
    st = _lib.pc_step(ctx, _ptr(x), _ptr(v), ctypes.byref(c), ctypes.byref(opts), _ptr(dv_out), ctypes.byref(info),
                      _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_step")
    return info, st


def pc_step_host(ctx, x: np.ndarray, v: np.ndarray, pairs: np.ndarray, w: np.ndarray, opts: pc_step_opts,
                 stream=None, allow_not_converged=False):
    """Host-buffer step: x, v (float32 [V,3], updated in place), pairs int32 [P,4], w float32 [P,3]."""
    assert x.dtype == np.float32 and v.dtype == np.float32 and x.flags.c_contiguous and v.flags.c_contiguous
    info = pc_step_info()
    P = 0 if pairs is None else int(pairs.shape[0])
    pp = pairs.ctypes.data_as(c_void_p) if P else c_void_p(None)
    wp = w.ctypes.data_as(c_void_p) if P else c_void_p(None)
    st = _lib.pc_step_host(ctx, x.ctypes.data_as(c_void_p), v.ctypes.data_as(c_void_p), P, pp, wp,
                           ctypes.byref(opts), ctypes.byref(info), _stream(stream))
    if not (allow_not_converged and st == PC_ERR_NOT_CONVERGED):
        _check(st, "pc_step_host")
    return info, st


# --------------------------------------------------------------------------- learned warm start


def adam_opts(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> pc_adam_opts:
    return pc_adam_opts(lr, beta1, beta2, eps)


def pc_mlp_features(ctx, v, dv_prev, b, h, feat, stream=None):
    _check(_lib.pc_mlp_features(ctx, _ptr(v), _ptr(dv_prev), _ptr(b), float(h), _ptr(feat), _stream(stream)),
           "pc_mlp_features")


def pc_mlp_create():
    m = c_void_p()
    _check(_lib.pc_mlp_create(ctypes.byref(m)), "pc_mlp_create")
    return m


def pc_mlp_destroy(m):
    _check(_lib.pc_mlp_destroy(m), "pc_mlp_destroy")


def pc_mlp_reset(m, stream=None):
    _check(_lib.pc_mlp_reset(m, _stream(stream)), "pc_mlp_reset")


def pc_mlp_stats(m, n, feat, target, stats, stream=None):
    _check(_lib.pc_mlp_stats(m, int(n), _ptr(feat), _ptr(target), _ptr(stats), _stream(stream)), "pc_mlp_stats")


def pc_mlp_infer(n, params, stats, feat, dv_prev, fixed, dv0, stream=None):
    _check(_lib.pc_mlp_infer(int(n), _ptr(params), _ptr(stats), _ptr(feat), _ptr(dv_prev), _ptr(fixed), _ptr(dv0),
                             _stream(stream)), "pc_mlp_infer")


def pc_mlp_grad(m, n, rows, params, stats, feat, target, grad, with_loss=True, stream=None):
    loss = c_double(float("nan"))
    _check(_lib.pc_mlp_grad(m, int(n), _ptr(rows), _ptr(params), _ptr(stats), _ptr(feat), _ptr(target), _ptr(grad),
                            ctypes.byref(loss) if with_loss else None, _stream(stream)), "pc_mlp_grad")
    return loss.value


def pc_mlp_train_step(m, n, rows, params, stats, feat, target, opts: pc_adam_opts, with_loss=False, stream=None):
    loss = c_double(float("nan"))
    _check(_lib.pc_mlp_train_step(m, int(n), _ptr(rows), _ptr(params), _ptr(stats), _ptr(feat), _ptr(target),
                                  ctypes.byref(opts), ctypes.byref(loss) if with_loss else None, _stream(stream)),
           "pc_mlp_train_step")
    return loss.value


def pc_mlp_adam_apply(m, params, grad, opts: pc_adam_opts, stream=None):
    _check(_lib.pc_mlp_adam_apply(m, _ptr(params), _ptr(grad), ctypes.byref(opts), _stream(stream)), "pc_mlp_adam_apply")


def pc_set_warm_mlp(ctx, params, stats):
    _check(_lib.pc_set_warm_mlp(ctx, _ptr(params), _ptr(stats)), "pc_set_warm_mlp")


def pc_launch_count(ctx) -> int:
    return int(_lib.pc_launch_count(ctx))


def pc_set_profiling(ctx, enable: bool):
    _check(_lib.pc_set_profiling(ctx, int(bool(enable))), "pc_set_profiling")


def pc_get_solution64(ctx, dv64, stream=None):
    _check(_lib.pc_get_solution64(ctx, _ptr(dv64), _stream(stream)), "pc_get_solution64")


def pc_assembly_stats(ctx):
    n, ms = c_int64(), c_double()
    _check(_lib.pc_assembly_stats(ctx, ctypes.byref(n), ctypes.byref(ms)), "pc_assembly_stats")
    return n.value, ms.value


def pc_cluster_stats(ctx):
    n, it, ms = c_int64(), c_int64(), c_double()
    _check(_lib.pc_cluster_stats(ctx, ctypes.byref(n), ctypes.byref(it), ctypes.byref(ms)), "pc_cluster_stats")
    return n.value, it.value, ms.value


def pc_spmv_stats(ctx):
    n, ms, nnzb = c_int64(), c_double(), c_int64()
    _check(_lib.pc_spmv_stats(ctx, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(nnzb)), "pc_spmv_stats")
    return n.value, ms.value, nnzb.value


# --------------------------------------------------------------------------- convenience


class Cloth:
    """One cloth on the GPU: a context plus device copies of the workload's state."""

    def __init__(self, wl, max_contacts: int | None = None, device="cuda"):
        self.wl = wl
        dev = torch.device(device)
        self.device = dev
        self.tris = torch.from_numpy(np.ascontiguousarray(wl.tris, np.int32)).to(dev)
        self.rest = torch.from_numpy(np.ascontiguousarray(wl.rest, np.float32)).to(dev)
        self.pins = torch.from_numpy(np.ascontiguousarray(wl.pins, np.int32)).to(dev)
        self.max_contacts = wl.n_contacts if max_contacts is None else max_contacts
        self.ctx = pc_create(wl.V, wl.T, self.tris, self.rest, self.pins, wl.material, self.max_contacts)
        self.V, self.T, self.H, self.static_nnzb = pc_get_sizes(self.ctx)
        self.x = torch.from_numpy(np.ascontiguousarray(wl.x0, np.float32)).to(dev)
        self.v = torch.from_numpy(np.ascontiguousarray(wl.v0, np.float32)).to(dev)
        self.h = wl.h

    def close(self):
        if getattr(self, "ctx", None) is not None:
            pc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def proximity(self, delta: float | None = None, x=None):
        """Contacts of the one-sided thickness model at positions x (the cloth's own by
        default): (pairs, w) views of context-sized device buffers."""
        if getattr(self, "_px_pairs", None) is None:
            self._px_pairs = torch.zeros((max(self.max_contacts, 1), 4), dtype=torch.int32, device=self.device)
            self._px_w = torch.zeros((max(self.max_contacts, 1), 3), dtype=torch.float32, device=self.device)
        d = self.wl.material.contact_thickness if delta is None else delta
        n = pc_proximity_query(self.ctx, self.x if x is None else x, d, self._px_pairs[: self.max_contacts],
                               self._px_w[: self.max_contacts])
        if n == 0:
            return None, None
        return self._px_pairs[:n], self._px_w[:n]

    def contacts_device(self, step: int):
        if self.wl.contact_kind == "proximity":
            return self.proximity()
        pairs, w = self.wl.contacts(step)
        if pairs.shape[0] == 0:
            return None, None
        return (torch.from_numpy(pairs).to(self.device), torch.from_numpy(w).to(self.device))

    def alloc_system(self, extra_blocks: int = 0):
        cap = ((self.static_nnzb + 6 * self.max_contacts + extra_blocks) + 3) // 4 * 4
        dev = self.device
        return {
            "row_ptr": torch.zeros(self.V + 1, dtype=torch.int32, device=dev),
            "col_idx": torch.zeros(cap, dtype=torch.int32, device=dev),
            "vals": torch.zeros(cap * 9, dtype=torch.float32, device=dev),
            "b": torch.zeros(self.V * 3, dtype=torch.float32, device=dev),
            "dres": torch.zeros(self.V * 9, dtype=torch.float32, device=dev),
        }

    def assemble(self, pairs=None, w=None, x=None, v=None, sysbuf=None):
        """Pattern + values of this step's system; returns the buffers and nnzb."""
        s = sysbuf if sysbuf is not None else self.alloc_system()
        nnzb = pc_assemble_pattern(self.ctx, pairs, w, s["row_ptr"], s["col_idx"])
        pc_assemble_values(self.ctx, s["row_ptr"], s["col_idx"], nnzb, self.x if x is None else x,
                           self.v if v is None else v, pairs, w, self.h, s["vals"], s["b"], s["dres"])
        s["nnzb"] = nnzb
        return s

    def step(self, pairs=None, w=None, tol=1e-6, precision=PC_PREC_FP32, warm_start=PC_WARM_ZERO, max_iter=20000,
             dv_out=None, precond=PC_PRECOND_JACOBI, allow_not_converged=False, feat_out=None, storage=None,
             fuse=True, schedule=PC_SCHED_AUTO):
        o = pc_step_opts()
        o.h = self.h
        o.solve = solve_opts(tol=tol, max_iter=max_iter, precision=precision, precond=precond, storage=storage,
                             fuse=fuse, schedule=schedule)
        o.warm_start = warm_start
        o.feat_out = _ptr(feat_out)
        info, st = pc_step(self.ctx, self.x, self.v, pairs, w, o, dv_out, allow_not_converged=allow_not_converged)
        return info, st
