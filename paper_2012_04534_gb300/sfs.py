"""Thin ctypes binding of libsfs (include/sfs.h).

Argument marshalling only: every step of the operator, the solver and the
reductions runs in the library's CUDA kernels.  PyTorch supplies device
memory (complex64 tensors) and the current CUDA stream.  The module-level
``sfs_*`` functions mirror the C entry points one to one; ``Geometry`` and
``Operator`` wrap the handles for convenience.  Importing this module does
not load the library; the first call does, and it raises if libsfs.so has
not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsfs.so")

SFS_OK = 0
SFS_ERR_INVALID_ARG = -1
SFS_ERR_BAND_TOO_NARROW = -2
SFS_ERR_CUDA = -3
SFS_ERR_OOM = -4
SFS_ERR_TIMEOUT = -5
SFS_ERR_NOT_CONVERGED = -6
SFS_ERR_NON_FINITE = -7

SFS_SEL_RANDOM = 0
SFS_SEL_CONTIGUOUS = 1
SFS_SEL_EQUISPACED = 2
SFS_SEL_MAXIMAL = 3
SFS_SEL_ENERGY = 4

SFS_PREC_FP32 = 0
SFS_PREC_TF32X3 = 1
SFS_PREC_BF16 = 2
SFS_PREC_BF16X2 = 3
SFS_PREC_FP16 = 4
SFS_PREC_FP16X2 = 5
PRECISION_NAMES = {"fp32": SFS_PREC_FP32, "tf32x3": SFS_PREC_TF32X3, "bf16": SFS_PREC_BF16,
                   "bf16x2": SFS_PREC_BF16X2, "fp16": SFS_PREC_FP16, "fp16x2": SFS_PREC_FP16X2}

SFS_MAX_BATCH = 256
SFS_MAX_GROUPS = 64

SFS_GROUPED_CHEAPEST_FIRST = 0
SFS_GROUPED_LARGEST_FIRST = 1
SFS_GROUPED_NO_PRIORITY = 2

SFS_FISTA_WARM_START = 1
SFS_FISTA_TIME_KERNELS = 2
SFS_FISTA_RESUME = 4

STATUS_NAMES = {0: "SFS_OK", -1: "SFS_ERR_INVALID_ARG", -2: "SFS_ERR_BAND_TOO_NARROW",
                -3: "SFS_ERR_CUDA", -4: "SFS_ERR_OOM", -5: "SFS_ERR_TIMEOUT",
                -6: "SFS_ERR_NOT_CONVERGED", -7: "SFS_ERR_NON_FINITE"}

# every symbol include/sfs.h declares
EXPORTS = ("sfs_create_geometry", "sfs_destroy_geometry", "sfs_select_indices",
           "sfs_select_freqs", "sfs_operator_from_indices", "sfs_operator_from_indices_prec",
           "sfs_destroy_operator",
           "sfs_operator_info", "sfs_apply_A", "sfs_apply_AH", "sfs_apply_AH_noalloc",
           "sfs_max_abs_AH", "sfs_apply_A_batched", "sfs_apply_AH_batched", "sfs_fista_batched",
           "sfs_lista_create", "sfs_lista_destroy", "sfs_lista_info", "sfs_lista_set_params",
           "sfs_lista_get_params", "sfs_lista_load_params_dev", "sfs_lista_forward",
           "sfs_lista_backward", "sfs_lista_nmse", "sfs_lista_adam", "sfs_frobenius",
           "sfs_fista_grouped", "sfs_fista_persistent", "sfs_autotune_persistent", "sfs_persistent_step_times", "sfs_crb", "sfs_mixing_band", "sfs_mixing_create", "sfs_mixing_destroy",
           "sfs_apply_A_mixed", "sfs_apply_AH_mixed", "sfs_lipschitz_mixed", "sfs_fista_mixed",
           "sfs_autotune_batch", "sfs_set_batch_tile", "sfs_fista_backtracking", "sfs_grouped_times",
           "sfs_set_grouped_order",
           "sfs_lipschitz", "sfs_fista", "sfs_kernel_times", "sfs_stage_times",
           "sfs_set_wait_timeout_ns", "sfs_shard_run", "sfs_operator_shard", "sfs_normal_residual",
           "sfs_prox_momentum", "sfs_vec_sumsq", "sfs_vec_max_abs", "sfs_vec_scale", "sfs_vec_randn",
           "sfs_inject_wait_timeout", "sfs_check_status", "sfs_last_error", "sfs_version")


class SfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class GeometryDesc(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int32), ("Ny", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("Nz", ctypes.c_int32), ("z0", ctypes.c_double), ("dz", ctypes.c_double),
                ("c", ctypes.c_double), ("fs", ctypes.c_double), ("Nt", ctypes.c_int32),
                ("t0", ctypes.c_double), ("fc", ctypes.c_double),
                ("frac_bw", ctypes.c_double), ("theta", ctypes.c_double),
                ("device", ctypes.c_int32)]


class OperatorInfo(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("M", ctypes.c_int32), ("V", ctypes.c_int32),
                ("Nz", ctypes.c_int32), ("U", ctypes.c_int32), ("Px", ctypes.c_int32),
                ("Py", ctypes.c_int32), ("Nkappa", ctypes.c_int32),
                ("k_lo", ctypes.c_int32), ("k_hi", ctypes.c_int32),
                ("band_db", ctypes.c_double), ("alpha", ctypes.c_double),
                ("t0", ctypes.c_double), ("table_bytes", ctypes.c_int64),
                ("launches_per_iter", ctypes.c_int32), ("Nslot", ctypes.c_int32),
                ("GS", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nshards", ctypes.c_int32), ("shard", ctypes.c_int32),
                ("shard_first", ctypes.c_int32), ("U_all", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libsfs.so (built in-tree by paper_2012_04534_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsfs.so is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                              ctypes.c_uint64, ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "sfs_create_geometry": [P(GeometryDesc), P(vp)],
        "sfs_destroy_geometry": [vp],
        "sfs_select_indices": [vp, i32, i32, i32, u64, P(ctypes.c_int32), P(ctypes.c_int32)],
        "sfs_select_freqs": [vp, i32, i32, i32, u64, P(ctypes.c_int32), P(ctypes.c_uint32), P(vp)],
        "sfs_operator_from_indices": [vp, i32, P(ctypes.c_int32), P(vp)],
        "sfs_operator_from_indices_prec": [vp, i32, P(ctypes.c_int32), i32, P(vp)],
        "sfs_destroy_operator": [vp],
        "sfs_operator_info": [vp, P(OperatorInfo)],
        "sfs_apply_A": [vp, vp, vp, vp],
        "sfs_apply_AH": [vp, vp, vp, vp],
        "sfs_apply_AH_noalloc": [vp, vp, vp, vp],
        "sfs_max_abs_AH": [vp, vp, P(dbl), vp],
        "sfs_frobenius": [vp, P(dbl), P(dbl)],
        "sfs_fista_grouped": [i32, P(vp), P(ctypes.c_int32), P(vp), P(dbl), dbl, i32, P(vp), vp],
        "sfs_fista_persistent": [i32, P(vp), P(ctypes.c_int32), P(vp), P(dbl), dbl, i32, P(vp), i32, vp],
        "sfs_autotune_persistent": [i32, P(vp), P(ctypes.c_int32), P(vp), P(dbl), dbl, i32, i32, P(vp),
                                    P(ctypes.c_int32), P(dbl), vp],
        "sfs_persistent_step_times": [P(dbl)],
        "sfs_crb": [vp, i32, i32, P(ctypes.c_int32), P(dbl), dbl, dbl, dbl, i32, P(dbl), P(dbl)],
        "sfs_mixing_band": [vp, P(ctypes.c_int32), P(ctypes.c_int32)],
        "sfs_mixing_create": [vp, i32, P(ctypes.c_int32), P(ctypes.c_int8), P(vp)],
        "sfs_mixing_destroy": [vp],
        "sfs_autotune_batch": [vp, i32, i32, P(ctypes.c_int32), P(dbl)],
        "sfs_set_batch_tile": [vp, i32, i32],
        "sfs_fista_backtracking": [vp, vp, dbl, dbl, dbl, i32, vp, P(dbl), vp],
        "sfs_grouped_times": [i32, P(ctypes.c_float)],
        "sfs_set_grouped_order": [i32],
        "sfs_apply_A_mixed": [vp, vp, vp, vp],
        "sfs_apply_AH_mixed": [vp, vp, vp, vp],
        "sfs_lipschitz_mixed": [vp, i32, dbl, u64, dbl, P(dbl), vp],
        "sfs_fista_mixed": [vp, vp, dbl, dbl, i32, vp, vp],
        "sfs_apply_A_batched": [vp, i32, vp, vp, vp],
        "sfs_apply_AH_batched": [vp, i32, vp, vp, vp],
        "sfs_fista_batched": [vp, i32, vp, dbl, dbl, i32, vp, u32, vp],
        "sfs_lipschitz": [vp, i32, dbl, u64, dbl, P(dbl), vp],
        "sfs_fista": [vp, vp, dbl, dbl, i32, vp, vp, u32, P(dbl), vp],
        "sfs_kernel_times": [vp, P(dbl), P(dbl), P(ctypes.c_int32)],
        "sfs_set_wait_timeout_ns": [vp, u64],
        "sfs_stage_times": [vp, P(dbl), P(ctypes.c_int32)],
        "sfs_check_status": [vp, vp],
        "sfs_inject_wait_timeout": [vp, i32],
        "sfs_shard_run": [i32, i32, i32, P(ctypes.c_int32), P(ctypes.c_int32)],
        "sfs_operator_shard": [vp, i32, P(ctypes.c_int32), i32, i32, i32, P(vp)],
        "sfs_normal_residual": [vp, vp, vp, vp, vp],
        "sfs_prox_momentum": [i32, vp, vp, vp, dbl, dbl, dbl, vp],
        "sfs_vec_sumsq": [vp, vp, i32, P(dbl), vp],
        "sfs_vec_max_abs": [vp, vp, i32, P(dbl), vp],
        "sfs_vec_scale": [vp, i32, dbl, vp],
        "sfs_vec_randn": [vp, i32, u64, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.sfs_last_error.restype = ctypes.c_char_p
    L.sfs_last_error.argtypes = []
    L.sfs_version.restype = ctypes.c_char_p
    L.sfs_version.argtypes = []
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != SFS_OK and rc not in allow:
        raise SfsError(rc, lib().sfs_last_error().decode())
    return rc


def _stream_ptr(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.complex64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s must be a contiguous complex64 tensor of %d elements "
                         "(got %s %s %d)" % (name, numel, t.dtype, tuple(t.shape), t.numel()))
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names ---

def sfs_create_geometry(**params) -> ctypes.c_void_p:
    d = GeometryDesc()
    d.Nx = int(params["Nx"]); d.Ny = int(params["Ny"])
    d.dx = float(params["dx"]); d.dy = float(params.get("dy", params["dx"]))
    d.Nz = int(params["Nz"]); d.z0 = float(params["z0"]); d.dz = float(params["dz"])
    d.c = float(params["c"]); d.fs = float(params["fs"]); d.Nt = int(params["Nt"])
    d.t0 = float(params.get("t0", math.nan)); d.fc = float(params["fc"])
    d.frac_bw = float(params["frac_bw"]); d.theta = float(params.get("theta", 0.0))
    d.device = int(params.get("device", 0))
    h = ctypes.c_void_p()
    _check(lib().sfs_create_geometry(ctypes.byref(d), ctypes.byref(h)))
    return h


def sfs_select_indices(geom, strategy: int, M: int, per_position: bool, seed: int,
                       S: int):
    idx = np.zeros((S, M), dtype=np.int32)
    band = np.zeros(2, dtype=np.int32)
    _check(lib().sfs_select_indices(geom, strategy, M, int(per_position), seed,
                                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    band.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return idx, (int(band[0]), int(band[1]))


def sfs_select_freqs(geom, strategy: int, M: int, per_position: bool, seed: int, S: int,
                     Nt: int):
    idx = np.zeros((S, M), dtype=np.int32)
    words = (Nt // 2 + 1 + 31) // 32
    mask = np.zeros((S, words), dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(lib().sfs_select_freqs(geom, strategy, M, int(per_position), seed,
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                  ctypes.byref(h)))
    return h, idx, mask


def sfs_operator_from_indices(geom, idx):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().sfs_operator_from_indices(
        geom, idx.shape[1], idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(h)))
    return h


def sfs_operator_from_indices_prec(geom, idx, precision: int):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().sfs_operator_from_indices_prec(
        geom, idx.shape[1], idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(precision),
        ctypes.byref(h)))
    return h


def sfs_operator_info(op) -> dict:
    info = OperatorInfo()
    _check(lib().sfs_operator_info(op, ctypes.byref(info)))
    return info.as_dict()


def sfs_apply_A(op, x_dev_ptr, y_dev_ptr, stream_ptr):
    _check(lib().sfs_apply_A(op, x_dev_ptr, y_dev_ptr, stream_ptr))


def sfs_apply_AH(op, y_dev_ptr, x_dev_ptr, stream_ptr):
    _check(lib().sfs_apply_AH(op, y_dev_ptr, x_dev_ptr, stream_ptr))


def sfs_apply_AH_noalloc(op, y_dev_ptr, x_dev_ptr, stream_ptr):
    """A^H y with all intermediate data in the library's static device array
    (no allocation during the call); see include/sfs.h."""
    _check(lib().sfs_apply_AH_noalloc(op, y_dev_ptr, x_dev_ptr, stream_ptr))


def sfs_max_abs_AH(op, y_dev_ptr, stream_ptr) -> float:
    out = ctypes.c_double()
    _check(lib().sfs_max_abs_AH(op, y_dev_ptr, ctypes.byref(out), stream_ptr))
    return out.value


def sfs_lipschitz(op, max_iter, rtol, seed, safety, stream_ptr):
    out = ctypes.c_double()
    rc = _check(lib().sfs_lipschitz(op, max_iter, rtol, seed, safety, ctypes.byref(out),
                                    stream_ptr), allow=(SFS_ERR_NOT_CONVERGED,))
    return out.value, rc == SFS_OK


def sfs_fista(op, y_dev_ptr, lam, L, iters, x_dev_ptr, state_dev_ptr, flags, obj_hist, stream_ptr):
    ptr = None
    if obj_hist is not None:
        ptr = obj_hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().sfs_fista(op, y_dev_ptr, lam, L, iters, x_dev_ptr, state_dev_ptr, flags, ptr,
                           stream_ptr))


def shard_run(U: int, nshards: int, shard: int):
    """sfs_shard_run: (first union position, count) of run `shard`."""
    f, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sfs_shard_run(int(U), int(nshards), int(shard), ctypes.byref(f), ctypes.byref(c)))
    return f.value, c.value


def prox_momentum(x, gamma, grad, lam, L, beta, stream=None):
    """sfs_prox_momentum: x <- tau_{lam/L}(gamma - grad/L), gamma <- x + beta (x - x_prev)."""
    n = int(x.numel())
    _check(lib().sfs_prox_momentum(n, _dev_ptr(x, n, "x"), _dev_ptr(gamma, n, "gamma"),
                                   _dev_ptr(grad, n, "grad"), float(lam), float(L), float(beta),
                                   _stream_ptr(stream, x.device)))


def vec_scale(v, a, stream=None):
    _check(lib().sfs_vec_scale(_dev_ptr(v, v.numel(), "v"), int(v.numel()), float(a),
                               _stream_ptr(stream, v.device)))


def vec_randn(v, seed, stream=None):
    _check(lib().sfs_vec_randn(_dev_ptr(v, v.numel(), "v"), int(v.numel()), int(seed),
                               _stream_ptr(stream, v.device)))


def sfs_kernel_times(op):
    f, a, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().sfs_kernel_times(op, ctypes.byref(f), ctypes.byref(a), ctypes.byref(n)))
    return f.value, a.value, n.value


def sfs_stage_times(op):
    ms4 = (ctypes.c_double * 4)()
    n = ctypes.c_int32()
    _check(lib().sfs_stage_times(op, ms4, ctypes.byref(n)))
    return list(ms4), n.value


def sfs_set_wait_timeout_ns(op, ns: int):
    _check(lib().sfs_set_wait_timeout_ns(op, ns))


def sfs_inject_wait_timeout(op, enable: bool):
    _check(lib().sfs_inject_wait_timeout(op, int(enable)))


def sfs_check_status(op, stream_ptr) -> int:
    """SFS_OK, SFS_ERR_TIMEOUT or SFS_ERR_NON_FINITE (returned, not raised)."""
    return _check(lib().sfs_check_status(op, stream_ptr),
                  allow=(SFS_ERR_TIMEOUT, SFS_ERR_NON_FINITE))


def sfs_version() -> str:
    return lib().sfs_version().decode()


# --------------------------------------------------------------- wrappers ---

def _group_args(ops, ys, Ls, xs):
    import torch
    n = len(ops)
    if len(ys) != n or len(Ls) != n or (xs is not None and len(xs) != n):
        raise ValueError("one measurement tensor, one L (and one result tensor) per operator: "
                         "%d operators, %d y, %d L%s" % (n, len(ys), len(Ls),
                                                        "" if xs is None else ", %d x" % len(xs)))
    if xs is None:
        xs = [torch.empty((int(y.shape[0]),) + op.shape_x, dtype=torch.complex64, device=y.device)
              for op, y in zip(ops, ys)]
    VP = ctypes.c_void_p * n
    oph = VP(*[op.handle for op in ops])
    b = (ctypes.c_int32 * n)(*[int(y.shape[0]) for y in ys])
    yp = VP(*[_dev_ptr(y, int(y.shape[0]) * op.S * op.M, "y") for op, y in zip(ops, ys)])
    xp = VP(*[_dev_ptr(x, int(x.shape[0]) * op.V, "x") for op, x in zip(ops, xs)])
    Lv = (ctypes.c_double * n)(*[float(v) for v in Ls])
    return n, oph, b, yp, Lv, xp, xs


def fista_grouped(ops, ys, Ls, lam, iters, xs=None, stream=None, persistent=False, nb_policy=0):
    """sfs_fista_grouped: ops[g] solves the scenes ys[g] ([batch, S, M]
    complex64 CUDA tensors) with Lipschitz constant Ls[g]; returns the list
    of [batch, Nz, Ny, Nx] results.  persistent: sfs_fista_persistent (the
    loop of all groups in one persistent kernel, scenes per table tile by
    nb_policy: 0 each group's own, else 1, 2 or 4)."""
    n, oph, b, yp, Lv, xp, xs = _group_args(ops, ys, Ls, xs)
    if persistent:
        _check(lib().sfs_fista_persistent(n, oph, b, yp, Lv, float(lam), int(iters), xp, int(nb_policy),
                                          _stream_ptr(stream, ys[0].device)))
    else:
        _check(lib().sfs_fista_grouped(n, oph, b, yp, Lv, float(lam), int(iters), xp,
                                       _stream_ptr(stream, ys[0].device)))
    return xs


def fista_persistent(ops, ys, Ls, lam, iters, xs=None, stream=None, nb_policy=0):
    """sfs_fista_persistent: fista_grouped with the iteration loop of every
    group in one persistent kernel."""
    return fista_grouped(ops, ys, Ls, lam, iters, xs=xs, stream=stream, persistent=True,
                         nb_policy=nb_policy)


def persistent_step_times():
    """sfs_persistent_step_times: ms of the forward contractions, residual
    planes, adjoint contractions and update planes of the latest persistent
    solve, summed over its iterations, then the mean CTA busy time in each."""
    out = (ctypes.c_double * 8)()
    _check(lib().sfs_persistent_step_times(out))
    return [out[i] for i in range(8)]


def autotune_persistent(ops, ys, Ls, lam, probe_iters=10, reps=3, xs=None, stream=None):
    """sfs_autotune_persistent: (tile policy chosen, [ms per probe solve for
    policies 0, 1, 2, 4])."""
    n, oph, b, yp, Lv, xp, xs = _group_args(ops, ys, Ls, xs)
    c = ctypes.c_int32()
    ms = (ctypes.c_double * 4)()
    _check(lib().sfs_autotune_persistent(n, oph, b, yp, Lv, float(lam), int(probe_iters), int(reps), xp,
                                         ctypes.byref(c), ms, _stream_ptr(stream, ys[0].device)))
    return c.value, [ms[i] for i in range(4)]


def set_grouped_order(order):
    """sfs_set_grouped_order: priority order of the grouped graphs captured
    from now on (SFS_GROUPED_CHEAPEST_FIRST, _LARGEST_FIRST, _NO_PRIORITY)."""
    _check(lib().sfs_set_grouped_order(int(order)))


def grouped_times(n):
    """sfs_grouped_times: per-group completion (ms) of the latest grouped solve."""
    out = (ctypes.c_float * n)()
    _check(lib().sfs_grouped_times(int(n), out))
    return [float(v) for v in out]


class Geometry:
    """Scan / voxel grid and pulse (sfs_geometry_desc)."""

    def __init__(self, **params):
        self.params = dict(params)
        self.device = int(params.get("device", 0))
        self.handle = sfs_create_geometry(**params)
        self.Nx, self.Ny, self.Nz = int(params["Nx"]), int(params["Ny"]), int(params["Nz"])
        self.Nt = int(params["Nt"])
        self.S = self.Nx * self.Ny
        self.V = self.S * self.Nz

    def select_indices(self, strategy, M, per_position=True, seed=0):
        return sfs_select_indices(self.handle, strategy, M, per_position, seed, self.S)

    def crb(self, idx, pos, amp=1.0, phase=0.0, sigma2=1.0, mask=7):
        """sfs_crb: idx int32 [T][S][M] (or [S][M]); returns (crb [T][3] in
        m^2, NaN outside mask; fim [T][5][5])."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.ndim == 2:
            idx = idx[None]
        T, S, M = idx.shape
        if S != self.S:
            raise ValueError("index sets must have S = %d rows" % self.S)
        c = np.empty((T, 3), dtype=np.float64)
        J = np.empty((T, 5, 5), dtype=np.float64)
        p = (ctypes.c_double * 3)(*[float(v) for v in pos])
        _check(lib().sfs_crb(self.handle, T, M, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), p,
                             float(amp), float(phase), float(sigma2), int(mask),
                             c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             J.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return c, J

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sfs_destroy_geometry(h)
            self.handle = None


class Operator:
    """A = S F H and its adjoint on one GPU (sfs_operator)."""

    def __init__(self, geom: Geometry, handle):
        self.geom = geom
        self.handle = handle
        self.info = sfs_operator_info(handle)
        self.S, self.M, self.V = self.info["S"], self.info["M"], self.info["V"]
        self.shape_x = (geom.Nz, geom.Ny, geom.Nx)
        self.shape_y = (self.S, self.M)
        self.device = geom.device

    @classmethod
    def select(cls, geom: Geometry, strategy=SFS_SEL_RANDOM, M=32, per_position=True, seed=0,
               precision=None):
        """Selection plus operator; `precision` (an SFS_PREC_* value) goes
        through sfs_select_indices + sfs_operator_from_indices_prec."""
        if precision is not None:
            idx, _ = sfs_select_indices(geom.handle, strategy, M, per_position, seed, geom.S)
            return cls.from_indices(geom, idx, precision)
        h, idx, mask = sfs_select_freqs(geom.handle, strategy, M, per_position, seed,
                                        geom.S, geom.Nt)
        op = cls(geom, h)
        op.idx, op.mask = idx, mask
        return op

    @classmethod
    def from_indices(cls, geom: Geometry, idx, precision=None):
        if precision is None:
            h = sfs_operator_from_indices(geom.handle, idx)
        else:
            h = sfs_operator_from_indices_prec(geom.handle, idx, precision)
        op = cls(geom, h)
        op.idx = np.ascontiguousarray(idx, dtype=np.int32)
        return op

    @classmethod
    def shard(cls, geom: Geometry, idx, nshards: int, shard: int, precision: int = SFS_PREC_FP32):
        """sfs_operator_shard: the rows of run `shard` of the bin union cut in
        `nshards` (measurement layout stays [S][M])."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib().sfs_operator_shard(geom.handle, idx.shape[1],
                                        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        int(nshards), int(shard), int(precision), ctypes.byref(h)))
        op = cls(geom, h)
        op.idx = idx
        return op

    def normal_residual(self, x, y, out=None, stream=None):
        """sfs_normal_residual: A^H (A x - y) over this operator's rows."""
        g = self._new(self.shape_x) if out is None else out
        _check(lib().sfs_normal_residual(self.handle, _dev_ptr(x, self.V, "x"),
                                         _dev_ptr(y, self.S * self.M, "y"), _dev_ptr(g, self.V, "g"),
                                         _stream_ptr(stream, x.device)))
        return g

    def vec_sumsq(self, v, stream=None):
        out = ctypes.c_double()
        _check(lib().sfs_vec_sumsq(self.handle, _dev_ptr(v, v.numel(), "v"), int(v.numel()),
                                   ctypes.byref(out), _stream_ptr(stream, v.device)))
        return out.value

    def vec_max_abs(self, v, stream=None):
        out = ctypes.c_double()
        _check(lib().sfs_vec_max_abs(self.handle, _dev_ptr(v, v.numel(), "v"), int(v.numel()),
                                     ctypes.byref(out), _stream_ptr(stream, v.device)))
        return out.value

    def _new(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.complex64, device="cuda:%d" % self.device)

    def apply_A(self, x, out=None, stream=None):
        y = self._new(self.shape_y) if out is None else out
        sfs_apply_A(self.handle, _dev_ptr(x, self.V, "x"), _dev_ptr(y, self.S * self.M, "y"),
                    _stream_ptr(stream, x.device))
        return y

    def apply_AH(self, y, out=None, stream=None):
        x = self._new(self.shape_x) if out is None else out
        sfs_apply_AH(self.handle, _dev_ptr(y, self.S * self.M, "y"), _dev_ptr(x, self.V, "x"),
                     _stream_ptr(stream, y.device))
        return x

    # ---- batched scenes sharing this operator (leading dimension = scene) ----
    def apply_A_batched(self, x, out=None, stream=None):
        B = int(x.shape[0])
        y = self._new((B,) + self.shape_y) if out is None else out
        _check(lib().sfs_apply_A_batched(self.handle, B, _dev_ptr(x, B * self.V, "x"),
                                         _dev_ptr(y, B * self.S * self.M, "y"),
                                         _stream_ptr(stream, x.device)))
        return y

    def apply_AH_batched(self, y, out=None, stream=None):
        B = int(y.shape[0])
        x = self._new((B,) + self.shape_x) if out is None else out
        _check(lib().sfs_apply_AH_batched(self.handle, B, _dev_ptr(y, B * self.S * self.M, "y"),
                                          _dev_ptr(x, B * self.V, "x"),
                                          _stream_ptr(stream, y.device)))
        return x

    def fista_batched(self, y, lam, L, iters, x=None, warm_start=False, stream=None):
        """Scenes y[b] (same operator); lam < 0: lambda_b = -lam ||A^H y_b||_inf.
        warm_start: x holds every scene's x_0 on entry."""
        B = int(y.shape[0])
        if x is None:
            if warm_start:
                raise ValueError("warm_start needs x")
            x = self._new((B,) + self.shape_x)
        _check(lib().sfs_fista_batched(self.handle, B, _dev_ptr(y, B * self.S * self.M, "y"),
                                       float(lam), float(L), int(iters),
                                       _dev_ptr(x, B * self.V, "x"),
                                       SFS_FISTA_WARM_START if warm_start else 0,
                                       _stream_ptr(stream, y.device)))
        return x

    def autotune(self, batch, reps=5):
        """sfs_autotune_batch: (chosen scenes per table tile, ms per forward +
        adjoint pair for 1, 2, 4)."""
        nb = ctypes.c_int32()
        ms = (ctypes.c_double * 3)()
        _check(lib().sfs_autotune_batch(self.handle, int(batch), int(reps), ctypes.byref(nb), ms))
        return nb.value, [ms[0], ms[1], ms[2]]

    def set_batch_tile(self, batch, nb):
        _check(lib().sfs_set_batch_tile(self.handle, int(batch), int(nb)))

    def frobenius(self):
        """(||A||_F^2, sigma_hat) of Sec. IV-C (host computation)."""
        f, sh = ctypes.c_double(), ctypes.c_double()
        _check(lib().sfs_frobenius(self.handle, ctypes.byref(f), ctypes.byref(sh)))
        return f.value, sh.value

    def max_abs_AH(self, y, stream=None) -> float:
        return sfs_max_abs_AH(self.handle, _dev_ptr(y, self.S * self.M, "y"),
                              _stream_ptr(stream, y.device))

    def lipschitz(self, max_iter=500, rtol=1e-6, seed=0, safety=1e-3, stream=None):
        import torch
        return sfs_lipschitz(self.handle, max_iter, rtol, seed, safety,
                             _stream_ptr(stream, torch.device("cuda", self.device)))

    def new_fista_state(self):
        """Device buffer for sfs_fista's state (gamma, x, t, count):
        complex64 [2 V + 2], i.e. SFS_FISTA_STATE_BYTES(V) bytes."""
        return self._new((2 * self.V + 2,))

    def fista(self, y, lam, L, iters, x=None, warm_start=False, obj_hist=False,
              time_kernels=False, state=None, resume=False, stream=None):
        """lam >= 0: lambda; lam < 0: lambda = -lam * ||A^H y||_inf.
        state: buffer from new_fista_state() that receives the iteration
        state at the end; resume=True continues from it."""
        if x is None:
            x = self._new(self.shape_x)
        flags = (SFS_FISTA_WARM_START if warm_start else 0) | \
                (SFS_FISTA_TIME_KERNELS if time_kernels else 0) | \
                (SFS_FISTA_RESUME if resume else 0)
        hist = np.zeros(iters) if obj_hist else None
        sp = None if state is None else _dev_ptr(state, 2 * self.V + 2, "state")
        sfs_fista(self.handle, _dev_ptr(y, self.S * self.M, "y"), float(lam), float(L), iters,
                  _dev_ptr(x, self.V, "x"), sp, flags, hist, _stream_ptr(stream, y.device))
        return (x, hist) if obj_hist else x

    def fista_backtracking(self, y, lam, L0, eta, iters, x=None, stream=None):
        """sfs_fista_backtracking: (x, L_k per iteration)."""
        x = self._new(self.shape_x) if x is None else x
        hist = np.zeros(max(iters, 1))
        _check(lib().sfs_fista_backtracking(self.handle, _dev_ptr(y, self.S * self.M, "y"), float(lam),
                                            float(L0), float(eta), int(iters), _dev_ptr(x, self.V, "x"),
                                            hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            _stream_ptr(stream, y.device)))
        return x, hist[:iters]

    def kernel_times(self):
        return sfs_kernel_times(self.handle)

    def stage_times(self):
        """[forward contraction, residual planes, adjoint contraction, update
        planes] average ms per iteration of the last timed sfs_fista call."""
        return sfs_stage_times(self.handle)

    def set_wait_timeout_ns(self, ns: int):
        sfs_set_wait_timeout_ns(self.handle, ns)

    def inject_wait_timeout(self, enable: bool):
        sfs_inject_wait_timeout(self.handle, enable)

    def check_status(self, stream=None) -> int:
        import torch
        return sfs_check_status(self.handle, _stream_ptr(stream, torch.device("cuda", self.device)))

    def close(self):
        if self.handle and _lib is not None:
            _lib.sfs_destroy_operator(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class Mixing:
    """A_mix = Mix o A_band (sfs_mixing): Rademacher mixing of each A-scan
    before the DFT and selection.  band: Operator keeping the same signed
    bins at every position, at least the run ``Mixing.band_bins(geom)``;
    idx: int32 [S][M] kept bins; xi: int8 [S][Nt]."""

    @staticmethod
    def band_bins(geom: "Geometry"):
        """Signed bins (int32, ascending) within SFS_MIX_BAND_DB of the pulse
        peak: the spectrum a band operator for mixing must cover."""
        lo, hi = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sfs_mixing_band(geom.handle, ctypes.byref(lo), ctypes.byref(hi)))
        return np.arange(lo.value, hi.value + 1, dtype=np.int32)

    @classmethod
    def create(cls, geom: "Geometry", idx, xi, precision=None):
        """Band operator on ``band_bins(geom)`` (in `precision`) plus the
        mixing object on it; the mixing object keeps the band operator."""
        band = Operator.from_indices(geom, np.tile(cls.band_bins(geom), (geom.S, 1)), precision=precision)
        return cls(band, idx, xi)

    def __init__(self, band: "Operator", idx, xi):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        xi = np.ascontiguousarray(xi, dtype=np.int8)
        S, M = idx.shape
        if S != band.S or xi.shape != (band.S, band.geom.Nt):
            raise ValueError("idx must be [S][M] and xi [S][Nt]")
        self.band = band
        self.S, self.M, self.V = S, M, band.V
        self.shape_x = band.shape_x
        self.shape_y = (S, M)
        h = ctypes.c_void_p()
        _check(lib().sfs_mixing_create(band.handle, M, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       xi.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), ctypes.byref(h)))
        self.handle = h

    def _new(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.complex64, device="cuda:%d" % self.band.device)

    def apply_A(self, x, out=None, stream=None):
        y = self._new(self.shape_y) if out is None else out
        _check(lib().sfs_apply_A_mixed(self.handle, _dev_ptr(x, self.V, "x"), _dev_ptr(y, self.S * self.M, "y"),
                                       _stream_ptr(stream, x.device)))
        return y

    def apply_AH(self, y, out=None, stream=None):
        x = self._new(self.shape_x) if out is None else out
        _check(lib().sfs_apply_AH_mixed(self.handle, _dev_ptr(y, self.S * self.M, "y"), _dev_ptr(x, self.V, "x"),
                                        _stream_ptr(stream, y.device)))
        return x

    def lipschitz(self, max_iter=300, rtol=1e-6, seed=0, safety=1e-3, stream=None):
        out = ctypes.c_double()
        rc = _check(lib().sfs_lipschitz_mixed(self.handle, max_iter, rtol, seed, safety, ctypes.byref(out),
                                              _stream_ptr(stream, None)), allow=(SFS_ERR_NOT_CONVERGED,))
        return out.value, rc == SFS_OK

    def fista(self, y, lam, L, iters, x=None, stream=None):
        """lam >= 0: lambda; lam < 0: lambda = -lam * ||A_mix^H y||_inf."""
        x = self._new(self.shape_x) if x is None else x
        _check(lib().sfs_fista_mixed(self.handle, _dev_ptr(y, self.S * self.M, "y"), float(lam), float(L),
                                     int(iters), _dev_ptr(x, self.V, "x"), _stream_ptr(stream, y.device)))
        return x

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sfs_mixing_destroy(h)
            self.handle = None
