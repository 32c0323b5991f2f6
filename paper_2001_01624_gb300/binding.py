"""ctypes binding of the C ABI in include/ms.h -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it converts arguments (numpy arrays are passed as host
pointers, torch tensors as device pointers, torch streams as cudaStream_t),
calls the library, and raises :class:`MsError` on a failing status.  There is
no fallback: if the CUDA library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmsgb.so")

MS_OK, MS_ERR_INVALID_ARG, MS_ERR_OOM, MS_ERR_CUDA, MS_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
MS_ERR_COARSE_SINGULAR, MS_ERR_TIMEOUT, MS_ERR_STATE = 5, 6, 7
MS_PREC_FP64, MS_PREC_MIXED = 0, 1
MS_SMOOTHER_ILU0, MS_SMOOTHER_JACOBI = 0, 1
MS_OUTER_RICHARDSON, MS_OUTER_GMRES = 0, 1
MS_RESTRICT_GALERKIN, MS_RESTRICT_FV = 0, 1
MS_SUPPORT_BOX, MS_SUPPORT_HOP, MS_SUPPORT_BLOCK = 0, 1, 2

_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double


class MsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class ms_grid(C.Structure):
    _fields_ = [("nx", _i32), ("ny", _i32), ("nz", _i32), ("dx", _d), ("dy", _d), ("dz", _d),
                ("active", _vp), ("mult_x", _vp), ("mult_y", _vp), ("mult_z", _vp),
                ("n_nnc", _i32), ("nnc", _vp), ("nnc_axis", _vp), ("nnc_mult", _vp)]


class ms_system_info(C.Structure):
    _fields_ = [("n", _i64), ("n_faces", _i64), ("ell_width", _i32), ("n_levels", _i32), ("ref_cell", _i32)]


class ms_basis_opts(C.Structure):
    _fields_ = [("omega", _d), ("tol", _d), ("max_iter", _i32), ("precision", _i32), ("support", _i32),
                ("bx", _i32), ("by", _i32), ("bz", _i32)]


class ms_basis_info(C.Structure):
    _fields_ = [("M", _i32), ("nnz", _i64), ("max_overlap", _i32), ("iters", _i32), ("last_increment", _d)]


class ms_adapt_opts(C.Structure):
    _fields_ = [("n_bins", _i32), ("eps", _d), ("smoothed", _i32), ("omega", _d), ("tol", _d), ("max_iter", _i32),
                ("precision", _i32)]


class ms_solve_opts(C.Structure):
    _fields_ = [("tol", _d), ("max_iter", _i32), ("smoother", _i32), ("precision", _i32), ("jacobi_omega", _d),
                ("adapt_schedule", _i32), ("adapt", ms_adapt_opts), ("use_x0", _i32), ("outer", _i32),
                ("restart", _i32)]


class ms_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", _i64), ("timed_launches", _i64), ("total_ms", _d),
                ("bytes", _d)]


class ms_solve_info(C.Structure):
    _fields_ = [("iters", _i32), ("converged", _i32), ("rel_residual", _d), ("history", _vp),
                ("dyn_blocks", _vp), ("seconds", _d)]


class ms_fluid(C.Structure):
    _fields_ = [("mu_w", _d), ("mu_o", _d), ("n_w", _d), ("n_o", _d), ("s_wc", _d), ("s_or", _d),
                ("porosity", _d), ("cfl", _d)]


def fluid(mu_w=1.0, mu_o=3.0, n_w=2.0, n_o=2.0, s_wc=0.0, s_or=0.0, porosity=0.2, cfl=0.9) -> ms_fluid:
    return ms_fluid(mu_w, mu_o, n_w, n_o, s_wc, s_or, porosity, cfl)


class ms_cpr_fluid(C.Structure):
    _fields_ = [("mu_w", _d), ("mu_o", _d), ("n_w", _d), ("n_o", _d), ("s_wc", _d), ("s_or", _d), ("phi0", _d),
                ("rho_w0", _d), ("rho_o0", _d), ("c_w", _d), ("c_o", _d), ("c_r", _d), ("p_ref", _d)]


def cpr_fluid(mu_w=1e-3, mu_o=3e-3, n_w=2.0, n_o=2.0, s_wc=0.0, s_or=0.0, phi0=0.2, rho_w0=1000.0, rho_o0=800.0,
              c_w=4.5e-10, c_o=1.5e-9, c_r=5e-10, p_ref=2e7) -> ms_cpr_fluid:
    return ms_cpr_fluid(mu_w, mu_o, n_w, n_o, s_wc, s_or, phi0, rho_w0, rho_o0, c_w, c_o, c_r, p_ref)


class ms_batch_member(C.Structure):
    _fields_ = [("sys", _vp), ("stages", _vp), ("n_stages", _i32), ("q", _vp), ("p", _vp),
                ("info", C.POINTER(ms_solve_info)), ("rebuild", _vp), ("basis_iters", _i32), ("status", _i32)]


_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing): run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "ms_abi_version": ([], _i32),
        "ms_status_string": ([_i32], C.c_char_p),
        "ms_last_error": ([_vp], C.c_char_p),
        "ms_create": ([P(_vp), _i32, _vp], _i32),
        "ms_destroy": ([_vp], _i32),
        "ms_set_stream": ([_vp, _vp], _i32),
        "ms_system_create": ([_vp, P(ms_grid), _i32, P(_vp)], _i32),
        "ms_system_release": ([_vp], _i32),
        "ms_system_get_info": ([_vp, P(ms_system_info)], _i32),
        "ms_assemble_tpfa": ([_vp, _vp, _vp, _vp, _vp], _i32),
        "ms_system_get_matrix": ([_vp, _vp, _i32, _vp, _vp, _vp], _i32),
        "ms_spmv": ([_vp, _vp, _vp, _vp], _i32),
        "ms_ilu_apply": ([_vp, _vp, _i32, _vp, _vp], _i32),
        "ms_ilu_apply_noalloc": ([_vp, _vp, _vp, _vp], _i32),
        "ms_set_wait_limit": ([_vp, _vp, _d], _i32),
        "ms_debug_withhold_segments": ([_vp, _vp, _i32, _i32], _i32),
        "ms_plan_segments": ([_vp, _i32, _vp, _vp, _i32, _vp, P(_i32), _vp, _vp, P(_i32)], _i32),
        "ms_partition_cartesian": ([_vp, _vp, _i32, _i32, _i32, _vp, P(_i32)], _i32),
        "ms_partition_components": ([_vp, _vp, _vp, _vp, P(_i32)], _i32),
        "ms_partition_dynamic": ([_vp, _vp, _vp, _i32, _d, _vp, P(_i32)], _i32),
        "ms_build_basis": ([_vp, _vp, _vp, _i32, P(ms_basis_opts), P(_vp), P(_i32)], _i32),
        "ms_basis_rebuild": ([_vp, _vp, _vp, P(_i32)], _i32),
        "ms_basis_update": ([_vp, _vp, _vp, _d, _i32, P(_i32)], _i32),
        "ms_basis_release": ([_vp], _i32),
        "ms_basis_get_info": ([_vp, P(ms_basis_info)], _i32),
        "ms_basis_get": ([_vp, _vp, _vp, _vp, _vp], _i32),
        "ms_add_adaptive_basis": ([_vp, _vp, _vp, P(ms_adapt_opts), P(_vp)], _i32),
        "ms_galerkin": ([_vp, _vp, _vp, _i32, P(_vp)], _i32),
        "ms_coarse_create": ([_vp, _vp, _vp, _i32, _i32, P(_vp)], _i32),
        "ms_partition_wells": ([_vp, _vp, _i32, _vp, _vp, _vp, P(_i32)], _i32),
        "ms_dense_inverse": ([_vp, _i32, _vp, _vp], _i32),
        "ms_spd_inverse": ([_vp, _i32, _vp, _vp, _i32], _i32),
        "ms_coarse_get_inverse": ([_vp, _vp, _vp, P(_i32), P(_i32), P(_d), P(_i32)], _i32),
        "ms_cpr_pressure_system": ([_vp, _vp, _vp, P(ms_cpr_fluid), _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp],
                                   _i32),
        "ms_coarse_refresh": ([_vp, _vp, _vp], _i32),
        "ms_coarse_release": ([_vp], _i32),
        "ms_coarse_get": ([_vp, _vp, _vp, P(_i32)], _i32),
        "ms_solve": ([_vp, _vp, P(_vp), _i32, _vp, _vp, P(ms_solve_opts), P(ms_solve_info)], _i32),
        "ms_solve_batch": ([_vp, P(ms_batch_member), _i32, P(ms_solve_opts), _i32], _i32),
        "ms_basis_rebuild_batch": ([_vp, _vp, _vp, _i32, _vp], _i32),
        "ms_set_batch_tuning": ([_vp, _i32, _i32], _i32),
        "ms_total_mobility": ([_vp, _vp, P(ms_fluid), _vp, _vp], _i32),
        "ms_transport_step": ([_vp, _vp, P(ms_fluid), _vp, _vp, _d, _vp, P(_i32)], _i32),
        "ms_pressure_update": ([_vp, _vp, _vp, _vp, _vp], _i32),
        "ms_allocation_stats": ([P(_i64), P(_i64)], _i32),
        "ms_profile_enable": ([_i32], _i32),
        "ms_profile_reset": ([], _i32),
        "ms_profile_read": ([_vp, _i32, P(_i32), P(_i64)], _i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols() -> Sequence[str]:
    return ["ms_abi_version", "ms_status_string", "ms_last_error", "ms_create", "ms_destroy", "ms_set_stream",
            "ms_system_create", "ms_system_release", "ms_system_get_info", "ms_assemble_tpfa",
            "ms_system_get_matrix", "ms_spmv", "ms_ilu_apply", "ms_ilu_apply_noalloc", "ms_set_wait_limit",
            "ms_debug_withhold_segments", "ms_plan_segments", "ms_partition_cartesian", "ms_partition_components", "ms_partition_dynamic",
            "ms_partition_wells", "ms_coarse_create", "ms_dense_inverse", "ms_spd_inverse",
            "ms_coarse_get_inverse", "ms_cpr_pressure_system",
            "ms_build_basis", "ms_basis_rebuild", "ms_basis_update", "ms_basis_release", "ms_basis_get_info",
            "ms_basis_get", "ms_add_adaptive_basis", "ms_galerkin", "ms_coarse_refresh", "ms_coarse_release",
            "ms_coarse_get", "ms_solve", "ms_solve_batch", "ms_basis_rebuild_batch",
            "ms_set_batch_tuning", "ms_total_mobility", "ms_transport_step", "ms_pressure_update", "ms_allocation_stats", "ms_profile_enable", "ms_profile_reset", "ms_profile_read"]


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(st, ctx=None):
    if st != MS_OK:
        msg = lib().ms_last_error(ctx).decode() if ctx else ""
        name = lib().ms_status_string(st).decode()
        raise MsError(st, f"{name}: {msg}" if msg else name)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream        # torch.cuda.Stream


def _as(a, dtype):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ context
def ms_abi_version() -> int:
    return lib().ms_abi_version()


def ms_status_string(status: int) -> str:
    return lib().ms_status_string(status).decode()


def ms_last_error(ctx) -> str:
    return lib().ms_last_error(ctx).decode()


def ms_create(device: int = 0, stream=None):
    h = _vp()
    _check(lib().ms_create(C.byref(h), device, _stream_handle(stream)))
    return h


def ms_destroy(ctx):
    lib().ms_destroy(ctx)


def ms_set_stream(ctx, stream):
    _check(lib().ms_set_stream(ctx, _stream_handle(stream)), ctx)


# ------------------------------------------------------------------- system
def ms_system_create(ctx, grid, ref_cell: int = 0):
    keep = []

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    g = ms_grid(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, arr(grid.active, np.uint8),
                arr(grid.mult_x, np.float64), arr(grid.mult_y, np.float64), arr(grid.mult_z, np.float64),
                grid.n_nnc, arr(grid.nnc, np.int32) if grid.n_nnc else None,
                arr(grid.nnc_axis, np.int8) if grid.n_nnc else None,
                arr(grid.nnc_mult, np.float64) if grid.n_nnc else None)
    h = _vp()
    _check(lib().ms_system_create(ctx, C.byref(g), ref_cell, C.byref(h)), ctx)
    return h


def ms_system_release(sys):
    lib().ms_system_release(sys)


def ms_system_get_info(sys) -> dict:
    i = ms_system_info()
    _check(lib().ms_system_get_info(sys, C.byref(i)))
    return dict(n=i.n, n_faces=i.n_faces, ell_width=i.ell_width, n_levels=i.n_levels, ref_cell=i.ref_cell)


def ms_assemble_tpfa(ctx, sys, perm, mobility=None, p_prev=None):
    perm, mobility, p_prev = _as(perm, np.float64), _as(mobility, np.float64), _as(p_prev, np.float64)
    _check(lib().ms_assemble_tpfa(ctx, sys, _ptr(perm), _ptr(mobility), _ptr(p_prev)), ctx)


def ms_system_get_matrix(ctx, sys, pinned: bool = True):
    info = ms_system_get_info(sys)
    n, W = info["n"], info["ell_width"]
    col = np.empty(max(W * n, 1), np.int32)
    val = np.empty(max(W * n, 1))
    diag = np.empty(n)
    _check(lib().ms_system_get_matrix(ctx, sys, int(pinned), _ptr(col), _ptr(val), _ptr(diag)), ctx)
    return col[: W * n].reshape(W, n), val[: W * n].reshape(W, n), diag


def ms_spmv(ctx, sys, x, y):
    _check(lib().ms_spmv(ctx, sys, _ptr(_as(x, np.float64)), _ptr(y)), ctx)


def ms_ilu_apply(ctx, sys, r, z, precision: int = MS_PREC_FP64):
    _check(lib().ms_ilu_apply(ctx, sys, precision, _ptr(_as(r, np.float64)), _ptr(z)), ctx)


def ms_ilu_apply_noalloc(ctx, sys, r, z):
    """Allocation-free ILU(0) application: r and z must be device tensors."""
    _check(lib().ms_ilu_apply_noalloc(ctx, sys, _ptr(r), _ptr(z)), ctx)


def ms_set_wait_limit(ctx, sys, seconds: float):
    _check(lib().ms_set_wait_limit(ctx, sys, float(seconds)), ctx)


def ms_debug_withhold_segments(ctx, sys, count: int, precision: int = MS_PREC_FP64):
    _check(lib().ms_debug_withhold_segments(ctx, sys, precision, int(count)), ctx)


# --------------------------------------------------------------- partitions
def ms_partition_cartesian(ctx, sys, block):
    n = ms_system_get_info(sys)["n"]
    part = np.empty(n, np.int32)
    m = _i32()
    _check(lib().ms_partition_cartesian(ctx, sys, int(block[0]), int(block[1]), int(block[2]), _ptr(part),
                                        C.byref(m)), ctx)
    return part, m.value


def ms_plan_segments(rowptr, col, max_len: int = 256, ctx=None) -> dict:
    """Segments of the ILU(0) segment sweeps for a CSR row pattern (host only,
    no GPU needed): seg_off (starts, then n), the forward and backward
    hand-out orders, kg (most couplings of a row leaving its segment, towards
    lower / higher rows) and the widest level."""
    rp = np.ascontiguousarray(rowptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32) if len(col) else np.zeros(1, np.int32)
    n = len(rp) - 1
    off = np.empty(max(n, 0) + 1, np.int32)
    order = np.empty(max(2 * n, 1), np.int32)
    kg = np.empty(2, np.int32)
    ns, width = _i32(), _i32()
    _check(lib().ms_plan_segments(ctx, n, _ptr(rp), _ptr(cl), max_len, _ptr(off), C.byref(ns), _ptr(order), _ptr(kg),
                                  C.byref(width)), ctx)
    k = ns.value
    return dict(seg_off=off[:k + 1].copy(), order_fwd=order[:k].copy(), order_bwd=order[k:2 * k].copy(),
                kg=(int(kg[0]), int(kg[1])), width=width.value)


def ms_partition_wells(ctx, sys, wells):
    """wells: sequence of active-cell index lists; returns (part, n_blocks)."""
    n = ms_system_get_info(sys)["n"]
    ptr = np.zeros(len(wells) + 1, np.int32)
    for w, c in enumerate(wells):
        ptr[w + 1] = ptr[w] + len(c)
    cells = (np.concatenate([np.asarray(c, np.int32) for c in wells]) if len(wells) else np.zeros(1, np.int32))
    cells = np.ascontiguousarray(cells, np.int32)
    part = np.empty(n, np.int32)
    m = _i32()
    _check(lib().ms_partition_wells(ctx, sys, len(wells), _ptr(ptr), _ptr(cells), _ptr(part), C.byref(m)), ctx)
    return part, m.value


def ms_partition_components(ctx, sys, cls, part) -> int:
    m = _i32()
    _check(lib().ms_partition_components(ctx, sys, _ptr(_as(cls, np.int32)), _ptr(part), C.byref(m)), ctx)
    return m.value


def ms_partition_dynamic(ctx, sys, dp, part, n_bins: int = 8, eps: float = 1e-8) -> int:
    m = _i32()
    _check(lib().ms_partition_dynamic(ctx, sys, _ptr(_as(dp, np.float64)), n_bins, eps, _ptr(part), C.byref(m)),
           ctx)
    return m.value


# -------------------------------------------------------------------- basis
def ms_build_basis(ctx, sys, partition, n_blocks: int, omega=2.0 / 3.0, tol=1e-3, max_iter=500,
                   precision=MS_PREC_FP64, support=MS_SUPPORT_BOX, block=(1, 1, 1)):
    o = ms_basis_opts(omega, tol, max_iter, precision, support, int(block[0]), int(block[1]), int(block[2]))
    h = _vp()
    it = _i32()
    part = np.ascontiguousarray(partition, dtype=np.int32)
    _check(lib().ms_build_basis(ctx, sys, _ptr(part), n_blocks, C.byref(o), C.byref(h), C.byref(it)), ctx)
    return h, it.value


def ms_basis_rebuild(ctx, sys, basis) -> int:
    it = _i32()
    _check(lib().ms_basis_rebuild(ctx, sys, basis, C.byref(it)), ctx)
    return it.value


def ms_basis_update(ctx, sys, basis, tol: float, max_iter: int) -> int:
    it = _i32()
    _check(lib().ms_basis_update(ctx, sys, basis, tol, max_iter, C.byref(it)), ctx)
    return it.value


def ms_basis_release(basis):
    lib().ms_basis_release(basis)


def ms_basis_get_info(basis) -> dict:
    i = ms_basis_info()
    _check(lib().ms_basis_get_info(basis, C.byref(i)))
    return dict(M=i.M, nnz=i.nnz, max_overlap=i.max_overlap, iters=i.iters, last_increment=i.last_increment)


def ms_basis_get(ctx, basis):
    info = ms_basis_get_info(basis)
    cptr = np.empty(info["M"] + 1, np.int32)
    cells = np.empty(max(info["nnz"], 1), np.int32)
    val = np.empty(max(info["nnz"], 1))
    _check(lib().ms_basis_get(ctx, basis, _ptr(cptr), _ptr(cells), _ptr(val)), ctx)
    return cptr, cells[: info["nnz"]], val[: info["nnz"]]


def ms_add_adaptive_basis(ctx, sys, dp, n_bins=8, eps=1e-8, smoothed=0, omega=2.0 / 3.0, tol=1e-3, max_iter=500,
                          precision=MS_PREC_FP64):
    o = ms_adapt_opts(n_bins, eps, smoothed, omega, tol, max_iter, precision)
    h = _vp()
    _check(lib().ms_add_adaptive_basis(ctx, sys, _ptr(_as(dp, np.float64)), C.byref(o), C.byref(h)), ctx)
    return h


# ------------------------------------------------------------------- coarse
def ms_galerkin(ctx, sys, basis, precision=MS_PREC_FP64):
    h = _vp()
    _check(lib().ms_galerkin(ctx, sys, basis, precision, C.byref(h)), ctx)
    return h


def ms_coarse_create(ctx, sys, basis, precision=MS_PREC_FP64, restriction=MS_RESTRICT_GALERKIN):
    h = _vp()
    _check(lib().ms_coarse_create(ctx, sys, basis, precision, restriction, C.byref(h)), ctx)
    return h


def ms_dense_inverse(ctx, A):
    """A^{-1} by the finite-volume stages' Gauss-Jordan kernel (FP64)."""
    A = np.ascontiguousarray(A, np.float64)
    X = np.empty_like(A)
    _check(lib().ms_dense_inverse(ctx, A.shape[0], _ptr(A), _ptr(X)), ctx)
    return X


def ms_spd_inverse(ctx, A, precision=MS_PREC_FP64):
    """A^{-1} of a symmetric positive definite matrix by the coarse stages'
    blocked sweep (FP64, or FP32 on the tensor cores for MS_PREC_MIXED)."""
    A = np.ascontiguousarray(A, np.float64)
    X = np.empty_like(A)
    _check(lib().ms_spd_inverse(ctx, A.shape[0], _ptr(A), _ptr(X), precision), ctx)
    return X


def ms_cpr_pressure_system(ctx, sys, perm, fluid, p, s, p0, s0, q_w, q_o, dt, rhs=None, weights=None):
    """Replace the system's matrix by the CPR pressure matrix J* (quasi-IMPES)
    of the compressible two-phase step; returns rhs = -(W_w R_w + W_o R_o)
    (numpy unless an output tensor is given).  weights: optional 2n output."""
    n = ms_system_get_info(sys)["n"]
    out = np.empty(n) if rhs is None else rhs
    _check(lib().ms_cpr_pressure_system(ctx, sys, _ptr(_as(perm, np.float64)), C.byref(fluid), _ptr(_as(p, np.float64)),
                                        _ptr(_as(s, np.float64)), _ptr(_as(p0, np.float64)), _ptr(_as(s0, np.float64)),
                                        _ptr(_as(q_w, np.float64)), _ptr(_as(q_o, np.float64)), float(dt), _ptr(out),
                                        _ptr(weights)), ctx)
    return out


def ms_coarse_refresh(ctx, sys, coarse):
    _check(lib().ms_coarse_refresh(ctx, sys, coarse), ctx)


def ms_coarse_release(coarse):
    lib().ms_coarse_release(coarse)


def ms_coarse_get(ctx, coarse):
    m = _i32()
    _check(lib().ms_coarse_get(ctx, coarse, None, C.byref(m)), ctx)
    Ac = np.empty((m.value, m.value))
    _check(lib().ms_coarse_get(ctx, coarse, _ptr(Ac), C.byref(m)), ctx)
    return Ac


def ms_coarse_get_inverse(ctx, coarse):
    """dict(X, fp64, inv_error, refine_steps): the coarse inverse the stage applies."""
    m, f, k = _i32(), _i32(), _i32()
    e = _d()
    _check(lib().ms_coarse_get_inverse(ctx, coarse, None, C.byref(m), None, None, None), ctx)
    X = np.empty((m.value, m.value))
    _check(lib().ms_coarse_get_inverse(ctx, coarse, _ptr(X), C.byref(m), C.byref(f), C.byref(e), C.byref(k)), ctx)
    return dict(X=X, fp64=bool(f.value), inv_error=e.value, refine_steps=k.value)


# -------------------------------------------------------------------- solve
def ms_solve(ctx, sys, stages, q, p, tol=1e-6, max_iter=500, smoother=MS_SMOOTHER_ILU0, precision=MS_PREC_FP64,
             jacobi_omega=2.0 / 3.0, adapt_schedule=0, adapt: Optional[dict] = None, use_x0=False,
             raise_not_converged=False, outer=0, restart=30) -> dict:
    """Returns dict(status, iters, converged, rel_residual, history, dyn_blocks, seconds)."""
    ad = dict(n_bins=8, eps=1e-8, smoothed=0, omega=2.0 / 3.0, tol=1e-3, max_iter=500)
    ad.update(adapt or {})
    o = ms_solve_opts(tol, max_iter, smoother, precision, jacobi_omega, adapt_schedule,
                      ms_adapt_opts(ad["n_bins"], ad["eps"], ad["smoothed"], ad["omega"], ad["tol"], ad["max_iter"],
                                    precision),
                      int(use_x0), int(outer), int(restart))
    hist = np.zeros(max_iter + 1)
    dyn = np.zeros(max(max_iter, 1), np.int32)
    info = ms_solve_info(0, 0, 0.0, hist.ctypes.data, dyn.ctypes.data, 0.0)
    arr = (_vp * max(len(stages), 1))(*[s.value if isinstance(s, _vp) else s for s in stages])
    q = _as(q, np.float64)
    st = lib().ms_solve(ctx, sys, arr, len(stages), _ptr(q), _ptr(p), C.byref(o), C.byref(info))
    if st not in (MS_OK, MS_ERR_NOT_CONVERGED) or (st == MS_ERR_NOT_CONVERGED and raise_not_converged):
        _check(st, ctx)
    return dict(status=st, iters=info.iters, converged=bool(info.converged), rel_residual=info.rel_residual,
                history=hist[: info.iters + 1].copy(), dyn_blocks=dyn[: info.iters].copy(), seconds=info.seconds)


def ms_solve_batch(ctx, members: Sequence[dict], tol=1e-6, max_iter=500, smoother=MS_SMOOTHER_ILU0,
                   precision=MS_PREC_FP64, jacobi_omega=2.0 / 3.0, n_workers=0, outer=0, restart=30) -> list:
    """Batched solve of independent members.  Each member is a dict with
    keys sys, stages, q, p and optionally rebuild (a basis to re-smooth
    first).  Returns one dict per member: status, iters, converged,
    rel_residual, history, basis_iters, seconds."""
    o = ms_solve_opts(tol, max_iter, smoother, precision, jacobi_omega, 0, ms_adapt_opts(8, 1e-8, 0, 2.0 / 3.0, 1e-3, 500, precision), 0,
                      int(outer), int(restart))
    n = len(members)
    arr = (ms_batch_member * max(n, 1))()
    keep = []
    hists = []
    infos = (ms_solve_info * max(n, 1))()
    for k, m in enumerate(members):
        st_arr = (_vp * max(len(m["stages"]), 1))(*[s.value if isinstance(s, _vp) else s for s in m["stages"]])
        q = _as(m["q"], np.float64)
        hist = np.zeros(max_iter + 1)
        infos[k] = ms_solve_info(0, 0, 0.0, hist.ctypes.data, None, 0.0)
        keep += [st_arr, q]
        hists.append(hist)
        rb = m.get("rebuild")
        arr[k] = ms_batch_member(m["sys"].value if isinstance(m["sys"], _vp) else m["sys"], C.cast(st_arr, _vp),
                                 len(m["stages"]), _ptr(q), _ptr(m["p"]), C.pointer(infos[k]),
                                 (rb.value if isinstance(rb, _vp) else rb) if rb is not None else None, 0, -1)
    st = lib().ms_solve_batch(ctx, arr, n, C.byref(o), n_workers)
    if st not in (MS_OK, MS_ERR_NOT_CONVERGED):
        _check(st, ctx)
    out = []
    for k in range(n):
        i = infos[k]
        out.append(dict(status=arr[k].status, iters=i.iters, converged=bool(i.converged), rel_residual=i.rel_residual,
                        history=hists[k][: i.iters + 1].copy(), basis_iters=arr[k].basis_iters, seconds=i.seconds))
    return out


def _h(x):
    return x.value if isinstance(x, _vp) else x


def ms_pressure_update(ctx, sys, p, p_prev, dp):
    """dp = p - p_prev on the device (torch tensors of the context's device)."""
    _check(lib().ms_pressure_update(ctx, sys, _ptr(p), _ptr(p_prev), _ptr(dp)), ctx)


def ms_allocation_stats() -> dict:
    """dict(thread_bytes, allocations) of the library's device allocations."""
    b, n = _i64(), _i64()
    _check(lib().ms_allocation_stats(C.byref(b), C.byref(n)))
    return dict(thread_bytes=b.value, allocations=n.value)


def ms_basis_rebuild_batch(ctx, systems: Sequence, bases: Sequence) -> np.ndarray:
    """Re-smooth bases[m] of systems[m] from the block indicator, all in one
    persistent launch per precision; returns the iteration counts."""
    n = len(systems)
    sa = (_vp * max(n, 1))(*[_h(x) for x in systems])
    ba = (_vp * max(n, 1))(*[_h(x) for x in bases])
    it = np.zeros(max(n, 1), np.int32)
    _check(lib().ms_basis_rebuild_batch(ctx, C.cast(sa, _vp), C.cast(ba, _vp), n, _ptr(it)), ctx)
    return it[:n]


def ms_set_batch_tuning(ctx, tile_cells: int, ctas_per_sm: int):
    _check(lib().ms_set_batch_tuning(ctx, int(tile_cells), int(ctas_per_sm)), ctx)


# ---------------------------------------------------------------- two-phase
def ms_total_mobility(ctx, sys, fl: ms_fluid, S, lam=None):
    """lambda_t per active cell; S, lam: numpy arrays or device tensors."""
    S = _as(S, np.float64)
    if lam is None:
        lam = np.empty(len(S))
    _check(lib().ms_total_mobility(ctx, sys, C.byref(fl), _ptr(S), _ptr(lam)), ctx)
    return lam


def ms_transport_step(ctx, sys, fl: ms_fluid, p, q, dt, S) -> int:
    """Advance S (updated in place) over dt; returns the substep count."""
    p = _as(p, np.float64)
    q = _as(q, np.float64)
    k = _i32()
    _check(lib().ms_transport_step(ctx, sys, C.byref(fl), _ptr(p), _ptr(q), float(dt), _ptr(S), C.byref(k)), ctx)
    return k.value


# ------------------------------------------------------------------ tracing
def ms_profile_enable(on: bool = True):
    _check(lib().ms_profile_enable(int(on)))


def ms_profile_reset():
    _check(lib().ms_profile_reset())


def ms_profile_read() -> dict:
    """Per kernel family: dict(launches, timed_launches, total_ms, bytes); key
    '_total_launches' holds the launch count over all families."""
    cnt = _i32()
    tot = _i64()
    _check(lib().ms_profile_read(None, 0, C.byref(cnt), C.byref(tot)))
    arr = (ms_kernel_stat * max(cnt.value, 1))()
    _check(lib().ms_profile_read(arr, cnt.value, C.byref(cnt), C.byref(tot)))
    out = {a.name.decode(): dict(launches=a.launches, timed_launches=a.timed_launches, total_ms=a.total_ms,
                                 bytes=a.bytes) for a in arr[: cnt.value]}
    out["_total_launches"] = tot.value
    return out
