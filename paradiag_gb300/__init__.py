"""GB300-native ParaDiag-II: the alpha-circulant preconditioned all-at-once solver.

The compute path is the CUDA library ``lib/libparadiag.so`` (sm_103a) behind
the C ABI of ``include/paradiag.h``.  This module only marshals arguments:
the functions ``pd_*`` below have the names and argument order of the C
entry points and take raw device pointers; :class:`Plan` wraps them for torch
tensors and :class:`PDSolve` makes the solve differentiable (its backward is
the transposed all-at-once solve).  There is no CPU fallback: loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from ._build import build, lib_path

PD_OK, PD_ERR_ARG, PD_ERR_CUDA, PD_ERR_NOT_CONVERGED = 0, -1, -2, -3
PD_ERR_NONFINITE, PD_ERR_UNSUPPORTED, PD_ERR_NOMEM = -4, -5, -6
PD_BE, PD_CN, PD_THETA, PD_LEAPFROG = 0, 1, 2, 3
PD_DIRICHLET, PD_PERIODIC = 0, 1
PD_FP64, PD_MIXED = 0, 1
PD_STATIONARY, PD_GMRES = 0, 1


class pd_space(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nu", ctypes.c_double), ("ax", ctypes.c_double), ("ay", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double)]


class pd_problem(ctypes.Structure):
    _fields_ = [("space", pd_space), ("nt", ctypes.c_int), ("dt", ctypes.c_double),
                ("alpha", ctypes.c_double), ("scheme", ctypes.c_int), ("theta", ctypes.c_double)]


class PDError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{pd_status_string(status)} ({status}): {msg}")


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "pd_plan_create": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      _P, ctypes.POINTER(_P)]),
    "pd_plan_destroy": (ctypes.c_int, [_P]),
    "pd_plan_workspace": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd_apply_precond": (ctypes.c_int, [_P, _P, _P]),
    "pd_debug_xform_timeout": (ctypes.c_int, [_P, _P, _P]),
    "pd_residual": (ctypes.c_int, [_P, _P, _P, _P]),
    "pd_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "pd_apply_AT": (ctypes.c_int, [_P, _P, _P]),
    "pd_build_rhs": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pd_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, _I, _D]),
    "pd_solve_async": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int]),
    "pd_solve_result": (ctypes.c_int, [_P, _I, _D]),
    "pd_solve_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, _I, _D]),
    "pd_adjoint_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _I, _D]),
    "pd_profile_iteration": (ctypes.c_int, [_P, _P, _P, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_float)]),
    "pd_plan_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd_profile_precond": (ctypes.c_int, [_P, _P, _P, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_float)]),
    "pd_plan_uses_graph": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "pd_plan_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pd_plan_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "pd_plan_set_tuning": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pd_plan_xform_engine": (ctypes.c_int, [_P, _I]),
    "pd_plan_set_xform_engine": (ctypes.c_int, [_P, ctypes.c_int]),
    "pd_plan_time_cluster": (ctypes.c_int, [_P, _I]),
    "pd_plan_set_time_cluster": (ctypes.c_int, [_P, ctypes.c_int]),
    "pd_apply_precond_noalloc": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, _P, _P, _P,
                                                ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd_batch_create": (ctypes.c_int, [ctypes.POINTER(pd_problem), ctypes.c_int, ctypes.c_int, _P,
                                       ctypes.POINTER(_P)]),
    "pd_batch_destroy": (ctypes.c_int, [_P]),
    "pd_batch_offsets": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd_batch_build_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "pd_batch_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _I, _D]),
    "pd_batch_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd_batch_uses_graph": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "pd_batch_relres": (ctypes.c_int, [_P, _D]),
    "pd_precond_forward": (ctypes.c_int, [_P, _P]),
    "pd_plan_spectrum": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "pd_precond_solve_rows": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "pd_spectrum_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "pd_spectrum_put": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "pd_precond_backward": (ctypes.c_int, [_P, _P]),
    "pd_shard_norm2": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "pd_shard_update": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "pd_batch_tuned": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "pd_batch_profile_sweep": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "pd_batch_last_error": (ctypes.c_char_p, [_P]),
    "pd1_plan_create": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _P, ctypes.POINTER(_P)]),
    "pd1_plan_destroy": (ctypes.c_int, [_P]),
    "pd1_step_sizes": (ctypes.c_int, [_P, _D]),
    "pd1_condition": (ctypes.c_int, [_P, _D]),
    "pd1_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "pd1_build_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "pd1_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _I, _D]),
    "pd1_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd1_solve_windows": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int,
                                         _I, _D]),
    "pd_solve_windows": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _I, _D]),
    "pd_nl_build_rhs": (ctypes.c_int, [_P, _D, _P, _P, _P]),
    "pd_nl_residual": (ctypes.c_int, [_P, _D, _P, _P, _P, _D, _D]),
    "pd_nl_solve": (ctypes.c_int, [_P, _D, _P, _P, ctypes.c_double, ctypes.c_int, _I, _D]),
    "pd_nl_solve_windows": (ctypes.c_int, [_P, _D, _P, _P, ctypes.c_int, _P, ctypes.c_double,
                                           ctypes.c_int, _I, _D]),
    "pd1_profile_sweep": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "pd1_workspace": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pd1_last_error": (ctypes.c_char_p, [_P]),
    "pdh_plan_create": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "pdh_plan_destroy": (ctypes.c_int, [_P]),
    "pdh_eigenvalues": (ctypes.c_int, [_P, _D]),
    "pdh_wave_plan_create": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "pdh_wave_build_rhs": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pdh_condition": (ctypes.c_int, [_P, _D]),
    "pdh_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "pdh_build_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "pdh_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _I, _D]),
    "pdh_profile_sweep": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "pdh_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pdh_last_error": (ctypes.c_char_p, [_P]),
    "pdh_set_tensor_cores": (ctypes.c_int, [_P, ctypes.c_int]),
    "pdh_tensor_cores": (ctypes.c_int, [_P, _I]),
    "pdc_plan_create": (ctypes.c_int, [ctypes.POINTER(pd_space), ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "pdc_plan_destroy": (ctypes.c_int, [_P]),
    "pdc_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "pdc_apply_precond": (ctypes.c_int, [_P, _P, _P]),
    "pdc_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _I, _D]),
    "pdc_solve_left": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _I,
                                      _D]),
    "pdc_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pdc_last_error": (ctypes.c_char_p, [_P]),
    "pd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pd_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it is missing; there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"ParaDiag CUDA library not built: {path} is missing "
                           "(run paradiag_gb300.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


# --- the C entry points, same names and argument order ---------------------
def pd_status_string(status: int) -> str:
    return load().pd_status_string(status).decode()


def pd_last_error(plan) -> str:
    return load().pd_last_error(plan).decode()


def pd_plan_create(space: pd_space, nt, dt, alpha, scheme, theta, precision, stream):
    out = _P()
    st = load().pd_plan_create(ctypes.byref(space), nt, dt, alpha, scheme, theta, precision,
                               _P(stream), ctypes.byref(out))
    return st, out.value


def pd_plan_destroy(plan):
    return load().pd_plan_destroy(plan)


def pd_plan_workspace(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pd_plan_workspace(plan, ctypes.byref(v))
    return st, v.value


def pd_profile_iteration(plan, b, u, reps):
    ms = (ctypes.c_float * 5)()
    st = load().pd_profile_iteration(plan, b, u, reps, ms)
    return st, list(ms)


def pd_profile_precond(plan, r, z, reps):
    ms = (ctypes.c_float * 5)()
    st = load().pd_profile_precond(plan, r, z, reps, ms)
    return st, list(ms)


def pd_plan_launches(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pd_plan_launches(plan, ctypes.byref(v))
    return st, v.value


def pd_plan_uses_graph(plan):
    v = ctypes.c_int(0)
    st = load().pd_plan_uses_graph(plan, ctypes.byref(v))
    return st, v.value


def pd_plan_tuning(plan):
    tx = ctypes.c_int(0)
    lanes = ctypes.c_int(0)
    st = load().pd_plan_tuning(plan, ctypes.byref(tx), ctypes.byref(lanes))
    return st, tx.value, lanes.value


def pd_plan_get_tuning(plan):
    tx = ctypes.c_int(0)
    lanes = ctypes.c_int(0)
    rows = ctypes.c_int(0)
    st = load().pd_plan_get_tuning(plan, ctypes.byref(tx), ctypes.byref(lanes), ctypes.byref(rows))
    return st, tx.value, lanes.value, rows.value


def pd_plan_set_tuning(plan, tile_columns, tri_lanes, tri_rows):
    return load().pd_plan_set_tuning(plan, int(tile_columns), int(tri_lanes), int(tri_rows))


PD_XFORM_TENSOR, PD_XFORM_FFT, PD_XFORM_DENSE = 0, 1, 2


def pd_plan_xform_engine(plan):
    v = ctypes.c_int(0)
    st = load().pd_plan_xform_engine(plan, ctypes.byref(v))
    return st, v.value


def pd_plan_set_xform_engine(plan, engine):
    return load().pd_plan_set_xform_engine(plan, int(engine))


def pd_plan_time_cluster(plan):
    v = ctypes.c_int(0)
    st = load().pd_plan_time_cluster(plan, ctypes.byref(v))
    return st, v.value


def pd_plan_set_time_cluster(plan, blocks):
    return load().pd_plan_set_time_cluster(plan, int(blocks))


def pd_batch_uses_graph(batch):
    v = ctypes.c_int(0)
    st = load().pd_batch_uses_graph(batch, ctypes.byref(v))
    return st, v.value


def pd_apply_precond(plan, r, z):
    return load().pd_apply_precond(plan, r, z)


def pd_debug_xform_timeout(plan, r, z):
    return load().pd_debug_xform_timeout(plan, r, z)


def pd_apply_precond_noalloc(space, nt, dt, alpha, scheme, theta, r, z, stream):
    """Plan-free, allocation-free P^{-1} r for 1D Dirichlet problems; returns
    (status, scratch bytes the problem needs)."""
    need = ctypes.c_ulonglong(0)
    st = load().pd_apply_precond_noalloc(ctypes.byref(space), nt, dt, alpha, scheme, theta, r, z,
                                         _P(stream), ctypes.byref(need))
    return st, need.value


def pd_batch_create(problems, precision, stream):
    arr = (pd_problem * len(problems))(*problems)
    out = _P()
    st = load().pd_batch_create(arr, len(problems), precision, _P(stream), ctypes.byref(out))
    return st, out.value


def pd_batch_destroy(batch):
    return load().pd_batch_destroy(batch)


def pd_batch_offsets(batch, nprob):
    off = (ctypes.c_ulonglong * (nprob + 1))()
    st = load().pd_batch_offsets(batch, off)
    return st, list(off)


def pd_batch_build_rhs(batch, u0, f, b):
    return load().pd_batch_build_rhs(batch, u0, f, b)


def pd_batch_solve(batch, b, u, tol, maxit):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = load().pd_batch_solve(batch, b, u, tol, maxit, ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def pd_batch_launches(batch):
    v = ctypes.c_ulonglong(0)
    st = load().pd_batch_launches(batch, ctypes.byref(v))
    return st, v.value


def pd_batch_relres(batch, nprob):
    arr = (ctypes.c_double * nprob)()
    st = load().pd_batch_relres(batch, arr)
    return st, list(arr)


def pd_precond_forward(plan, r):
    return load().pd_precond_forward(plan, r)


def pd_plan_spectrum(plan):
    data = ctypes.c_void_p(0)
    nh, lines, pitch, eb = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    st = load().pd_plan_spectrum(plan, ctypes.byref(data), ctypes.byref(nh), ctypes.byref(lines),
                                 ctypes.byref(pitch), ctypes.byref(eb))
    return st, data.value, nh.value, lines.value, pitch.value, eb.value


def pd_spectrum_get(plan, k0, k1, l0, l1, dst):
    return load().pd_spectrum_get(plan, int(k0), int(k1), int(l0), int(l1), dst)


def pd_spectrum_put(plan, k0, k1, l0, l1, src):
    return load().pd_spectrum_put(plan, int(k0), int(k1), int(l0), int(l1), src)


def pd_precond_solve_rows(plan, k0, k1, data):
    return load().pd_precond_solve_rows(plan, int(k0), int(k1), data)


def pd_precond_backward(plan, z):
    return load().pd_precond_backward(plan, z)


def pd_shard_norm2(plan, x, first_line, nlines):
    v = ctypes.c_double(0.0)
    st = load().pd_shard_norm2(plan, x, int(first_line), int(nlines), ctypes.byref(v))
    return st, v.value


def pd_shard_update(plan, z, u, first_line, nlines):
    return load().pd_shard_update(plan, z, u, int(first_line), int(nlines))


def pd_batch_tuned(batch):
    v = ctypes.c_int(0)
    st = load().pd_batch_tuned(batch, ctypes.byref(v))
    return st, v.value


def pd_batch_profile_sweep(batch, b, u, reps):
    ms = (ctypes.c_float * 3)()
    st = load().pd_batch_profile_sweep(batch, b, u, int(reps), ms)
    return st, list(ms)


def pd_batch_last_error(batch):
    return load().pd_batch_last_error(batch).decode()


def pd_residual(plan, b, u, r):
    return load().pd_residual(plan, b, u, r)


def pd_apply_A(plan, u, y):
    return load().pd_apply_A(plan, u, y)


def pd_apply_AT(plan, u, y):
    return load().pd_apply_AT(plan, u, y)


def pd_build_rhs(plan, u0, u1, f, b):
    return load().pd_build_rhs(plan, u0, u1, f, b)


def _solve_call(fn, plan, b, u, mode, tol, maxit, restart):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = fn(plan, b, u, mode, tol, maxit, restart, ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def pd_solve(plan, b, u, mode, tol, maxit, restart):
    return _solve_call(load().pd_solve, plan, b, u, mode, tol, maxit, restart)


def pd_solve_async(plan, b, u, tol, maxit):
    return load().pd_solve_async(plan, b, u, tol, maxit)


def pd_solve_result(plan):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd_solve_result(plan, ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def pd_solve_host(plan, b, u, mode, tol, maxit, restart):
    return _solve_call(load().pd_solve_host, plan, b, u, mode, tol, maxit, restart)


def pd_adjoint_solve(plan, g, lam, mode, tol, maxit, restart):
    return _solve_call(load().pd_adjoint_solve, plan, g, lam, mode, tol, maxit, restart)


# --- torch convenience layer ----------------------------------------------
def pd1_plan_create(space: pd_space, nt, dt_last, tau, scheme, column_scaling, precision, stream):
    out = _P()
    st = load().pd1_plan_create(ctypes.byref(space), nt, dt_last, tau, scheme, column_scaling,
                                precision, _P(stream), ctypes.byref(out))
    return st, out.value


def pd1_plan_destroy(plan):
    return load().pd1_plan_destroy(plan)


def pd1_step_sizes(plan, nt):
    buf = (ctypes.c_double * nt)()
    st = load().pd1_step_sizes(plan, buf)
    return st, list(buf)


def pd1_condition(plan):
    v = ctypes.c_double(0.0)
    st = load().pd1_condition(plan, ctypes.byref(v))
    return st, v.value


def pd1_apply_A(plan, u, y):
    return load().pd1_apply_A(plan, u, y)


def pd1_build_rhs(plan, u0, f, b):
    return load().pd1_build_rhs(plan, u0, f, b)


def pd1_solve(plan, b, u, tol, max_refine):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd1_solve(plan, b, u, tol, max_refine, ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def pd1_profile_sweep(plan, b, u, reps):
    ms = (ctypes.c_float * 3)()
    st = load().pd1_profile_sweep(plan, b, u, reps, ms)
    return st, list(ms)


def pd1_solve_windows(plan, u0, f, nwin, u, tol, max_refine):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd1_solve_windows(plan, u0, f, nwin, u, tol, max_refine, ctypes.byref(it),
                                  ctypes.byref(rr))
    return st, it.value, rr.value


def pd_solve_windows(plan, u0, f, nwin, u, mode, tol, maxit, restart):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd_solve_windows(plan, u0, f, nwin, u, mode, tol, maxit, restart,
                                 ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def _reaction(a):
    if len(a) != 3:
        raise ValueError("reaction coefficients: (a1, a2, a3)")
    return (ctypes.c_double * 3)(*[float(v) for v in a])


def pd_nl_build_rhs(plan, a, u0, f, b):
    return load().pd_nl_build_rhs(plan, _reaction(a), u0, f, b)


def pd_nl_residual(plan, a, b, u, r, scalars=True):
    """scalars=False: no sigma / ||r||^2 read-back (no stream synchronisation)."""
    if not scalars:
        return load().pd_nl_residual(plan, _reaction(a), b, u, r, None, None), None, None
    sig = ctypes.c_double(0.0)
    rn2 = ctypes.c_double(0.0)
    st = load().pd_nl_residual(plan, _reaction(a), b, u, r, ctypes.byref(sig), ctypes.byref(rn2))
    return st, sig.value, rn2.value


def pd_nl_solve(plan, a, b, u, tol, maxit):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd_nl_solve(plan, _reaction(a), b, u, tol, maxit, ctypes.byref(it),
                            ctypes.byref(rr))
    return st, it.value, rr.value


def pd_nl_solve_windows(plan, a, u0, f, nwin, u, tol, maxit):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pd_nl_solve_windows(plan, _reaction(a), u0, f, nwin, u, tol, maxit,
                                    ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def pd1_launches(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pd1_launches(plan, ctypes.byref(v))
    return st, v.value


def pd1_workspace(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pd1_workspace(plan, ctypes.byref(v))
    return st, v.value


def pd1_last_error(plan) -> str:
    return load().pd1_last_error(plan).decode()


def pdh_plan_create(space: pd_space, nt, dt, precision, stream):
    out = _P()
    st = load().pdh_plan_create(ctypes.byref(space), nt, dt, precision, _P(stream),
                                ctypes.byref(out))
    return st, out.value


def pdh_wave_plan_create(space: pd_space, nt, dt, precision, stream):
    out = _P()
    st = load().pdh_wave_plan_create(ctypes.byref(space), nt, dt, precision, _P(stream),
                                     ctypes.byref(out))
    return st, out.value


def pdh_wave_build_rhs(plan, u0, v0, f, b):
    return load().pdh_wave_build_rhs(plan, u0, v0, f, b)


def pdh_plan_destroy(plan):
    return load().pdh_plan_destroy(plan)


def pdh_eigenvalues(plan, nt):
    buf = (ctypes.c_double * (2 * nt))()
    st = load().pdh_eigenvalues(plan, buf)
    return st, [complex(buf[2 * i], buf[2 * i + 1]) for i in range(nt)]


def pdh_condition(plan):
    v = ctypes.c_double(0.0)
    st = load().pdh_condition(plan, ctypes.byref(v))
    return st, v.value


def pdh_apply_A(plan, u, y):
    return load().pdh_apply_A(plan, u, y)


def pdh_build_rhs(plan, u0, f, b):
    return load().pdh_build_rhs(plan, u0, f, b)


def pdh_solve(plan, b, u, tol, max_refine):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().pdh_solve(plan, b, u, tol, max_refine, ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def pdh_profile_sweep(plan, b, u, reps):
    ms = (ctypes.c_float * 4)()
    st = load().pdh_profile_sweep(plan, b, u, reps, ms)
    return st, list(ms)


def pdh_launches(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pdh_launches(plan, ctypes.byref(v))
    return st, v.value


def pdh_last_error(plan) -> str:
    return load().pdh_last_error(plan).decode()


def pdh_set_tensor_cores(plan, on):
    return load().pdh_set_tensor_cores(plan, int(on))


def pdh_tensor_cores(plan):
    v = ctypes.c_int(0)
    st = load().pdh_tensor_cores(plan, ctypes.byref(v))
    return st, v.value


def pdc_plan_create(space: pd_space, nt, T, gamma, precision, stream):
    out = _P()
    st = load().pdc_plan_create(ctypes.byref(space), nt, T, gamma, precision, _P(stream),
                                ctypes.byref(out))
    return st, out.value


def pdc_plan_destroy(plan):
    return load().pdc_plan_destroy(plan)


def pdc_apply_A(plan, x, y):
    return load().pdc_apply_A(plan, x, y)


def pdc_apply_precond(plan, r, z):
    return load().pdc_apply_precond(plan, r, z)


def pdc_solve(plan, b, x, tol, maxit, restart, left=False):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    fn = load().pdc_solve_left if left else load().pdc_solve
    st = fn(plan, b, x, tol, maxit, restart, ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def pdc_solve_left(plan, b, x, tol, maxit, restart):
    return pdc_solve(plan, b, x, tol, maxit, restart, left=True)


def pdc_launches(plan):
    v = ctypes.c_ulonglong(0)
    st = load().pdc_launches(plan, ctypes.byref(v))
    return st, v.value


def pdc_last_error(plan) -> str:
    return load().pdc_last_error(plan).decode()


def _space_of(space) -> pd_space:
    """pd_space from a mapping or an object with the pd_space fields."""
    g = (lambda k, d=0: space.get(k, d)) if isinstance(space, dict) else \
        (lambda k, d=0: getattr(space, k, d))
    return pd_space(int(g("dim", 1)), int(g("nx")), int(g("ny", 1) or 1),
                    float(g("nu", 1.0)), float(g("ax", 0.0)), float(g("ay", 0.0)),
                    int(g("bc_x", 0)), int(g("bc_y", 0)), float(g("lx", 1.0)),
                    float(g("ly", 1.0)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Plan:
    """A ParaDiag-II plan on the current CUDA device and stream.

    ``space`` is a mapping or object with the pd_space fields (dim, nx, ny, nu,
    ax, ay, bc_x, bc_y, lx, ly).  Tensors passed to the methods are CUDA float64
    tensors of shape (nt, S) (or anything with nt*S contiguous elements).
    """

    def __init__(self, space, nt, dt, alpha, scheme=PD_BE, theta=1.0, precision=PD_MIXED,
                 stream=None):
        import torch
        self.space = _space_of(space)
        self.nt, self.dt, self.alpha = int(nt), float(dt), float(alpha)
        self.scheme, self.theta, self.precision = int(scheme), float(theta), int(precision)
        self.S = self.space.nx * (self.space.ny if self.space.dim == 2 else 1)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, h = pd_plan_create(self.space, self.nt, self.dt, self.alpha, self.scheme, self.theta,
                               self.precision, self.stream.cuda_stream)
        if st != PD_OK:
            raise PDError(st, "pd_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            pd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != PD_OK:
            raise PDError(st, f"{what}: {pd_last_error(self._h)}")

    def _check_t(self, t, n=None):
        import torch
        n = self.nt * self.S if n is None else n
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"expected a contiguous CUDA float64 tensor with {n} elements")

    def workspace_bytes(self):
        st, v = pd_plan_workspace(self._h)
        self._check(st, "pd_plan_workspace")
        return v

    def launches(self):
        st, v = pd_plan_launches(self._h)
        self._check(st, "pd_plan_launches")
        return v

    def tuning(self):
        """(spatial columns per time-kernel block, lanes per tridiagonal system)"""
        st, tx, lanes = pd_plan_tuning(self._h)
        self._check(st, "pd_plan_tuning")
        return tx, lanes

    def get_tuning(self):
        """(spatial columns per time-kernel block, lanes per tridiagonal system,
        rows per lane the tridiagonal solver holds in registers)"""
        st, tx, lanes, rows = pd_plan_get_tuning(self._h)
        self._check(st, "pd_plan_get_tuning")
        return tx, lanes, rows

    def set_tuning(self, tile_columns, tri_lanes, tri_rows):
        """Pin the kernel shapes (see pd_plan_set_tuning)."""
        self._check(pd_plan_set_tuning(self._h, tile_columns, tri_lanes, tri_rows),
                    "pd_plan_set_tuning")

    @property
    def xform_engine(self):
        """PD_XFORM_TENSOR, PD_XFORM_FFT or PD_XFORM_DENSE (-1: no x-transform)."""
        st, v = pd_plan_xform_engine(self._h)
        self._check(st, "pd_plan_xform_engine")
        return v

    def set_xform_engine(self, engine):
        """Pin the engine of the x-eigentransform (see pd_plan_set_xform_engine)."""
        self._check(pd_plan_set_xform_engine(self._h, engine), "pd_plan_set_xform_engine")

    @property
    def time_cluster(self):
        """Blocks per time tile (1, or a cluster of 2, 4 or 8; see pd_plan_time_cluster)."""
        st, v = pd_plan_time_cluster(self._h)
        self._check(st, "pd_plan_time_cluster")
        return v

    def set_time_cluster(self, blocks):
        """Pin the blocks per time tile (see pd_plan_set_time_cluster)."""
        self._check(pd_plan_set_time_cluster(self._h, blocks), "pd_plan_set_time_cluster")

    def uses_graph(self):
        st, v = pd_plan_uses_graph(self._h)
        self._check(st, "pd_plan_uses_graph")
        return bool(v)

    def profile_iteration(self, b, u, reps=5):
        """Average ms per launch of [K1 residual+FFT, x-fwd, tridiagonal, x-inv, K3]."""
        self._check_t(b); self._check_t(u)
        st, ms = pd_profile_iteration(self._h, _ptr(b), _ptr(u), reps)
        self._check(st, "pd_profile_iteration")
        return ms

    def profile_precond(self, r, z, reps=5):
        """Average ms of [forward time kernel (standalone), x-fwd, tridiagonal,
        x-inv, inverse time kernel (FP64 output)] of pd_apply_precond."""
        self._check_t(r); self._check_t(z)
        st, ms = pd_profile_precond(self._h, _ptr(r), _ptr(z), reps)
        self._check(st, "pd_profile_precond")
        return ms

    def apply_precond(self, r, z=None):
        import torch
        self._check_t(r)
        z = torch.empty_like(r) if z is None else z
        self._check(pd_apply_precond(self._h, _ptr(r), _ptr(z)), "pd_apply_precond")
        return z

    def residual(self, b, u, r=None):
        import torch
        self._check_t(b); self._check_t(u)
        r = torch.empty_like(b) if r is None else r
        self._check(pd_residual(self._h, _ptr(b), _ptr(u), _ptr(r)), "pd_residual")
        return r

    def apply_A(self, u, y=None, transpose=False):
        import torch
        self._check_t(u)
        y = torch.empty_like(u) if y is None else y
        fn = pd_apply_AT if transpose else pd_apply_A
        self._check(fn(self._h, _ptr(u), _ptr(y)), "pd_apply_A")
        return y

    def build_rhs(self, u0, u1=None, f=None, b=None):
        import torch
        self._check_t(u0, self.S)
        if u1 is not None:
            self._check_t(u1, self.S)
        if f is not None:
            self._check_t(f, (self.nt + 1) * self.S)
        b = torch.empty((self.nt, self.S), dtype=torch.float64, device=u0.device) if b is None else b
        self._check(pd_build_rhs(self._h, _ptr(u0), _ptr(u1), _ptr(f), _ptr(b)), "pd_build_rhs")
        return b

    def solve(self, b, u=None, mode=PD_STATIONARY, tol=1e-10, maxit=50, restart=30,
              allow_not_converged=False):
        import torch
        self._check_t(b)
        u = torch.zeros_like(b) if u is None else u
        self._check_t(u)
        st, it, rel = pd_solve(self._h, _ptr(b), _ptr(u), mode, tol, maxit, restart)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pd_solve")
        return u, it, rel

    def solve_async(self, b, u, tol=1e-10, maxit=50):
        """Enqueue a stationary solve (no host wait on mixed plans); read the
        outcome with result()."""
        self._check_t(b); self._check_t(u)
        self._check(pd_solve_async(self._h, _ptr(b), _ptr(u), tol, maxit), "pd_solve_async")

    def result(self, allow_not_converged=False):
        """(iterations, relative residual) of the last asynchronous solve."""
        st, it, rel = pd_solve_result(self._h)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pd_solve_result")
        return it, rel

    def solve_host(self, b_host, u_host, mode=PD_STATIONARY, tol=1e-10, maxit=50, restart=30):
        st, it, rel = pd_solve_host(self._h, _ptr(b_host), _ptr(u_host), mode, tol, maxit, restart)
        if st != PD_OK:
            self._check(st, "pd_solve_host")
        return u_host, it, rel

    def solve_windows(self, u0, nwin, f=None, u=None, mode=PD_STATIONARY, tol=1e-10, maxit=50,
                      restart=30):
        """nwin consecutive windows of the plan's nt steps (window w starts from
        the last level of window w-1); returns (u [nwin, nt, S], total iterations,
        largest relative residual)."""
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (nwin * self.nt + 1) * self.S)
        u = torch.empty((nwin, self.nt, self.S), dtype=torch.float64, device=u0.device) \
            if u is None else u
        self._check_t(u, nwin * self.nt * self.S)
        st, it, rel = pd_solve_windows(self._h, _ptr(u0), _ptr(f), nwin, _ptr(u), mode, tol,
                                       maxit, restart)
        self._check(st, "pd_solve_windows")
        return u, it, rel

    # nonlinear problems U' + K U + phi(U) = f, phi(u) = a1 u + a2 u^2 + a3 u^3
    def nl_build_rhs(self, a, u0, f=None, b=None):
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (self.nt + 1) * self.S)
        b = torch.empty((self.nt, self.S), dtype=torch.float64, device=u0.device) if b is None else b
        self._check(pd_nl_build_rhs(self._h, a, _ptr(u0), _ptr(f), _ptr(b)), "pd_nl_build_rhs")
        return b

    def nl_residual(self, a, b, u, r=None):
        """(r, sigma = mean phi'(u), ||r||^2)"""
        import torch
        self._check_t(b); self._check_t(u)
        r = torch.empty_like(b) if r is None else r
        st, sig, rn2 = pd_nl_residual(self._h, a, _ptr(b), _ptr(u), _ptr(r))
        self._check(st, "pd_nl_residual")
        return r, sig, rn2

    def nl_solve(self, a, b, u=None, tol=1e-10, maxit=100, allow_not_converged=False):
        """Simplified Newton (eq. 1.5) from u (zeros if None); (u, corrections, relres)."""
        import torch
        self._check_t(b)
        u = torch.zeros_like(b) if u is None else u
        self._check_t(u)
        st, it, rel = pd_nl_solve(self._h, a, _ptr(b), _ptr(u), tol, maxit)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pd_nl_solve")
        return u, it, rel

    def nl_solve_windows(self, a, u0, nwin, f=None, u=None, tol=1e-10, maxit=100):
        """nwin nonlinear windows of the plan's nt steps (window w starts from the
        last level of window w-1); returns (u [nwin, nt, S], total corrections,
        largest relative residual)."""
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (nwin * self.nt + 1) * self.S)
        u = torch.empty((nwin, self.nt, self.S), dtype=torch.float64, device=u0.device) \
            if u is None else u
        self._check_t(u, nwin * self.nt * self.S)
        st, it, rel = pd_nl_solve_windows(self._h, a, _ptr(u0), _ptr(f), nwin, _ptr(u), tol, maxit)
        self._check(st, "pd_nl_solve_windows")
        return u, it, rel

    def adjoint_solve(self, g, lam=None, mode=PD_STATIONARY, tol=1e-10, maxit=50, restart=30):
        import torch
        self._check_t(g)
        lam = torch.zeros_like(g) if lam is None else lam
        st, it, rel = pd_adjoint_solve(self._h, _ptr(g), _ptr(lam), mode, tol, maxit, restart)
        self._check(st, "pd_adjoint_solve")
        return lam, it, rel


class Plan1:
    """A ParaDiag-I plan (geometric time steps, Section 2.1.1) on the current
    CUDA device and stream: the direct all-at-once solver of eq. 2.7 for one
    window of ``nt`` theta-method steps dt_n = dt_last tau^(n - nt).

    ``space`` as for Plan; tensors are CUDA float64 of shape (nt, S).
    """

    def __init__(self, space, nt, dt_last, tau, scheme=PD_BE, column_scaling=True,
                 precision=PD_FP64, stream=None):
        import torch
        self.space = _space_of(space)
        self.nt, self.dt_last, self.tau = int(nt), float(dt_last), float(tau)
        self.scheme, self.precision = int(scheme), int(precision)
        self.column_scaling = bool(column_scaling)
        self.S = self.space.nx * (self.space.ny if self.space.dim == 2 else 1)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, h = pd1_plan_create(self.space, self.nt, self.dt_last, self.tau, self.scheme,
                                int(self.column_scaling), self.precision, self.stream.cuda_stream)
        if st != PD_OK:
            raise PDError(st, "pd1_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            pd1_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != PD_OK:
            raise PDError(st, f"{what}: {pd1_last_error(self._h)}")

    def _check_t(self, t, n=None):
        import torch
        n = self.nt * self.S if n is None else n
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"expected a contiguous CUDA float64 tensor with {n} elements")

    def step_sizes(self):
        st, v = pd1_step_sizes(self._h, self.nt)
        self._check(st, "pd1_step_sizes")
        return v

    def condition(self):
        st, v = pd1_condition(self._h)
        self._check(st, "pd1_condition")
        return v

    def launches(self):
        st, v = pd1_launches(self._h)
        self._check(st, "pd1_launches")
        return v

    def workspace_bytes(self):
        st, v = pd1_workspace(self._h)
        self._check(st, "pd1_workspace")
        return v

    def apply_A(self, u, y=None):
        import torch
        self._check_t(u)
        y = torch.empty_like(u) if y is None else y
        self._check(pd1_apply_A(self._h, _ptr(u), _ptr(y)), "pd1_apply_A")
        return y

    def build_rhs(self, u0, f=None, b=None):
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (self.nt + 1) * self.S)
        b = torch.empty((self.nt, self.S), dtype=torch.float64, device=u0.device) if b is None else b
        self._check(pd1_build_rhs(self._h, _ptr(u0), _ptr(f), _ptr(b)), "pd1_build_rhs")
        return b

    def solve_windows(self, u0, nwin, f=None, u=None, tol=0.0, max_refine=0):
        """nwin consecutive windows (window w starts from the last level of
        window w-1); returns (u [nwin, nt, S], total sweeps, largest relres)."""
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (nwin * self.nt + 1) * self.S)
        u = torch.empty((nwin, self.nt, self.S), dtype=torch.float64, device=u0.device) \
            if u is None else u
        self._check_t(u, nwin * self.nt * self.S)
        st, it, rel = pd1_solve_windows(self._h, _ptr(u0), _ptr(f), nwin, _ptr(u), tol, max_refine)
        self._check(st, "pd1_solve_windows")
        return u, it, rel

    def profile_sweep(self, b, u, reps=5):
        """Average ms of [step (a) + residual, step (b), step (c) + update]."""
        self._check_t(b); self._check_t(u)
        st, ms = pd1_profile_sweep(self._h, _ptr(b), _ptr(u), reps)
        self._check(st, "pd1_profile_sweep")
        return ms

    def solve(self, b, u=None, tol=0.0, max_refine=0, allow_not_converged=False):
        """u = A^{-1} b; returns (u, refinement sweeps, relative residual)."""
        import torch
        self._check_t(b)
        u = torch.empty_like(b) if u is None else u
        self._check_t(u)
        st, it, rel = pd1_solve(self._h, _ptr(b), _ptr(u), tol, max_refine)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pd1_solve")
        return u, it, rel


class PlanHybrid:
    """A plan for ParaDiag-I with the hybrid midpoint + backward-Euler time
    discretisation (Section 2.1.2) on the current CUDA device and stream: nt
    uniform steps of size dt.  ``space`` as for Plan; tensors are CUDA float64
    of shape (nt, S)."""

    def __init__(self, space, nt, dt, precision=PD_FP64, stream=None, order=1):
        """order 1: U' + K U = f; order 2: U'' + K U = f (B_2nd = B^2)."""
        import torch
        self.space = _space_of(space)
        self.nt, self.dt, self.precision = int(nt), float(dt), int(precision)
        self.order = int(order)
        self.S = self.space.nx * (self.space.ny if self.space.dim == 2 else 1)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        create = pdh_wave_plan_create if self.order == 2 else pdh_plan_create
        st, h = create(self.space, self.nt, self.dt, self.precision, self.stream.cuda_stream)
        if st != PD_OK:
            raise PDError(st, "pdh_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            pdh_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != PD_OK:
            raise PDError(st, f"{what}: {pdh_last_error(self._h)}")

    def _check_t(self, t, n=None):
        import torch
        n = self.nt * self.S if n is None else n
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"expected a contiguous CUDA float64 tensor with {n} elements")

    def eigenvalues(self):
        st, v = pdh_eigenvalues(self._h, self.nt)
        self._check(st, "pdh_eigenvalues")
        return v

    def condition(self):
        st, v = pdh_condition(self._h)
        self._check(st, "pdh_condition")
        return v

    def launches(self):
        st, v = pdh_launches(self._h)
        self._check(st, "pdh_launches")
        return v

    @property
    def tensor_cores(self):
        """True when steps (a) and (c) run as tcgen05 GEMMs."""
        st, v = pdh_tensor_cores(self._h)
        self._check(st, "pdh_tensor_cores")
        return bool(v)

    def set_tensor_cores(self, on):
        """Pick the engine of the time contractions (raises on plans without
        the tensor-core form)."""
        self._check(pdh_set_tensor_cores(self._h, on), "pdh_set_tensor_cores")

    def apply_A(self, u, y=None):
        import torch
        self._check_t(u)
        y = torch.empty_like(u) if y is None else y
        self._check(pdh_apply_A(self._h, _ptr(u), _ptr(y)), "pdh_apply_A")
        return y

    def build_rhs(self, u0, f=None, b=None):
        import torch
        self._check_t(u0, self.S)
        if f is not None:
            self._check_t(f, (self.nt + 1) * self.S)
        b = torch.empty((self.nt, self.S), dtype=torch.float64, device=u0.device) if b is None else b
        self._check(pdh_build_rhs(self._h, _ptr(u0), _ptr(f), _ptr(b)), "pdh_build_rhs")
        return b

    def build_rhs_wave(self, u0, v0, f=None, b=None):
        """Second-order plans: b = F_v + B F_u from u0, v0 and f ([nt+1, S])."""
        import torch
        self._check_t(u0, self.S)
        self._check_t(v0, self.S)
        if f is not None:
            self._check_t(f, (self.nt + 1) * self.S)
        b = torch.empty((self.nt, self.S), dtype=torch.float64, device=u0.device) if b is None else b
        self._check(pdh_wave_build_rhs(self._h, _ptr(u0), _ptr(v0), _ptr(f), _ptr(b)),
                    "pdh_wave_build_rhs")
        return b

    def profile_sweep(self, b, u, reps=5):
        """Average ms of [residual, step (a), step (b), step (c) + update]."""
        self._check_t(b); self._check_t(u)
        st, ms = pdh_profile_sweep(self._h, _ptr(b), _ptr(u), reps)
        self._check(st, "pdh_profile_sweep")
        return ms

    def solve(self, b, u=None, tol=0.0, max_refine=0, allow_not_converged=False):
        """u = A^{-1} b; returns (u, refinement sweeps, relative residual)."""
        import torch
        self._check_t(b)
        u = torch.empty_like(b) if u is None else u
        self._check_t(u)
        st, it, rel = pdh_solve(self._h, _ptr(b), _ptr(u), tol, max_refine)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pdh_solve")
        return u, it, rel


class PlanControl:
    """A plan for the optimal control of the wave equation (Section 4): the
    leap-frog saddle-point system in (u, p), FGMRES with the gamma-balanced
    block circulant preconditioner.  Tensors are CUDA float64 of shape
    (2, nt, S): the state field, then the adjoint field."""

    def __init__(self, space, nt, T, gamma, precision=PD_FP64, stream=None):
        import torch
        self.space = _space_of(space)
        self.nt, self.T, self.gamma, self.precision = int(nt), float(T), float(gamma), int(precision)
        self.S = self.space.nx * (self.space.ny if self.space.dim == 2 else 1)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, h = pdc_plan_create(self.space, self.nt, self.T, self.gamma, self.precision,
                                self.stream.cuda_stream)
        if st != PD_OK:
            raise PDError(st, "pdc_plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            pdc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != PD_OK:
            raise PDError(st, f"{what}: {pdc_last_error(self._h)}")

    def _check_t(self, t):
        import torch
        n = 2 * self.nt * self.S
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"expected a contiguous CUDA float64 tensor with {n} elements")

    def launches(self):
        st, v = pdc_launches(self._h)
        self._check(st, "pdc_launches")
        return v

    def apply_A(self, x, y=None):
        import torch
        self._check_t(x)
        y = torch.empty_like(x) if y is None else y
        self._check(pdc_apply_A(self._h, _ptr(x), _ptr(y)), "pdc_apply_A")
        return y

    def profile_precond(self, r, z, reps=5):
        """Average ms of [forward time kernel (standalone), x-fwd, tridiagonal,
        x-inv, inverse time kernel (FP64 output)] of pd_apply_precond."""
        self._check_t(r); self._check_t(z)
        st, ms = pd_profile_precond(self._h, _ptr(r), _ptr(z), reps)
        self._check(st, "pd_profile_precond")
        return ms

    def apply_precond(self, r, z=None):
        import torch
        self._check_t(r)
        z = torch.empty_like(r) if z is None else z
        self._check(pdc_apply_precond(self._h, _ptr(r), _ptr(z)), "pdc_apply_precond")
        return z

    def solve(self, b, x=None, tol=1e-7, maxit=100, restart=30, allow_not_converged=False,
              left=False):
        """(u, p) for the right-hand side (f, g); returns (x, iterations, relres).
        left=True: left preconditioning, relres on the preconditioned residual."""
        import torch
        self._check_t(b)
        x = torch.empty_like(b) if x is None else x
        self._check_t(x)
        st, it, rel = pdc_solve(self._h, _ptr(b), _ptr(x), tol, maxit, restart, left)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            self._check(st, "pdc_solve")
        return x, it, rel


class Batch:
    """Many independent 1D problems solved together (packed FP64 arrays).

    ``problems``: list of dicts with keys space (pd_space fields), nt, dt, alpha,
    scheme, theta.  Problem i occupies ``offsets[i]:offsets[i+1]`` of the packed
    arrays ([nt_i][nx_i] each)."""

    def __init__(self, problems, precision=PD_MIXED, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        items = []
        for q in problems:
            sp = q["space"]
            items.append(pd_problem(pd_space(1, int(sp["nx"]), 1, float(sp.get("nu", 1.0)),
                                             float(sp.get("ax", 0.0)), 0.0, PD_DIRICHLET,
                                             PD_DIRICHLET, float(sp.get("lx", 1.0)), 1.0),
                                    int(q["nt"]), float(q["dt"]), float(q["alpha"]),
                                    int(q.get("scheme", PD_BE)), float(q.get("theta", 1.0))))
        st, h = pd_batch_create(items, precision, self.stream.cuda_stream)
        if st != PD_OK:
            raise PDError(st, "pd_batch_create")
        self._h = h
        self.np = len(items)
        st, self.offsets = pd_batch_offsets(h, self.np)
        self.total = self.offsets[-1]

    def close(self):
        if getattr(self, "_h", None):
            pd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launches(self):
        return pd_batch_launches(self._h)[1]

    def uses_graph(self):
        st, v = pd_batch_uses_graph(self._h)
        if st != PD_OK:
            raise PDError(st, "pd_batch_uses_graph")
        return bool(v)

    def build_rhs(self, u0, f=None):
        import torch
        b = torch.empty(self.total, dtype=torch.float64, device=u0.device)
        st = pd_batch_build_rhs(self._h, _ptr(u0), _ptr(f), _ptr(b))
        if st != PD_OK:
            raise PDError(st, pd_batch_last_error(self._h))
        return b

    def solve(self, b, u=None, tol=1e-10, maxit=50, allow_not_converged=False):
        import torch
        u = torch.zeros_like(b) if u is None else u
        st, it, rel = pd_batch_solve(self._h, _ptr(b), _ptr(u), tol, maxit)
        if not (st == PD_OK or (allow_not_converged and st == PD_ERR_NOT_CONVERGED)):
            raise PDError(st, pd_batch_last_error(self._h))
        return u, it, rel

    def relres(self):
        """Relative residual of every problem at the last check of solve()."""
        return pd_batch_relres(self._h, self.np)[1]

    def tuned(self):
        """True when the kernel shapes were chosen by timing at creation."""
        st, v = pd_batch_tuned(self._h)
        if st != PD_OK:
            raise PDError(st, "pd_batch_tuned")
        return bool(v)

    def profile_sweep(self, b, u, reps=5):
        """[forward time kernels, tridiagonal solves, inverse time kernels] in ms
        per sweep (u is overwritten)."""
        st, ms = pd_batch_profile_sweep(self._h, _ptr(b), _ptr(u), reps)
        if st != PD_OK:
            raise PDError(st, pd_batch_last_error(self._h))
        return ms


def _make_pdsolve():
    import torch

    class PDSolve(torch.autograd.Function):
        """u = A^{-1} b with the ParaDiag-II solver; backward: dL/db = A^{-T} dL/du.

        forward(plan, b, mode, tol, maxit) -> u.  The backward pass solves the
        transposed all-at-once system (backward in time) with the same plan's
        kernels (pd_adjoint_solve).
        """

        @staticmethod
        def forward(ctx, plan, b, mode=PD_STATIONARY, tol=1e-10, maxit=50):
            ctx.plan, ctx.mode, ctx.tol, ctx.maxit = plan, mode, tol, maxit
            u, _, _ = plan.solve(b.detach().contiguous(), mode=mode, tol=tol, maxit=maxit)
            return u

        @staticmethod
        def backward(ctx, g):
            lam, _, _ = ctx.plan.adjoint_solve(g.contiguous(), mode=ctx.mode, tol=ctx.tol,
                                              maxit=ctx.maxit)
            return None, lam, None, None, None

    return PDSolve


class _Lazy:
    _cls = None

    def __getattr__(self, k):
        if _Lazy._cls is None:
            _Lazy._cls = _make_pdsolve()
        return getattr(_Lazy._cls, k)


PDSolve = _Lazy()

__all__ = ["build", "lib_path", "load", "Plan", "Plan1", "PlanHybrid", "PlanControl", "Batch", "PDSolve", "PDError", "pd_space",
           "pd_problem",
           "exported_symbols"] + [k for k in _SIGS]
