"""ctypes binding of libdgw.so (include/dgw.h), with the same names.

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built -- there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgw.so")
# the build with device-side checks (DGW_DEBUG_CHECKS); loaded when the
# environment variable DGW_DEBUG_CHECKS is 1
LIB_DEBUG_PATH = os.path.join(HERE, "libdgw_debug.so")

DGW_OK = 0
STATUS = {0: "DGW_OK", -1: "DGW_ERR_ARG", -2: "DGW_ERR_STATE", -3: "DGW_ERR_OOM", -4: "DGW_ERR_CUDA",
          -5: "DGW_ERR_UNSTABLE", -6: "DGW_ERR_TIMEOUT", -7: "DGW_ERR_UNSUPPORTED"}
DGW_PRECISION_FP64 = 0
DGW_PRECISION_MIXED = 1
DGW_PRECISION_MIXED_TC_FP16 = 2
DGW_PRECISION_MIXED_TC_BF16 = 3
DGW_BC_INTERIOR, DGW_BC_FREE_SURFACE, DGW_BC_ABSORBING = 0, 1, 2
DGW_BATCH_MAX_SOLVES = 128
DGW_SYSTEM_ELASTIC, DGW_SYSTEM_TRANSPORT, DGW_SYSTEM_SHALLOW_WATER = 0, 1, 2
DGW_BC_WALL = 1


class dgw_config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("flux_tau", ctypes.c_int), ("precision", ctypes.c_int),
                ("cfl", ctypes.c_double), ("system", ctypes.c_int), ("beta", ctypes.c_double * 3)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64

# name -> (restype, argtypes); exactly the functions declared in include/dgw.h
SIGNATURES = {
    "dgw_abi_version": (_I, []),
    "dgw_reference_nodes": (_I, [_I, _P, _P]),
    "dgw_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(dgw_config)]),
    "dgw_destroy": (_I, [_P]),
    "dgw_mesh_upload": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "dgw_material_upload": (_I, [_P, _P, _P, _P]),
    "dgw_rhs": (_I, [_P, _P, _P, _D, _P]),
    "dgw_stage": (_I, [_P, _P, _P, _P, _I, _D, _D, _P]),
    "dgw_stage_energy": (_I, [_P, _P, _P, _P, _I, _D, _D, ctypes.POINTER(_D), _P]),
    "dgw_step": (_I, [_P, _P, _P, _D, _D, _I, _P]),
    "dgw_step_energy": (_I, [_P, _P, _P, _D, _D, _I, ctypes.POINTER(_D), _P]),
    "dgw_energy": (_I, [_P, _P, ctypes.POINTER(_D), _P]),
    "dgw_source_set": (_I, [_P, _I64, _P, _P, _D, _D]),
    "dgw_receivers_set": (_I, [_P, _I, _P, _P]),
    "dgw_receivers_sample": (_I, [_P, _P, _P, _P]),
    "dgw_receivers_adjoint": (_I, [_P, _P, _P, _P]),
    "dgw_adjoint_step": (_I, [_P, _P, _P, _P, _P, _D, _D, _I, _P]),
    "dgw_adjoint_traces": (_I, [_P, _P, _P, _P, _P, _P, _D, _D, _I, _P]),
    "dgw_dt_cfl": (_I, [_P, ctypes.POINTER(_D)]),
    "dgw_batch_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I]),
    "dgw_batch_destroy": (_I, [_P]),
    "dgw_batch_set": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "dgw_batch_run": (_I, [_P, _I, _P]),
    "dgw_batch_last_error": (ctypes.c_char_p, [_P]),
    "dgw_energy_static": (_I, [_I, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "dgw_ihdg_setup": (_I, [_P, _D, _P]),
    "dgw_ihdg_solve": (_I, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "dgw_probe_fp64_rate": (_I, [_I, ctypes.POINTER(_D)]),
    "dgw_debug_status": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "dgw_state_bytes": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "dgw_get_state": (_I, [_P, _P, _P, _D, _I64, _P, ctypes.c_size_t, _P]),
    "dgw_set_state": (_I, [_P, _P, ctypes.c_size_t, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_I64), _P]),
    "dgw_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


class DGWError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str = None):
    """Load libdgw.so (built by ``paper_1711_01175_gb300.build.build()``), or
    libdgw_debug.so (``build(debug=True)``) when DGW_DEBUG_CHECKS=1."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_DEBUG_PATH if os.environ.get("DGW_DEBUG_CHECKS") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, ctx=None):
    if status != DGW_OK:
        msg = load().dgw_last_error(ctx).decode(errors="replace")
        raise DGWError(status, msg)
    return status


# Thin wrappers with the C names (pointers are ints; see solver.py for tensors).
def dgw_abi_version():
    return load().dgw_abi_version()


def dgw_reference_nodes(N, r_ptr, w_ptr):
    return load().dgw_reference_nodes(N, r_ptr, w_ptr)


def dgw_create(device, cfg):
    h = _P()
    st = load().dgw_create(ctypes.byref(h), device, ctypes.byref(cfg))
    return st, h


def dgw_destroy(ctx):
    return load().dgw_destroy(ctx)


def dgw_mesh_upload(ctx, nel, x, etoe, etof, orient, bc):
    return load().dgw_mesh_upload(ctx, nel, x, etoe, etof, orient, bc)


def dgw_material_upload(ctx, rho, lam, mu):
    return load().dgw_material_upload(ctx, rho, lam, mu)


def dgw_rhs(ctx, u, rhs, t, stream):
    return load().dgw_rhs(ctx, u, rhs, t, stream)


def dgw_stage(ctx, u_in, u_out, res, stage, t, dt, stream):
    return load().dgw_stage(ctx, u_in, u_out, res, stage, t, dt, stream)


def dgw_stage_energy(ctx, u_in, u_out, res, stage, t, dt, stream):
    out = _D()
    st = load().dgw_stage_energy(ctx, u_in, u_out, res, stage, t, dt, ctypes.byref(out), stream)
    return st, out.value


def dgw_step(ctx, u, res, t0, dt, nsteps, stream):
    return load().dgw_step(ctx, u, res, t0, dt, nsteps, stream)


def dgw_step_energy(ctx, u, res, t0, dt, nsteps, stream):
    out = _D()
    st = load().dgw_step_energy(ctx, u, res, t0, dt, nsteps, ctypes.byref(out), stream)
    return st, out.value


def dgw_energy(ctx, u, stream):
    out = _D()
    st = load().dgw_energy(ctx, u, ctypes.byref(out), stream)
    return st, out.value


def dgw_source_set(ctx, element, xi, force, f0, t0):
    return load().dgw_source_set(ctx, element, xi, force, f0, t0)


def dgw_receivers_set(ctx, n, elements, xi):
    return load().dgw_receivers_set(ctx, n, elements, xi)


def dgw_receivers_sample(ctx, u, out, stream):
    return load().dgw_receivers_sample(ctx, u, out, stream)


def dgw_receivers_adjoint(ctx, lam_u, g, stream):
    return load().dgw_receivers_adjoint(ctx, lam_u, g, stream)


def dgw_adjoint_step(ctx, lam_u, lam_res, grad_mat, u_ckpt, t0, dt, nsteps, stream):
    return load().dgw_adjoint_step(ctx, lam_u, lam_res, grad_mat, u_ckpt, t0, dt, nsteps, stream)


def dgw_adjoint_traces(ctx, lam_u, lam_res, grad_mat, u_ckpt, g_traces, t0, dt, nsteps, stream):
    return load().dgw_adjoint_traces(ctx, lam_u, lam_res, grad_mat, u_ckpt, g_traces, t0, dt, nsteps, stream)


def dgw_probe_fp64_rate(device):
    out = _D()
    st = load().dgw_probe_fp64_rate(device, ctypes.byref(out))
    return st, out.value


def dgw_state_bytes(ctx, with_res):
    out = ctypes.c_size_t()
    st = load().dgw_state_bytes(ctx, int(with_res), ctypes.byref(out))
    return st, out.value


def dgw_get_state(ctx, u, res, t, step, buf, buf_bytes, stream):
    return load().dgw_get_state(ctx, u, res, t, step, buf, buf_bytes, stream)


def dgw_set_state(ctx, buf, buf_bytes, u, res, stream):
    t, step = _D(), _I64()
    st = load().dgw_set_state(ctx, buf, buf_bytes, u, res, ctypes.byref(t), ctypes.byref(step), stream)
    return st, t.value, step.value


def dgw_debug_status(ctx):
    code, el, cnt = _I(), _I64(), _I64()
    st = load().dgw_debug_status(ctx, ctypes.byref(code), ctypes.byref(el), ctypes.byref(cnt))
    return st, code.value, el.value, cnt.value


def dgw_dt_cfl(ctx):
    out = _D()
    st = load().dgw_dt_cfl(ctx, ctypes.byref(out))
    return st, out.value


def dgw_batch_create(device, N, precision, flux_tau, max_solves=DGW_BATCH_MAX_SOLVES):
    h = _P()
    st = load().dgw_batch_create(ctypes.byref(h), device, N, precision, flux_tau, max_solves)
    return st, h


def dgw_batch_destroy(b):
    return load().dgw_batch_destroy(b)


def dgw_batch_set(b, n, ctxs, u, res, dt, t0, stream):
    return load().dgw_batch_set(b, n, ctxs, u, res, dt, t0, stream)


def dgw_batch_run(b, npairs, stream):
    return load().dgw_batch_run(b, npairs, stream)


def dgw_batch_last_error(b):
    return load().dgw_batch_last_error(b).decode(errors="replace")


def dgw_energy_static(N, nel, x, u, rho, lam, mu, energy_out, stream):
    return load().dgw_energy_static(N, nel, x, u, rho, lam, mu, energy_out, stream)


def dgw_ihdg_setup(ctx, sigma, stream):
    return load().dgw_ihdg_setup(ctx, sigma, stream)


def dgw_ihdg_solve(ctx, u_prev, f, u, tol, max_iter, stream):
    its = _I()
    change = _D()
    st = load().dgw_ihdg_solve(ctx, u_prev, f, u, tol, max_iter, ctypes.byref(its), ctypes.byref(change), stream)
    return st, its.value, change.value


def dgw_last_error(ctx):
    return load().dgw_last_error(ctx).decode(errors="replace")
