"""Tensor-level front end over the C ABI: one ``Solver`` per mesh and medium.

Field tensors are ``[m, nel, Np]`` float64 (m = 9 for elasticity, 1 for
transport, 3 for shallow water), either CUDA tensors (device
pointers; the work is enqueued on torch's current stream) or CPU tensors /
numpy arrays (host pointers; the library stages them through its own device
buffers).  PyTorch only provides device memory and streams here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi


def _stream_handle(stream=None):
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a):
    """Raw pointer of a contiguous torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(a.data_ptr())


def reference_nodes(N: int):
    """GLL nodes and weights the library uses (numpy float64, length N+1)."""
    r = np.zeros(N + 1)
    w = np.zeros(N + 1)
    capi.check(capi.dgw_reference_nodes(N, _ptr(r), _ptr(w)))
    return r, w


# precision names -> dgw_config.precision: "mixed" FP32 volume/flux/lift on CUDA
# cores; "mixed_tc" (FP16) and "mixed_tc_bf16" the same with the volume term's
# derivative contractions on the tensor cores (split 16-bit operands).
PRECISIONS = {"fp64": capi.DGW_PRECISION_FP64, "mixed": capi.DGW_PRECISION_MIXED,
              "mixed_tc": capi.DGW_PRECISION_MIXED_TC_FP16, "mixed_tc_bf16": capi.DGW_PRECISION_MIXED_TC_BF16}

SYSTEMS = {"elastic": (capi.DGW_SYSTEM_ELASTIC, 9), "transport": (capi.DGW_SYSTEM_TRANSPORT, 1),
           "shallow_water": (capi.DGW_SYSTEM_SHALLOW_WATER, 3)}


class Solver:
    """A DG operator on one mesh (and, for elasticity, one medium); owns a dgw_ctx.

    system: "elastic" (default), "transport" (velocity ``beta``) or
    "shallow_water" (Phi = 1); the last two take no medium and run in FP64."""

    def __init__(self, N: int, tau: int = 1, precision: str = "fp64", cfl: float = 0.5, device: int = 0,
                 system: str = "elastic", beta=(0.0, 0.0, 0.0)):
        prec = PRECISIONS[precision]
        sys_id, self.m = SYSTEMS[system]
        self.system = system
        self.N, self.tau, self.precision = int(N), int(tau), precision
        self.Np = (self.N + 1) ** 3
        cfg = capi.dgw_config(self.N, self.tau, prec, float(cfl), sys_id, (ctypes.c_double * 3)(*[float(b) for b in beta]))
        st, h = capi.dgw_create(int(device), cfg)
        capi.check(st)
        self._ctx = h
        self.nel = 0
        self._source = None

    def close(self):
        if getattr(self, "_ctx", None):
            capi.dgw_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        return capi.check(st, self._ctx)

    def upload_mesh(self, x, etoe, etof, orient, bc):
        x = np.ascontiguousarray(x, dtype=np.float64)
        nel = x.shape[0]
        if x.shape != (nel, self.Np, 3):
            raise ValueError(f"x must be [nel, {self.Np}, 3]")
        arrs = [np.ascontiguousarray(etoe, dtype=np.int64), np.ascontiguousarray(etof, dtype=np.int8),
                np.ascontiguousarray(orient, dtype=np.int8), np.ascontiguousarray(bc, dtype=np.int8)]
        for a in arrs:
            if a.shape != (nel, 6):
                raise ValueError("connectivity arrays must be [nel, 6]")
        self._check(capi.dgw_mesh_upload(self._ctx, nel, _ptr(x), *[_ptr(a) for a in arrs]))
        self.nel = nel

    def upload_material(self, rho, lam, mu):
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho, lam, mu)]
        for a in arrs:
            if a.shape != (self.nel,):
                raise ValueError("material arrays must be [nel]")
        self._check(capi.dgw_material_upload(self._ctx, *[_ptr(a) for a in arrs]))
        if self._source is not None:          # the point force depends on rho: set it again
            self.set_point_force(**self._source)

    def _field_check(self, a, name):
        if self.nel == 0:
            return          # no mesh yet: the C ABI reports the call-order error
        shape = tuple(a.shape)
        if shape != (self.m, self.nel, self.Np):
            raise ValueError(f"{name} must be [{self.m}, {self.nel}, {self.Np}], got {shape}")
        if str(a.dtype) not in ("float64", "torch.float64"):
            raise ValueError(f"{name} must be float64")

    def set_point_force(self, element: int, xi, force, f0: float, t0: float):
        """Ricker point force in `element` at reference point xi (element -1 clears)."""
        xi_a = np.ascontiguousarray(xi, dtype=np.float64)
        force_a = np.ascontiguousarray(force, dtype=np.float64)
        self._check(capi.dgw_source_set(self._ctx, int(element), _ptr(xi_a), _ptr(force_a), float(f0), float(t0)))
        self._source = None if int(element) < 0 else dict(element=int(element), xi=list(xi_a), force=list(force_a),
                                                             f0=float(f0), t0=float(t0))

    def rhs(self, u, out, t: float = 0.0, stream=None):
        self._field_check(u, "u")
        self._field_check(out, "out")
        self._check(capi.dgw_rhs(self._ctx, _ptr(u), _ptr(out), float(t), _stream_handle(stream)))
        return out

    def stage(self, u_in, u_out, res, s: int, dt: float, t: float = 0.0, stream=None):
        for a, nm in ((u_in, "u_in"), (u_out, "u_out"), (res, "res")):
            self._field_check(a, nm)
        self._check(capi.dgw_stage(self._ctx, _ptr(u_in), _ptr(u_out), _ptr(res), int(s), float(t),
                                   float(dt), _stream_handle(stream)))

    def stage_energy(self, u_in, u_out, res, s: int, dt: float, t: float = 0.0, stream=None) -> float:
        """dgw_stage plus the energy of u_out, fused into the same kernel."""
        for a, nm in ((u_in, "u_in"), (u_out, "u_out"), (res, "res")):
            self._field_check(a, nm)
        st, val = capi.dgw_stage_energy(self._ctx, _ptr(u_in), _ptr(u_out), _ptr(res), int(s), float(t),
                                        float(dt), _stream_handle(stream))
        self._check(st)
        return val

    def step(self, u, res, dt: float, nsteps: int = 1, t0: float = 0.0, stream=None):
        """nsteps LSRK(5,4) steps in place on u; res receives the last stage's
        register (None: the context keeps it)."""
        self._field_check(u, "u")
        if res is not None:
            self._field_check(res, "res")
        self._check(capi.dgw_step(self._ctx, _ptr(u), None if res is None else _ptr(res), float(t0), float(dt),
                                  int(nsteps), _stream_handle(stream)))

    def step_energy(self, u, res, dt: float, nsteps: int = 1, t0: float = 0.0, stream=None) -> float:
        """step, with the energy of the new state accumulated in its last stage."""
        self._field_check(u, "u")
        if res is not None:
            self._field_check(res, "res")
        st, val = capi.dgw_step_energy(self._ctx, _ptr(u), None if res is None else _ptr(res), float(t0),
                                       float(dt), int(nsteps), _stream_handle(stream))
        self._check(st)
        return val

    def energy(self, u, stream=None) -> float:
        self._field_check(u, "u")
        st, val = capi.dgw_energy(self._ctx, _ptr(u), _stream_handle(stream))
        self._check(st)
        return val

    def ihdg_setup(self, sigma: float, stream=None):
        """iHDG-II: build and invert sigma I - L_K^self per element (transport N <= 4,
        shallow water N <= 3, FP64 elastic N <= 3)."""
        self._check(capi.dgw_ihdg_setup(self._ctx, float(sigma), _stream_handle(stream)))

    def ihdg_solve(self, u, u_prev=None, f=None, tol: float = 1e-10, max_iter: int = 1000, stream=None):
        """Iterate iHDG-II from the guess in u (device [m, nel, Np], overwritten) for
        sigma u - L(u) = sigma u_prev + f; returns (iterations, last ||u^k - u^{k-1}||)."""
        self._field_check(u, "u")
        for a, name in ((u_prev, "u_prev"), (f, "f")):
            if a is not None:
                self._field_check(a, name)
        st, its, change = capi.dgw_ihdg_solve(self._ctx, None if u_prev is None else _ptr(u_prev),
                                              None if f is None else _ptr(f), _ptr(u), float(tol), int(max_iter),
                                              _stream_handle(stream))
        self._check(st)
        return its, change

    def set_receivers(self, elements, xi):
        el = np.ascontiguousarray(elements, dtype=np.int64)
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        self._check(capi.dgw_receivers_set(self._ctx, int(el.size), _ptr(el), _ptr(xi)))
        self.nrec = int(el.size)

    def sample_receivers(self, u, out, stream=None):
        """out [nrec, 3] (device) = receiver velocities of u (device)."""
        self._check(capi.dgw_receivers_sample(self._ctx, _ptr(u), _ptr(out), _stream_handle(stream)))
        return out

    def receivers_adjoint(self, lam_u, g, stream=None):
        self._check(capi.dgw_receivers_adjoint(self._ctx, _ptr(lam_u), _ptr(g), _stream_handle(stream)))

    def adjoint_step(self, lam_u, lam_res, grad, u_ckpt, dt: float, nsteps: int = 1, t0: float = 0.0, stream=None):
        """Adjoint of nsteps steps from u_ckpt at t0; grad [3, nel] is incremented."""
        self._check(capi.dgw_adjoint_step(self._ctx, _ptr(lam_u), _ptr(lam_res), _ptr(grad), _ptr(u_ckpt),
                                          float(t0), float(dt), int(nsteps), _stream_handle(stream)))

    def adjoint_traces(self, lam_u, lam_res, grad, u_ckpt, g_traces, dt: float, nsteps: int, t0: float = 0.0,
                       stream=None):
        """Adjoint of the nsteps steps from u_ckpt at t0 with receiver-trace sources
        g_traces [nsteps, nrec, 3] (device); grad [3, nel] is incremented."""
        self._check(capi.dgw_adjoint_traces(self._ctx, _ptr(lam_u), _ptr(lam_res), _ptr(grad), _ptr(u_ckpt),
                                            _ptr(g_traces), float(t0), float(dt), int(nsteps), _stream_handle(stream)))

    def get_state(self, u, res=None, t: float = 0.0, step: int = 0, stream=None):
        """Checkpoint of (u, res, t, step) as a host uint8 array (dgw_get_state)."""
        st, nbytes = capi.dgw_state_bytes(self._ctx, res is not None)
        self._check(st)
        buf = np.empty(nbytes, dtype=np.uint8)
        self._check(capi.dgw_get_state(self._ctx, _ptr(u), None if res is None else _ptr(res), float(t), int(step),
                                       _ptr(buf), nbytes, _stream_handle(stream)))
        return buf

    def set_state(self, buf, u, res=None, stream=None):
        """Load a checkpoint into u (and res); returns its (t, step) (dgw_set_state)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        st, t, step = capi.dgw_set_state(self._ctx, _ptr(buf), buf.nbytes, _ptr(u),
                                         None if res is None else _ptr(res), _stream_handle(stream))
        self._check(st)
        return t, step

    def dt_cfl(self) -> float:
        """dt = cfl h_min / (c_max N^2), the convention of the paper's transport
        experiments (Section 6.1).  For the elastic system the default cfl 0.5 is
        stable from N = 3 on; rough states need about 0.125 at N = 1 and 0.45 at
        N = 2 (pass cfl= to the constructor)."""
        st, val = capi.dgw_dt_cfl(self._ctx)
        self._check(st)
        return val
