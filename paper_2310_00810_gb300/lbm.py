"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (``liblbm.so``).

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors become device pointers, the current torch
CUDA stream becomes the ``cudaStream_t``.  All lattice work runs in the
library's CUDA kernels.  There is no CPU fallback: if the library has not
been built (``python -m paper_2310_00810_gb300.build``) loading fails loudly.

``Solver`` bundles one plan with the device buffers it needs (allocated by
torch) for the common single-instance use.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_UNSUPPORTED, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT = range(7)
LBM_LOSS_VEC, LBM_LOSS_NORM = 0, 1
LBM_NORM_SUM, LBM_NORM_MEAN_FLUID = 0, 1
LBM_INLET_CONST, LBM_INLET_PROFILE = 0, 1
LBM_GEOM_CHANNEL, LBM_GEOM_DISKS, LBM_GEOM_SPHERES, LBM_GEOM_MASK = 0, 1, 2, 3
LBM_LINK_SOLID = 0x80000000

LBM_FAMILY_AUTO, LBM_FAMILY_SCALAR, LBM_FAMILY_VEC, LBM_FAMILY_TMA = 0, 1, 2, 3
LBM_ABB_U_NODE, LBM_ABB_U_EXTRAP = 0, 1
LBM_COLLISION_BGK, LBM_COLLISION_MRT = 0, 1

ENTRY_POINTS = (
    "lbm_plan_create", "lbm_plan_destroy", "lbm_plan_set_kernels", "lbm_plan_get_kernels", "lbm_workspace_size", "lbm_init_geometry", "lbm_bind_geometry",
    "lbm_compact_size", "lbm_compact_bind", "lbm_set_abb_velocity", "lbm_get_abb_velocity",
    "lbm_set_collision", "lbm_get_collision", "lbm_set_periodic_y", "lbm_set_velocity_inlet",
    "lbm_set_velocity_ramp", "lbm_adjoint_window",
    "lbm_forward", "lbm_step", "lbm_loss_grad", "lbm_loss_grad_noalloc", "lbm_probe_loss_grad", "lbm_spline_basis",
    "lbm_spline_profile", "lbm_spline_grad", "lbm_adjoint", "lbm_macroscopic", "lbm_darcy", "lbm_adam_step",
    "lbm_get_status", "lbm_error_string", "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_layout",
    "lbm_batch_init_geometry", "lbm_batch_forward", "lbm_batch_loss_grad", "lbm_batch_adjoint",
    "lbm_batch_compact_size", "lbm_batch_compact_bind", "lbm_batch_get_status",
    "unet_param_layout", "unet_workspace_size", "unet_pack_input", "unet_prepare_weights", "unet_forward",
    "unet_backward", "unet_adam", "unet_set_engine", "unet_get_status",
)


class lbm_desc(C.Structure):
    _fields_ = [("q", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("precision", C.c_int32), ("n_steps", C.c_int32), ("ckpt_stride", C.c_int32),
                ("loss_kind", C.c_int32), ("loss_norm", C.c_int32), ("inlet_kind", C.c_int32)]


class lbm_kernel_choice(C.Structure):
    _fields_ = [("step_family", C.c_int32), ("adjoint_family", C.c_int32), ("vec", C.c_int32),
                ("tma_rows", C.c_int32), ("pdl", C.c_int32), ("persist", C.c_int32), ("overlap", C.c_int32),
                ("adjoint_tma_rows", C.c_int32), ("steps_per_launch", C.c_int32), ("recompute_family", C.c_int32),
                ("aa", C.c_int32)]


class lbm_geom_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("r_min", C.c_int32), ("r_max", C.c_int32), ("hydro_q8", C.c_int32),
                ("inlet_buffer", C.c_int32), ("fill_isolated", C.c_int32), ("max_rejections", C.c_int64),
                ("seed", C.c_uint64), ("target_porosity", C.c_double)]


_lock = threading.Lock()
_lib = None


class LBMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lbm_error_string(status)} (status {status})")


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblbm.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_2310_00810_gb300.build`")
            lib = C.CDLL(path)
            vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
            sig = {
                "lbm_plan_create": [C.POINTER(lbm_desc), C.POINTER(vp)],
                "lbm_plan_destroy": [vp],
                "lbm_plan_set_kernels": [vp, C.POINTER(lbm_kernel_choice)],
                "lbm_plan_get_kernels": [vp, C.POINTER(lbm_kernel_choice)],
                "lbm_workspace_size": [vp, C.POINTER(C.c_size_t)],
                "lbm_init_geometry": [vp, C.POINTER(lbm_geom_desc), vp, vp, vp, vp, vp],
                "lbm_bind_geometry": [vp, vp],
                "lbm_compact_size": [vp, C.c_int64, C.POINTER(C.c_size_t)],
                "lbm_compact_bind": [vp, C.c_int64, vp, vp],
                "lbm_set_abb_velocity": [vp, i32],
                "lbm_set_collision": [vp, i32, f64, f64, f64],
                "lbm_set_periodic_y": [vp, i32],
                "lbm_set_velocity_inlet": [vp, i32, f64, f64, f64],
                "lbm_set_velocity_ramp": [vp, i32],
                "lbm_adjoint_window": [vp, vp, vp, f64, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
                "lbm_get_collision": [vp, C.POINTER(C.c_int32), vp],
                "lbm_get_abb_velocity": [vp, C.POINTER(C.c_int32)],
                "lbm_probe_loss_grad": [vp, vp, C.c_int64, vp, vp, f64, vp, vp, vp, vp],
                "lbm_spline_basis": [i32, i32, vp],
                "lbm_spline_profile": [vp, i32, i32, vp, vp, vp, f64, vp, vp],
                "lbm_spline_grad": [vp, i32, i32, vp, vp, vp, vp, vp],
                "lbm_forward": [vp, vp, vp, f64, vp, vp, vp],
                "lbm_step": [vp, vp, vp, f64, vp, vp, i32, vp, vp],
                "lbm_loss_grad": [vp, vp, vp, vp, vp, vp, vp, vp],
                "lbm_loss_grad_noalloc": [vp, vp, vp, vp, vp, vp, vp],
                "lbm_adjoint": [vp, vp, vp, f64, vp, vp, vp, vp, vp],
                "lbm_macroscopic": [vp, vp, vp, vp, vp],
                "lbm_darcy": [vp, vp, vp, vp, f64, i32, vp, vp, vp],
                "lbm_adam_step": [i32, vp, vp, vp, vp, vp, f64, f64, i32, f64, f64, f64, f64, vp],
                "lbm_get_status": [vp, C.POINTER(C.c_int)],
                "lbm_batch_create": [C.POINTER(lbm_desc), i32, vp, vp, vp, C.POINTER(vp)],
                "lbm_batch_destroy": [vp],
                "lbm_batch_layout": [vp, vp, vp, vp, vp, C.POINTER(C.c_size_t)],
                "lbm_batch_init_geometry": [vp, vp, vp, vp, vp, vp, vp, vp],
                "lbm_batch_forward": [vp, vp, vp, f64, vp, vp, vp],
                "lbm_batch_loss_grad": [vp, vp, vp, vp, vp, vp, vp, vp],
                "lbm_batch_adjoint": [vp, vp, vp, f64, vp, vp, vp, vp, vp],
                "lbm_batch_compact_size": [vp, vp, C.POINTER(C.c_size_t)],
                "lbm_batch_compact_bind": [vp, vp, vp, vp, vp],
                "lbm_batch_get_status": [vp, vp, C.POINTER(C.c_int)],
                "lbm_error_string": [C.c_int],
                "unet_param_layout": [i32, vp, vp, vp, vp],
                "unet_workspace_size": [vp, C.POINTER(C.c_size_t)],
                "unet_pack_input": [vp, vp, vp, f64, vp, vp],
                "unet_prepare_weights": [vp, vp, vp, vp],
                "unet_forward": [vp, vp, vp, vp, vp],
                "unet_backward": [vp, vp, vp, vp, vp, vp, vp],
                "unet_adam": [C.c_int64, vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float, vp],
                "unet_set_engine": [i32],
                "unet_get_status": [],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = C.c_char_p if name == "lbm_error_string" else C.c_int
            _lib = lib
        return _lib


def _ptr(t: torch.Tensor | None, dtype: torch.dtype | None = None, numel: int | None = None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor has {t.numel()} elements, needs {numel}")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(st: int, where: str) -> None:
    if st != LBM_OK:
        raise LBMError(st, where)


def lbm_error_string(status: int) -> str:
    return load().lbm_error_string(int(status)).decode()


class Plan:
    """Owns an ``lbm_plan*``; attributes mirror ``lbm_desc``."""

    def __init__(self, q, nx, ny, nz=1, precision=4, n_steps=1, ckpt_stride=0, loss_kind=LBM_LOSS_VEC,
                 loss_norm=LBM_NORM_SUM, inlet_kind=LBM_INLET_CONST):
        self.desc = lbm_desc(q, nx, ny, nz, precision, n_steps, ckpt_stride, loss_kind, loss_norm, inlet_kind)
        h = C.c_void_p()
        _check(load().lbm_plan_create(C.byref(self.desc), C.byref(h)), "lbm_plan_create")
        self.handle = h
        self.q, self.nx, self.ny, self.nz = q, nx, ny, nz
        self.precision, self.n_steps = precision, n_steps
        self.inlet_kind = inlet_kind
        self.d = 2 if q == 9 else 3
        self.N = nx * ny * nz
        self.n_in = ny * nz if inlet_kind == LBM_INLET_PROFILE else 1
        self.dtype = torch.float32 if precision == 4 else torch.float64

    @property
    def shape(self):
        """Node-field shape: (ny, nx) for D2Q9, (nz, ny, nx) for D3Q19."""
        return (self.ny, self.nx) if self.q == 9 else (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.lbm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_plan_create(q, nx, ny, nz=1, precision=4, n_steps=1, ckpt_stride=0, loss_kind=LBM_LOSS_VEC,
                    loss_norm=LBM_NORM_SUM, inlet_kind=LBM_INLET_CONST) -> Plan:
    return Plan(q, nx, ny, nz, precision, n_steps, ckpt_stride, loss_kind, loss_norm, inlet_kind)


def lbm_plan_destroy(plan: Plan) -> None:
    plan.close()


def lbm_plan_set_kernels(plan: Plan, step_family=LBM_FAMILY_AUTO, adjoint_family=LBM_FAMILY_AUTO, vec=4,
                         tma_rows=8, pdl=1, persist=0, overlap=1, adjoint_tma_rows=0, steps_per_launch=1,
                         aa=0, recompute_family=LBM_FAMILY_AUTO) -> None:
    k = lbm_kernel_choice(step_family, adjoint_family, vec, tma_rows, pdl, persist, overlap, adjoint_tma_rows,
                          steps_per_launch, recompute_family, aa)
    _check(load().lbm_plan_set_kernels(plan.handle, C.byref(k)), "lbm_plan_set_kernels")


def lbm_plan_get_kernels(plan: Plan) -> dict:
    k = lbm_kernel_choice()
    _check(load().lbm_plan_get_kernels(plan.handle, C.byref(k)), "lbm_plan_get_kernels")
    return {f: getattr(k, f) for f, _ in lbm_kernel_choice._fields_}


def lbm_workspace_size(plan: Plan) -> int:
    n = C.c_size_t()
    _check(load().lbm_workspace_size(plan.handle, C.byref(n)), "lbm_workspace_size")
    return n.value


def lbm_init_geometry(plan: Plan, mask, link, info, porosity=None, kind=LBM_GEOM_CHANNEL, seed=0, r_min=6,
                      r_max=12, target_porosity=1.0, hydro_q8=256, inlet_buffer=8, fill_isolated=True,
                      max_rejections=1_000_000, stream=None) -> None:
    g = lbm_geom_desc(kind, r_min, r_max, hydro_q8, inlet_buffer, 1 if fill_isolated else 0, max_rejections,
                      seed, float(target_porosity))
    _check(load().lbm_init_geometry(plan.handle, C.byref(g), _ptr(mask, torch.uint8, plan.N),
                                    _ptr(link, torch.int32, plan.N), _ptr(porosity, torch.float64, 1),
                                    _ptr(info, torch.int64, 4), _stream(stream)), "lbm_init_geometry")
    plan._link = link  # keep the bound geometry alive with the plan
    plan._mask = mask


def lbm_bind_geometry(plan: Plan, link) -> None:
    _check(load().lbm_bind_geometry(plan.handle, _ptr(link, torch.int32, plan.N)), "lbm_bind_geometry")
    plan._link = link


def lbm_compact_size(plan: Plan, n_fluid: int) -> int:
    n = C.c_size_t()
    _check(load().lbm_compact_size(plan.handle, int(n_fluid), C.byref(n)), "lbm_compact_size")
    return n.value


def lbm_compact_bind(plan: Plan, n_fluid: int, tables, stream=None) -> None:
    _check(load().lbm_compact_bind(plan.handle, int(n_fluid), _ptr(tables, torch.uint8), _stream(stream)),
           "lbm_compact_bind")
    plan._tables = tables  # the plan reads the tables while it is bound to them


def lbm_set_abb_velocity(plan: Plan, mode: int) -> None:
    _check(load().lbm_set_abb_velocity(plan.handle, int(mode)), "lbm_set_abb_velocity")


def lbm_get_abb_velocity(plan: Plan) -> int:
    m = C.c_int32()
    _check(load().lbm_get_abb_velocity(plan.handle, C.byref(m)), "lbm_get_abb_velocity")
    return m.value


def lbm_set_collision(plan: Plan, mode: int, s_e: float = 1.0, s_eps: float = 1.0, s_q: float = 1.0) -> None:
    _check(load().lbm_set_collision(plan.handle, int(mode), float(s_e), float(s_eps), float(s_q)),
           "lbm_set_collision")


def lbm_set_periodic_y(plan: Plan, on: bool) -> None:
    _check(load().lbm_set_periodic_y(plan.handle, 1 if on else 0), "lbm_set_periodic_y")


def lbm_set_velocity_inlet(plan: Plan, u) -> None:
    """u = (ux, uy[, uz]) turns the velocity inlet on; None turns it off (Eq. 6)."""
    v = [0.0, 0.0, 0.0] if u is None else [float(a) for a in u] + [0.0] * (3 - len(u))
    _check(load().lbm_set_velocity_inlet(plan.handle, 0 if u is None else 1, *v), "lbm_set_velocity_inlet")


def lbm_set_velocity_ramp(plan: Plan, steps: int) -> None:
    """Gradual start of the velocity inlet over `steps` steps (0: none)."""
    _check(load().lbm_set_velocity_ramp(plan.handle, int(steps)), "lbm_set_velocity_ramp")


def lbm_adjoint_window(plan: Plan, rho_in, tau, rho_out: float, f_T, steps, u_targets, roi, scratch_f,
                       scratch_lam, loss, grad_rho_in, grad_tau, ws, stream=None) -> None:
    """Window loss sum_k L(f^{t_k}) and its gradient in one reverse sweep
    (after lbm_forward); steps: host int sequence, u_targets [n_obs, D, ...]."""
    import numpy as np

    st = np.ascontiguousarray(np.asarray(steps, np.int32))
    n = int(st.size)
    _check(load().lbm_adjoint_window(plan.handle, _ptr(rho_in, torch.float64, plan.n_in), _ptr(tau, torch.float64, 1),
                                     float(rho_out), _ptr(f_T, plan.dtype, plan.q * plan.N), n,
                                     st.ctypes.data_as(C.c_void_p), _ptr(u_targets, torch.float64, n * plan.d * plan.N),
                                     _ptr(roi, torch.uint8, plan.N), _ptr(scratch_f, plan.dtype, plan.q * plan.N),
                                     _ptr(scratch_lam, plan.dtype, plan.q * plan.N), _ptr(loss, torch.float64, 1),
                                     _ptr(grad_rho_in, torch.float64, plan.n_in), _ptr(grad_tau, torch.float64, 1),
                                     _ptr(ws, torch.uint8), _stream(stream)), "lbm_adjoint_window")


def lbm_get_collision(plan: Plan):
    """(mode, (s_e, s_eps, s_q))."""
    m = C.c_int32()
    r = (C.c_double * 3)()
    _check(load().lbm_get_collision(plan.handle, C.byref(m), C.cast(r, C.c_void_p)), "lbm_get_collision")
    return m.value, tuple(r)


def lbm_forward(plan: Plan, rho_in, tau, rho_out: float, f, ws, stream=None) -> None:
    _check(load().lbm_forward(plan.handle, _ptr(rho_in, torch.float64, plan.n_in), _ptr(tau, torch.float64, 1),
                              float(rho_out), _ptr(f, plan.dtype, plan.q * plan.N), _ptr(ws, torch.uint8),
                              _stream(stream)), "lbm_forward")


def lbm_step(plan: Plan, rho_in, tau, rho_out: float, f_in, f_out, n_steps: int, ws, stream=None) -> None:
    _check(load().lbm_step(plan.handle, _ptr(rho_in, torch.float64, plan.n_in), _ptr(tau, torch.float64, 1),
                           float(rho_out), _ptr(f_in, plan.dtype, plan.q * plan.N),
                           _ptr(f_out, plan.dtype, plan.q * plan.N), int(n_steps), _ptr(ws, torch.uint8),
                           _stream(stream)), "lbm_step")


def lbm_loss_grad(plan: Plan, f, u_target, roi, loss, lam, ws, stream=None) -> None:
    _check(load().lbm_loss_grad(plan.handle, _ptr(f, plan.dtype, plan.q * plan.N),
                                _ptr(u_target, torch.float64, plan.d * plan.N), _ptr(roi, torch.uint8, plan.N),
                                _ptr(loss, torch.float64, 1), _ptr(lam, plan.dtype, plan.q * plan.N),
                                _ptr(ws, torch.uint8), _stream(stream)), "lbm_loss_grad")


LBM_NOALLOC_MAX_BLOCKS = 65536


def lbm_loss_grad_noalloc(plan: Plan, f, u_target, roi, loss, lam, stream=None) -> None:
    """lbm_loss_grad without a workspace, for callers that cannot allocate
    device memory: the reduction scratch is the library's own fixed device
    array (see include/lbm.h), shared by every call."""
    blocks = -(-plan.nx // 128) * plan.ny * plan.nz
    if blocks > LBM_NOALLOC_MAX_BLOCKS:
        raise LBMError(LBM_ERR_INVALID_ARG, f"lbm_loss_grad_noalloc: the loss grid needs {blocks} blocks, more "
                                            f"than the fixed scratch holds ({LBM_NOALLOC_MAX_BLOCKS})")
    _check(load().lbm_loss_grad_noalloc(plan.handle, _ptr(f, plan.dtype, plan.q * plan.N),
                                        _ptr(u_target, torch.float64, plan.d * plan.N),
                                        _ptr(roi, torch.uint8, plan.N), _ptr(loss, torch.float64, 1),
                                        _ptr(lam, plan.dtype, plan.q * plan.N), _stream(stream)),
           "lbm_loss_grad_noalloc")


def lbm_probe_loss_grad(plan: Plan, f, nodes, rho_target, weight: float, loss, lam, ws, stream=None) -> None:
    n = 0 if nodes is None else int(nodes.numel())
    _check(load().lbm_probe_loss_grad(plan.handle, _ptr(f, plan.dtype, plan.q * plan.N), n,
                                      _ptr(nodes, torch.int64, n) if n else None,
                                      _ptr(rho_target, torch.float64, n) if n else None, float(weight),
                                      _ptr(loss, torch.float64, 1), _ptr(lam, plan.dtype, plan.q * plan.N),
                                      _ptr(ws, torch.uint8), _stream(stream)), "lbm_probe_loss_grad")


def lbm_spline_basis(n_knots: int, n: int):
    """Host basis B[n, n_knots] of the natural cubic spline (a float64 numpy array)."""
    import numpy as np

    out = np.zeros((int(n), int(n_knots)), np.float64)
    _check(load().lbm_spline_basis(int(n_knots), int(n), out.ctypes.data_as(C.c_void_p)), "lbm_spline_basis")
    return out


def lbm_spline_profile(plan: Plan, by, bz, knots, rho_out: float, rho_in, stream=None) -> None:
    ky, kz = by.shape[1], bz.shape[1]
    _check(load().lbm_spline_profile(plan.handle, ky, kz, _ptr(by, torch.float64, plan.ny * ky),
                                     _ptr(bz, torch.float64, plan.nz * kz), _ptr(knots, torch.float64, ky * kz),
                                     float(rho_out), _ptr(rho_in, torch.float64, plan.n_in), _stream(stream)),
           "lbm_spline_profile")


def lbm_spline_grad(plan: Plan, by, bz, grad_rho_in, grad_knots, stream=None) -> None:
    ky, kz = by.shape[1], bz.shape[1]
    _check(load().lbm_spline_grad(plan.handle, ky, kz, _ptr(by, torch.float64, plan.ny * ky),
                                  _ptr(bz, torch.float64, plan.nz * kz), _ptr(grad_rho_in, torch.float64, plan.n_in),
                                  _ptr(grad_knots, torch.float64, ky * kz), _stream(stream)), "lbm_spline_grad")


def lbm_adjoint(plan: Plan, rho_in, tau, rho_out: float, lam, grad_rho_in, grad_tau, ws, stream=None) -> None:
    _check(load().lbm_adjoint(plan.handle, _ptr(rho_in, torch.float64, plan.n_in), _ptr(tau, torch.float64, 1),
                              float(rho_out), _ptr(lam, plan.dtype, plan.q * plan.N),
                              _ptr(grad_rho_in, torch.float64, plan.n_in), _ptr(grad_tau, torch.float64, 1),
                              _ptr(ws, torch.uint8), _stream(stream)), "lbm_adjoint")


def lbm_macroscopic(plan: Plan, f, rho, u, stream=None) -> None:
    _check(load().lbm_macroscopic(plan.handle, _ptr(f, plan.dtype, plan.q * plan.N), _ptr(rho, torch.float64, plan.N),
                                  _ptr(u, torch.float64, plan.d * plan.N), _stream(stream)), "lbm_macroscopic")


def lbm_darcy(plan: Plan, f, rho_in, tau, rho_out: float, xs: int, k, flux=None, stream=None) -> None:
    _check(load().lbm_darcy(plan.handle, _ptr(f, plan.dtype, plan.q * plan.N), _ptr(rho_in, torch.float64, plan.n_in),
                            _ptr(tau, torch.float64, 1), float(rho_out), int(xs), _ptr(k, torch.float64, 1),
                            _ptr(flux, torch.float64, 1), _stream(stream)), "lbm_darcy")


def lbm_adam_step(theta, m, v, grad_p, p, p_offset: float, p_scale: float, t: int, lr: float, beta1=0.9,
                  beta2=0.999, eps=1e-8, stream=None) -> None:
    n = theta.numel()
    _check(load().lbm_adam_step(n, _ptr(theta, torch.float64), _ptr(m, torch.float64, n), _ptr(v, torch.float64, n),
                                _ptr(grad_p, torch.float64, n), _ptr(p, torch.float64, n), float(p_offset),
                                float(p_scale), int(t), float(lr), float(beta1), float(beta2), float(eps),
                                _stream(stream)), "lbm_adam_step")


def lbm_get_status(plan: Plan) -> int:
    st = C.c_int()
    _check(load().lbm_get_status(plan.handle, C.byref(st)), "lbm_get_status")
    return st.value


class Solver:
    """One plan with its geometry and workspace held in torch device memory.

    ``geometry``: dict of ``lbm_init_geometry`` keyword arguments (kind, seed,
    r_min, r_max, target_porosity, ...), or a uint8 mask tensor (kind MASK).

    ``layout``: "dense" (every node stored), "compact" (fluid nodes only,
    ``lbm_compact_bind``), or "auto" (compact for D3Q19, dense for D2Q9).
    The default comes from the LBM_LAYOUT environment variable, else "auto".
    Every array the caller sees is dense either way."""

    def __init__(self, q, nx, ny, nz=1, precision=4, n_steps=1, ckpt_stride=0, loss_kind=LBM_LOSS_VEC,
                 loss_norm=LBM_NORM_SUM, inlet_kind=LBM_INLET_CONST, geometry=None, device="cuda", link=None,
                 mask=None, layout=None, periodic_y=False):
        self.device = torch.device(device)
        self.plan = Plan(q, nx, ny, nz, precision, n_steps, ckpt_stride, loss_kind, loss_norm, inlet_kind)
        self.periodic_y = bool(periodic_y)
        if periodic_y:  # before the geometry: it shapes the link words (fluid-only layout only)
            lbm_set_periodic_y(self.plan, True)
            layout = "compact"
        # the library replays its T-step sweeps as CUDA graphs on a non-default stream
        self.stream = torch.cuda.Stream(device=self.device)
        p = self.plan
        self.ws = torch.zeros(lbm_workspace_size(p), dtype=torch.uint8, device=self.device)
        if link is not None:
            self.link, self.mask = link, mask
            lbm_bind_geometry(p, link)
            self.info = None
            self.porosity = None
        else:
            self.mask = torch.zeros(((p.N + 3) // 4) * 4, dtype=torch.uint8, device=self.device)
            self.link = torch.zeros(p.N, dtype=torch.int32, device=self.device)
            self.info = torch.zeros(4, dtype=torch.int64, device=self.device)
            self.porosity = torch.zeros(1, dtype=torch.float64, device=self.device)
            if isinstance(geometry, torch.Tensor):
                self.mask[: p.N].copy_(geometry.reshape(-1).to(torch.uint8))
                lbm_init_geometry(p, self.mask, self.link, self.info, self.porosity, kind=LBM_GEOM_MASK,
                                  fill_isolated=False)
            else:
                lbm_init_geometry(p, self.mask, self.link, self.info, self.porosity, **(geometry or {}))
        self.layout, self.tables = "dense", None
        layout = layout or os.environ.get("LBM_LAYOUT", "auto")
        if layout not in ("dense", "compact", "auto"):
            raise ValueError(f"layout must be dense, compact or auto, not {layout!r}")
        self.set_layout(("compact" if q == 19 else "dense") if layout == "auto" else layout)

    def set_layout(self, layout: str) -> None:
        """Switches the plan between the dense and the fluid-only state layout
        (results are the same; the workspace is reallocated)."""
        p = self.plan
        if layout == self.layout:
            return
        if layout == "compact":
            with torch.cuda.device(self.device):
                torch.cuda.current_stream().synchronize()
            nf = int(self.info[3].item()) if self.info is not None else int((self.link[: p.N] >= 0).sum().item())
            if nf == 0:
                return  # nothing to compact: an all-solid lattice stays dense
            tables = torch.empty(max(lbm_compact_size(p, nf), 256), dtype=torch.uint8, device=self.device)
            self.run(lambda: lbm_compact_bind(p, nf, tables, self.stream))
            self.tables, self.n_fluid = tables, nf
        elif layout == "dense":
            self.run(lambda: lbm_compact_bind(p, 0, None, self.stream))
            self.tables = None
        else:
            raise ValueError(f"layout must be dense or compact, not {layout!r}")
        self.layout = layout
        self.ws = torch.zeros(lbm_workspace_size(p), dtype=torch.uint8, device=self.device)

    def run(self, fn):
        """Runs fn() on the solver's stream, ordered after and before the caller's stream."""
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            out = fn()
        cur.wait_stream(self.stream)
        return out

    @property
    def mask_field(self) -> torch.Tensor:
        return self.mask[: self.plan.N].reshape(self.plan.shape)

    def new_state(self) -> torch.Tensor:
        return torch.empty((self.plan.q, *self.plan.shape), dtype=self.plan.dtype, device=self.device)

    def set_kernels(self, **choice) -> None:
        """lbm_plan_set_kernels, then a larger workspace where the choice needs one."""
        lbm_plan_set_kernels(self.plan, **choice)
        self._fit_ws()

    def _fit_ws(self) -> None:
        # clearing the in-place schedule (aa) after the workspace was sized for it grows the need by two states
        need = lbm_workspace_size(self.plan)
        if need > self.ws.numel():
            self.ws = torch.zeros(need, dtype=torch.uint8, device=self.device)

    def forward(self, rho_in, tau, rho_out, f=None):
        f = self.new_state() if f is None else f
        self._fit_ws()
        self.run(lambda: lbm_forward(self.plan, rho_in, tau, rho_out, f, self.ws))
        return f

    def step(self, rho_in, tau, rho_out, f_in, n_steps, f_out=None):
        f_out = torch.empty_like(f_in) if f_out is None else f_out
        self._fit_ws()
        self.run(lambda: lbm_step(self.plan, rho_in, tau, rho_out, f_in, f_out, n_steps, self.ws))
        return f_out

    def loss_grad(self, f, u_target, roi=None, loss=None, lam=None):
        loss = torch.zeros(1, dtype=torch.float64, device=self.device) if loss is None else loss
        lam = self.new_state() if lam is None else lam
        self.run(lambda: lbm_loss_grad(self.plan, f, u_target, roi, loss, lam, self.ws))
        return loss, lam

    def probe_loss_grad(self, f, nodes, rho_target, weight, loss, lam):
        """Adds the density-probe term to loss and its seed to lam (after loss_grad)."""
        self.run(lambda: lbm_probe_loss_grad(self.plan, f, nodes, rho_target, weight, loss, lam, self.ws))
        return loss, lam

    def set_collision(self, mode: int, s_e: float = 1.0, s_eps: float = 1.0, s_q: float = 1.0) -> None:
        """LBM_COLLISION_BGK (default) or LBM_COLLISION_MRT with the free rates (D2Q9)."""
        lbm_set_collision(self.plan, mode, s_e, s_eps, s_q)

    def set_velocity_inlet(self, u) -> None:
        """A velocity inlet u = (ux, uy[, uz]) through x = -1/2 (None: Eq. 6).  It runs in the
        fluid-only layout, which this switches to."""
        lbm_set_velocity_inlet(self.plan, u)
        if u is not None and self.layout != "compact":
            self.set_layout("compact")

    def set_abb_velocity(self, mode: int) -> None:
        """LBM_ABB_U_NODE (default) or LBM_ABB_U_EXTRAP: where Eq. 6 takes its velocity."""
        lbm_set_abb_velocity(self.plan, mode)

    def adjoint(self, rho_in, tau, rho_out, lam, g_in=None, g_tau=None):
        g_in = torch.zeros(self.plan.n_in, dtype=torch.float64, device=self.device) if g_in is None else g_in
        g_tau = torch.zeros(1, dtype=torch.float64, device=self.device) if g_tau is None else g_tau
        self.run(lambda: lbm_adjoint(self.plan, rho_in, tau, rho_out, lam, g_in, g_tau, self.ws))
        return g_in, g_tau

    def set_velocity_ramp(self, steps: int) -> None:
        """The velocity inlet starts gradually over `steps` steps."""
        lbm_set_velocity_ramp(self.plan, steps)

    def adjoint_window(self, rho_in, tau, rho_out, f_T, steps, u_targets, roi=None):
        """(L, dL/drho_in, dL/dtau) of the window loss sum_k L(f^{t_k}) against
        u_targets [n_obs, D, ...] at the host steps t_k, after forward() with
        the same parameters returned f_T."""
        if not hasattr(self, "_win_scratch") or self._win_scratch[0].numel() != self.plan.q * self.plan.N:
            self._win_scratch = (self.new_state(), self.new_state())
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        g_in = torch.zeros(self.plan.n_in, dtype=torch.float64, device=self.device)
        g_tau = torch.zeros(1, dtype=torch.float64, device=self.device)
        a, b = self._win_scratch
        self.run(lambda: lbm_adjoint_window(self.plan, rho_in, tau, rho_out, f_T, steps, u_targets.contiguous(), roi,
                                            a, b, loss, g_in, g_tau, self.ws))
        return loss, g_in, g_tau

    def macroscopic(self, f):
        rho = torch.empty(self.plan.shape, dtype=torch.float64, device=self.device)
        u = torch.empty((self.plan.d, *self.plan.shape), dtype=torch.float64, device=self.device)
        self.run(lambda: lbm_macroscopic(self.plan, f, rho, u))
        return rho, u

    def darcy(self, f, rho_in, tau, rho_out, xs=None):
        k = torch.zeros(1, dtype=torch.float64, device=self.device)
        flux = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.run(lambda: lbm_darcy(self.plan, f, rho_in, tau, rho_out, self.plan.nx // 2 if xs is None else xs, k,
                                   flux))
        return k, flux

    def status(self) -> int:
        return lbm_get_status(self.plan)


# ----------------------------------------------------------------- batches

class Batch:
    """Many independent lattices of different sizes advanced together
    (lbm_batch_*).  ``sizes``: list of (nx, ny, nz); ``geometries``: one
    lbm_init_geometry keyword dict per instance; ``layout``: "dense" or
    "compact" (every instance's fluid nodes packed, lbm_batch_compact_bind).
    Packed device buffers are allocated with torch; ``view_*`` give
    per-instance views into them."""

    def __init__(self, q, sizes, precision=4, n_steps=1, ckpt_stride=0, loss_kind=LBM_LOSS_VEC,
                 loss_norm=LBM_NORM_SUM, inlet_kind=LBM_INLET_CONST, geometries=None, device="cuda", layout="dense"):
        import numpy as np

        self.device = torch.device(device)
        self.q, self.d, self.n = q, 2 if q == 9 else 3, len(sizes)
        self.sizes = [tuple(int(v) for v in sz) for sz in sizes]
        self.precision, self.n_steps, self.inlet_kind = precision, n_steps, inlet_kind
        self.dtype = torch.float32 if precision == 4 else torch.float64
        desc = lbm_desc(q, 0, 0, 0, precision, n_steps, ckpt_stride, loss_kind, loss_norm, inlet_kind)
        nx = (C.c_int32 * self.n)(*[sz[0] for sz in self.sizes])
        ny = (C.c_int32 * self.n)(*[sz[1] for sz in self.sizes])
        nz = (C.c_int32 * self.n)(*[sz[2] for sz in self.sizes])
        h = C.c_void_p()
        _check(load().lbm_batch_create(C.byref(desc), self.n, nx, ny, nz, C.byref(h)), "lbm_batch_create")
        self.handle = h
        offs = [np.zeros(self.n + 1, np.int64) for _ in range(4)]
        wsb = C.c_size_t()
        _check(load().lbm_batch_layout(h, *[o.ctypes.data_as(C.c_void_p) for o in offs], C.byref(wsb)),
               "lbm_batch_layout")
        self.state_off, self.node_off, self.vel_off, self.inlet_off = offs
        self.ws = torch.zeros(wsb.value, dtype=torch.uint8, device=self.device)
        nodes = int(self.node_off[-1])
        self.mask = torch.zeros(((nodes + 3) // 4) * 4, dtype=torch.uint8, device=self.device)
        self.link = torch.zeros(nodes, dtype=torch.int32, device=self.device)
        self.porosity = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        self.info = torch.zeros(4 * self.n, dtype=torch.int64, device=self.device)
        self.geometries = [dict(g) for g in (geometries or [{}] * self.n)]
        self.ckpt_stride, self.loss_kind, self.loss_norm = ckpt_stride, loss_kind, loss_norm
        geoms = (lbm_geom_desc * self.n)()
        for i, g in enumerate(geometries or [{}] * self.n):
            a = dict(kind=LBM_GEOM_CHANNEL, seed=0, r_min=6, r_max=12, target_porosity=1.0, hydro_q8=256,
                     inlet_buffer=8, fill_isolated=True, max_rejections=1_000_000)
            a.update(g)
            geoms[i] = lbm_geom_desc(a["kind"], a["r_min"], a["r_max"], a["hydro_q8"], a["inlet_buffer"],
                                     1 if a["fill_isolated"] else 0, a["max_rejections"], a["seed"],
                                     float(a["target_porosity"]))
        self.stream = torch.cuda.Stream(device=self.device)
        _check(load().lbm_batch_init_geometry(h, geoms, _ptr(self.mask), _ptr(self.link), _ptr(self.porosity),
                                              _ptr(self.info), _ptr(self.ws), _stream(None)),
               "lbm_batch_init_geometry")

        self.layout, self.tables = "dense", None
        self.set_layout(layout)

    def _run(self, fn):
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            fn()
        cur.wait_stream(self.stream)

    def set_layout(self, layout: str) -> None:
        """Dense or packed fluid-only ("compact") internal states (the same
        results; the packed arrays the caller sees do not change)."""
        if layout == self.layout:
            return
        if layout == "compact":
            import numpy as np

            torch.cuda.current_stream(self.device).synchronize()
            nf = self.info.view(self.n, 4)[:, 3].cpu().numpy().astype(np.int64)
            nbytes = C.c_size_t()
            _check(load().lbm_batch_compact_size(self.handle, nf.ctypes.data_as(C.c_void_p), C.byref(nbytes)),
                   "lbm_batch_compact_size")
            tables = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
            self._run(lambda: _check(load().lbm_batch_compact_bind(self.handle, nf.ctypes.data_as(C.c_void_p),
                                                                   _ptr(tables), _ptr(self.ws),
                                                                   _stream(self.stream)), "lbm_batch_compact_bind"))
            self.tables = tables
        elif layout == "dense":
            self._run(lambda: _check(load().lbm_batch_compact_bind(self.handle, None, None, _ptr(self.ws),
                                                                   _stream(self.stream)), "lbm_batch_compact_bind"))
            self.tables = None
        else:
            raise ValueError(f"layout must be dense or compact, not {layout!r}")
        self.layout = layout

    def status(self) -> int:
        """Reads and clears the batch's device status word."""
        st = C.c_int()
        _check(load().lbm_batch_get_status(self.handle, _ptr(self.ws), C.byref(st)), "lbm_batch_get_status")
        return st.value

    # sizes of the packed buffers
    def new_state(self):
        return torch.empty(int(self.state_off[-1]), dtype=self.dtype, device=self.device)

    def new_velocity(self):
        return torch.zeros(int(self.vel_off[-1]), dtype=torch.float64, device=self.device)

    def new_inlet(self):
        return torch.zeros(int(self.inlet_off[-1]), dtype=torch.float64, device=self.device)

    def shape(self, i):
        nx, ny, nz = self.sizes[i]
        return (ny, nx) if self.q == 9 else (nz, ny, nx)

    def nodes(self, i):
        nx, ny, nz = self.sizes[i]
        return nx * ny * nz

    def view_state(self, t, i):
        o = int(self.state_off[i])
        return t[o:o + self.q * self.nodes(i)].view(self.q, *self.shape(i))

    def view_mask(self, i):
        o = int(self.node_off[i])
        return self.mask[o:o + self.nodes(i)].view(*self.shape(i))

    def view_velocity(self, t, i):
        o = int(self.vel_off[i])
        return t[o:o + self.d * self.nodes(i)].view(self.d, *self.shape(i))

    def view_inlet(self, t, i):
        o = int(self.inlet_off[i])
        n = self.sizes[i][1] * self.sizes[i][2] if self.inlet_kind == LBM_INLET_PROFILE else 1
        return t[o:o + n]

    def velocity(self, f):
        """Packed velocity fields (Eq. 1-2, solids 0) of a packed state: per
        instance, lbm_macroscopic on a plan bound to its link words."""
        u = self.new_velocity()
        for i in range(self.n):
            nx, ny, nz = self.sizes[i]
            p = Plan(self.q, nx, ny, nz, self.precision, 1)
            o = int(self.node_off[i])
            lbm_bind_geometry(p, self.link[o:o + nx * ny * nz])
            ui = torch.empty((self.d, *self.shape(i)), dtype=torch.float64, device=self.device)
            self._run(lambda: lbm_macroscopic(p, self.view_state(f, i).contiguous(), None, ui, self.stream))
            self.view_velocity(u, i).copy_(ui)
        return u

    def forward(self, rho_in, tau, rho_out, f=None):
        f = self.new_state() if f is None else f
        self._run(lambda: _check(load().lbm_batch_forward(self.handle, _ptr(rho_in, torch.float64),
                                                          _ptr(tau, torch.float64, self.n), float(rho_out),
                                                          _ptr(f, self.dtype), _ptr(self.ws),
                                                          _stream(self.stream)), "lbm_batch_forward"))
        return f

    def loss_grad(self, f, u_target, roi=None, loss=None, lam=None):
        loss = torch.zeros(self.n, dtype=torch.float64, device=self.device) if loss is None else loss
        lam = self.new_state() if lam is None else lam
        self._run(lambda: _check(load().lbm_batch_loss_grad(self.handle, _ptr(f, self.dtype),
                                                            _ptr(u_target, torch.float64), _ptr(roi, torch.uint8),
                                                            _ptr(loss, torch.float64, self.n),
                                                            _ptr(lam, self.dtype), _ptr(self.ws),
                                                            _stream(self.stream)), "lbm_batch_loss_grad"))
        return loss, lam

    def adjoint(self, rho_in, tau, rho_out, lam, g_in=None, g_tau=None):
        g_in = self.new_inlet() if g_in is None else g_in
        g_tau = torch.zeros(self.n, dtype=torch.float64, device=self.device) if g_tau is None else g_tau
        self._run(lambda: _check(load().lbm_batch_adjoint(self.handle, _ptr(rho_in, torch.float64),
                                                          _ptr(tau, torch.float64, self.n), float(rho_out),
                                                          _ptr(lam, self.dtype), _ptr(g_in, torch.float64),
                                                          _ptr(g_tau, torch.float64, self.n), _ptr(self.ws),
                                                          _stream(self.stream)), "lbm_batch_adjoint"))
        return g_in, g_tau

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
