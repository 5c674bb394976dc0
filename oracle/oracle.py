"""Python access to the FP64 CPU oracle (``lbm_oracle.c``, ``geometry.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product package never imports it, and it imports nothing from the
product package.

Arrays follow the oracle's dense layout: populations ``f[Q, nz, ny, nx]``
(unshifted), velocities ``u[D, nz, ny, nx]``, masks ``uint8[nz, ny, nx]``.
Every routine here is a thin ctypes marshalling layer over the C code; the
arithmetic is all in C.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_CS = os.path.join(_BUILD, "liboracle_cs.so")
_SRC = [os.path.join(_HERE, "lbm_oracle.c"), os.path.join(_HERE, "geometry.c")]
_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-fopenmp"]

_lock = threading.Lock()
_libs: dict = {}

LOSS_VEC, LOSS_NORM = 0, 1
NORM_SUM, NORM_MEAN_FLUID = 0, 1
GEOM_CHANNEL, GEOM_DISKS, GEOM_SPHERES = 0, 1, 2
UW_NODE, UW_EXTRAP = 0, 1


def build(force: bool = False) -> None:
    """Compile the oracle with gcc (plain C, no -ffast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    jobs = [
        (_LIB, _SRC, []),
        (_LIB_CS, [_SRC[0]], ["-DORC_COMPLEX"]),
    ]
    for out, srcs, extra in jobs:
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        tmp = out + ".tmp"
        subprocess.check_call(["gcc", *_CFLAGS, *extra, "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, out)


def _lib(cs: bool = False):
    key = "cs" if cs else "re"
    with _lock:
        if key not in _libs:
            build()
            _libs[key] = C.CDLL(_LIB_CS if cs else _LIB)
        return _libs[key]


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _dims(q: int, shape) -> tuple[int, int, int]:
    if q == 9:
        ny, nx = shape[-2:]
        return nx, ny, 1
    nz, ny, nx = shape[-3:]
    return nx, ny, nz


def set_threads(n: int) -> int:
    """OpenMP threads for the per-node loops (results do not depend on it)."""
    return int(_lib().orc_set_threads(int(n)))


def set_abb_velocity(mode: int) -> None:
    """Where Eq. 6 takes its velocity: UW_NODE (the boundary node's own, the
    default) or UW_EXTRAP (extrapolated to the pressure plane).  Applies to
    every later call, in both the real and the complex-step builds."""
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_abb_velocity if cs else lib.orc_set_abb_velocity
        _check(fn(int(mode)), "set_abb_velocity")


COLL_BGK, COLL_MRT = 0, 1


def set_collision(mode: int, s_e: float = 1.0, s_eps: float = 1.0, s_q: float = 1.0) -> None:
    """BGK (default) or the D2Q9 MRT operator of Eq. 16-18 with the free
    rates s_e, s_eps, s_q (the stress rates are 1/tau); applies to every later
    call, in both builds."""
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_collision if cs else lib.orc_set_collision
        fn.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        _check(fn(int(mode), float(s_e), float(s_eps), float(s_q)), "set_collision")


class collision:
    """``with collision(COLL_MRT, s_e, s_eps, s_q): ...`` sets the operator for the block."""

    def __init__(self, mode: int, s_e: float = 1.0, s_eps: float = 1.0, s_q: float = 1.0):
        self.args = (mode, s_e, s_eps, s_q)

    def __enter__(self):
        set_collision(*self.args)
        return self

    def __exit__(self, *exc):
        set_collision(COLL_BGK)
        return False


def set_periodic_y(on: bool) -> None:
    """Periodic top and bottom (both builds; every later call)."""
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_periodic_y if cs else lib.orc_set_periodic_y
        _check(fn(1 if on else 0), "set_periodic_y")


def set_velocity_inlet(u) -> None:
    """Velocity inlet u = (u_x, u_y[, u_z]) through x = -1/2, or None for Eq. 6 (both builds)."""
    v = [0.0, 0.0, 0.0] if u is None else [float(a) for a in u] + [0.0] * (3 - len(u))
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_velocity_inlet if cs else lib.orc_set_velocity_inlet
        fn.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        _check(fn(0 if u is None else 1, *v), "set_velocity_inlet")


def set_velocity_ramp(steps: int) -> None:
    """Gradual start of the velocity inlet over `steps` steps (0: none): the
    step producing f^t uses u_in sin^2(pi t / (2 steps)) for t < steps (both builds)."""
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_velocity_ramp if cs else lib.orc_set_velocity_ramp
        _check(fn(int(steps)), "set_velocity_ramp")


def set_time(t_next: int) -> None:
    """The time level a lone step() call produces (forward and gradient set
    it themselves); matters only with a velocity ramp (both builds)."""
    for cs in (False, True):
        lib = _lib(cs)
        fn = lib.orc_cs_set_time if cs else lib.orc_set_time
        _check(fn(int(t_next)), "set_time")


class wake_options:
    """``with wake_options(periodic_y=True, velocity_inlet=(0.05, 0), ramp=500): ...``"""

    def __init__(self, periodic_y=False, velocity_inlet=None, ramp=0):
        self.p, self.u, self.r = periodic_y, velocity_inlet, ramp

    def __enter__(self):
        set_periodic_y(self.p)
        set_velocity_inlet(self.u)
        set_velocity_ramp(self.r)
        return self

    def __exit__(self, *exc):
        set_periodic_y(False)
        set_velocity_inlet(None)
        set_velocity_ramp(0)
        set_time(1)
        return False


class abb_velocity:
    """``with abb_velocity(UW_EXTRAP): ...`` sets the Eq. 6 velocity for the block."""

    def __init__(self, mode: int):
        self.mode = mode

    def __enter__(self):
        set_abb_velocity(self.mode)
        return self

    def __exit__(self, *exc):
        set_abb_velocity(UW_NODE)
        return False


def lattice(q: int):
    """Return (c[Q,3] int, w[Q] float64, opp[Q] int) as the oracle defines them."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    opp = np.zeros(q, np.int32)
    _check(_lib().orc_lattice(q, _p(c), _p(w), _p(opp)), "lattice")
    return c, w, opp


def splitmix64(seed: int, n: int) -> list[int]:
    """First n outputs of SplitMix64 from state ``seed``."""
    lib = _lib()
    lib.orc_splitmix64_next.restype = C.c_uint64
    s = C.c_uint64(seed)
    return [int(lib.orc_splitmix64_next(C.byref(s))) for _ in range(n)]


def geometry(q, nx, ny, nz=1, kind=GEOM_CHANNEL, seed=0, r_min=6, r_max=12, porosity=1.0, hydro_q8=256,
             buffer=8, max_rejections=1_000_000, fill=True):
    """Seeded grain packing (geometry.c).  Returns (mask uint8[nz,ny,nx] or [ny,nx], info int64[4])."""
    mask = np.zeros(nx * ny * nz, np.uint8)
    info = np.zeros(4, np.int64)
    lib = _lib()
    lib.orc_geometry.argtypes = [C.c_int] * 5 + [C.c_uint64, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                                 C.c_long, C.c_int, C.c_void_p, C.c_void_p]
    _check(lib.orc_geometry(q, nx, ny, nz, kind, seed, r_min, r_max, float(porosity), hydro_q8, buffer,
                            max_rejections, 1 if fill else 0, _p(mask), _p(info)), "geometry")
    shape = (ny, nx) if q == 9 else (nz, ny, nx)
    return mask.reshape(shape), info


def links(q: int, mask: np.ndarray) -> np.ndarray:
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros(m.shape, np.uint32)
    _check(_lib().orc_links(q, nx, ny, nz, _p(m), _p(out)), "links")
    return out


def rest(q: int, shape) -> np.ndarray:
    """f^0 = w_i at every node (fluid at rest, rho = 1)."""
    _, w, _ = lattice(q)
    return np.broadcast_to(w.reshape((q,) + (1,) * len(shape)), (q, *shape)).astype(np.float64).copy()


def _real_args(rho_in, rho_out, tau, dtype):
    rin = np.ascontiguousarray(np.atleast_1d(np.asarray(rho_in, dtype)))
    rout = np.array([rho_out], dtype)
    t = np.array([tau], dtype)
    return rin, rout, t


def collide(q, f, tau):
    """BGK collision alone on an array f[Q, ...] of independent nodes."""
    fi = np.ascontiguousarray(f, np.float64)
    fo = np.empty_like(fi)
    t = np.array([tau], np.float64)
    _check(_lib().orc_collide(q, C.c_long(fi[0].size), _p(fi), _p(fo), _p(t)), "collide")
    return fo


def equilibrium(q, rho, u):
    """f^eq[Q, ...] (Eq. 5) for rho[...] and u[D, ...]."""
    r = np.ascontiguousarray(rho, np.float64)
    uu = np.ascontiguousarray(u, np.float64)
    fo = np.empty((q,) + r.shape, np.float64)
    _check(_lib().orc_equilibrium(q, C.c_long(r.size), _p(r), _p(uu), _p(fo)), "equilibrium")
    return fo


def step(q, mask, f, rho_in, rho_out, tau, complex_step=False):
    """One step f^{t+1} = stream(collide(f^t)).  rho_in: scalar (const head) or array [ny] / [nz, ny]."""
    dt = np.complex128 if complex_step else np.float64
    lib = _lib(complex_step)
    fn = lib.orc_cs_step if complex_step else lib.orc_step
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    fi = np.ascontiguousarray(f, dt)
    fo = np.empty_like(fi)
    rin, rout, t = _real_args(rho_in, rho_out, tau, dt)
    prof = 1 if rin.size > 1 else 0
    _check(fn(q, nx, ny, nz, _p(m), _p(fi), _p(fo), _p(rin), prof, _p(rout), _p(t)), "step")
    return fo


def forward(q, mask, rho_in, rho_out, tau, T, f0=None, tape=False, complex_step=False):
    """T steps from f0 (None: rest).  Returns f^T, or (f^T, tape[T, Q, ...]) with tape=True."""
    dt = np.complex128 if complex_step else np.float64
    lib = _lib(complex_step)
    fn = lib.orc_cs_forward if complex_step else lib.orc_forward
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    shape = (q,) + m.shape
    fT = np.empty(shape, dt)
    f0c = None if f0 is None else np.ascontiguousarray(f0, dt)
    tp = np.empty((T,) + shape, dt) if tape else None
    rin, rout, t = _real_args(rho_in, rho_out, tau, dt)
    prof = 1 if rin.size > 1 else 0
    _check(fn(q, nx, ny, nz, _p(m), _p(rin), prof, _p(rout), _p(t), int(T), _p(f0c), _p(fT), _p(tp)), "forward")
    return (fT, tp) if tape else fT


def macroscopic(q, mask, f):
    """(rho[...], u[D, ...]); solid nodes give 0."""
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    fi = np.ascontiguousarray(f, np.float64)
    d = 2 if q == 9 else 3
    rho = np.empty(m.shape, np.float64)
    u = np.empty((d,) + m.shape, np.float64)
    _check(_lib().orc_macroscopic(q, nx, ny, nz, _p(m), _p(fi), _p(rho), _p(u)), "macroscopic")
    return rho, u


def loss(q, mask, f, u_target, roi=None, kind=LOSS_VEC, norm=NORM_SUM, seed=True, complex_step=False):
    """Final-step loss; returns (L, lam = dL/df) or L if seed=False."""
    dt = np.complex128 if complex_step else np.float64
    lib = _lib(complex_step)
    fn = lib.orc_cs_loss if complex_step else lib.orc_loss
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    fi = np.ascontiguousarray(f, dt)
    ut = np.ascontiguousarray(u_target, np.float64)
    r = None if roi is None else np.ascontiguousarray(roi, np.uint8)
    out = np.zeros(1, dt)
    lam = np.empty_like(fi) if seed else None
    _check(fn(q, nx, ny, nz, _p(m), _p(fi), _p(ut), _p(r), kind, norm, _p(out), _p(lam)), "loss")
    return (out[0], lam) if seed else out[0]


def probe_loss(q, mask, f, nodes, rho_target, weight=1.0, complex_step=False):
    """Density-probe loss w sum_p (rho(x_p) - rho_p)^2 and its seed dL/df
    (nonzero only at the probe nodes); nodes are dense node indices."""
    dt = np.complex128 if complex_step else np.float64
    lib = _lib(complex_step)
    fn = lib.orc_cs_probe_loss if complex_step else lib.orc_probe_loss
    fn.argtypes = [C.c_int] * 4 + [C.c_void_p, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p, C.c_double,
                                   C.c_void_p, C.c_void_p]
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    fi = np.ascontiguousarray(f, dt)
    idx = np.ascontiguousarray(nodes, np.int64)
    rt = np.ascontiguousarray(rho_target, np.float64)
    assert idx.shape == rt.shape
    out = np.zeros(1, dt)
    lam = np.zeros_like(fi)
    _check(fn(q, nx, ny, nz, _p(m), _p(fi), idx.size, _p(idx), _p(rt), float(weight), _p(out), _p(lam)),
           "probe_loss")
    return out[0], lam


def adjoint_step(q, mask, f_t, lam_next, rho_in, rho_out, tau):
    """One reverse step: returns (lam_t, dL/drho_in contribution, dL/domega contribution)."""
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    ft = np.ascontiguousarray(f_t, np.float64)
    ln = np.ascontiguousarray(lam_next, np.float64)
    lo = np.empty_like(ln)
    rin, rout, t = _real_args(rho_in, rho_out, tau, np.float64)
    prof = 1 if rin.size > 1 else 0
    g_in = np.zeros(rin.size, np.float64)
    g_om = np.zeros(1, np.float64)
    _check(_lib().orc_adjoint_step(q, nx, ny, nz, _p(m), _p(ft), _p(ln), _p(lo), _p(rin), prof, _p(rout), _p(t),
                                   _p(g_in), _p(g_om)), "adjoint_step")
    return lo, g_in, g_om[0]


def gradient(q, mask, rho_in, rho_out, tau, T, u_target, roi=None, kind=LOSS_VEC, norm=NORM_SUM, ckpt_stride=0,
             f0=None, return_fT=False, probes=None):
    """Loss and gradients of the final-step loss: (L, dL/drho_in, dL/dtau[, f^T]).
    probes = (nodes, rho_target, weight) adds the density-probe term (probe_loss)."""
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    rin, rout, t = _real_args(rho_in, rho_out, tau, np.float64)
    prof = 1 if rin.size > 1 else 0
    ut = np.ascontiguousarray(u_target, np.float64)
    r = None if roi is None else np.ascontiguousarray(roi, np.uint8)
    f0c = None if f0 is None else np.ascontiguousarray(f0, np.float64)
    L = np.zeros(1)
    g_in = np.zeros(rin.size)
    g_tau = np.zeros(1)
    fT = np.empty((q,) + m.shape) if return_fT else None
    if probes is None:
        pn, pr, pw = np.zeros(0, np.int64), np.zeros(0), 0.0
    else:
        pn, pr = np.ascontiguousarray(probes[0], np.int64), np.ascontiguousarray(probes[1], np.float64)
        pw = float(probes[2])
        assert pn.shape == pr.shape
    _check(_lib().orc_gradient(q, nx, ny, nz, _p(m), _p(rin), prof, _p(rout), _p(t), int(T), _p(f0c), _p(ut), _p(r),
                               kind, norm, C.c_long(pn.size), _p(pn), _p(pr), C.c_double(pw), int(ckpt_stride),
                               _p(L), _p(g_in), _p(g_tau), _p(fT)), "gradient")
    g = g_in if prof else g_in[0]
    return (L[0], g, g_tau[0], fT) if return_fT else (L[0], g, g_tau[0])


def gradient_window(q, mask, rho_in, rho_out, tau, T, obs_steps, u_targets, roi=None, kind=LOSS_VEC,
                    norm=NORM_SUM, ckpt_stride=0):
    """Loss over a time window, L = sum_k L_k(f^{t_k}) (u_targets[k] the k-th
    target [D, ...], obs_steps the t_k in 0..T), and its gradient by one
    reverse sweep: (L, dL/drho_in, dL/dtau)."""
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    rin, rout, t = _real_args(rho_in, rho_out, tau, np.float64)
    prof = 1 if rin.size > 1 else 0
    obs = np.ascontiguousarray(obs_steps, np.int32)
    ut = np.ascontiguousarray(u_targets, np.float64)
    assert ut.shape[0] == obs.size
    r = None if roi is None else np.ascontiguousarray(roi, np.uint8)
    L = np.zeros(1)
    g_in = np.zeros(rin.size)
    g_tau = np.zeros(1)
    _check(_lib().orc_gradient_window(q, nx, ny, nz, _p(m), _p(rin), prof, _p(rout), _p(t), int(T), int(obs.size),
                                      _p(obs), _p(ut), _p(r), kind, norm, int(ckpt_stride), _p(L), _p(g_in),
                                      _p(g_tau)), "gradient_window")
    return L[0], (g_in if prof else g_in[0]), g_tau[0]


def adam(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays theta, m, v."""
    lib = _lib()
    lib.orc_adam.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                             C.c_double, C.c_double, C.c_double]
    g = np.ascontiguousarray(grad, np.float64)
    lib.orc_adam(theta.size, _p(theta), _p(g), _p(m), _p(v), int(t), lr, beta1, beta2, eps)


def darcy(q, mask, f, rho_in, rho_out, tau, xs=None):
    """(k, superficial mass flux J) at cross-section xs (default nx // 2), Eq. 12."""
    nx, ny, nz = _dims(q, mask.shape)
    m = np.ascontiguousarray(mask, np.uint8)
    fi = np.ascontiguousarray(f, np.float64)
    rin = np.ascontiguousarray(np.atleast_1d(np.asarray(rho_in, np.float64)))
    prof = 1 if rin.size > 1 else 0
    k = C.c_double()
    J = C.c_double()
    lib = _lib()
    lib.orc_darcy.argtypes = [C.c_int] * 4 + [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                              C.c_int, C.c_void_p, C.c_void_p]
    _check(lib.orc_darcy(q, nx, ny, nz, _p(m), _p(fi), _p(rin), prof, float(rho_out), float(tau),
                         nx // 2 if xs is None else int(xs), C.byref(k), C.byref(J)), "darcy")
    return k.value, J.value
