"""Parity at the benchmark's full lattice sizes, in the launch configuration
the benchmark uses (autotuned layout and kernel family).

The 512x256 D2Q9 disk packing (20000 steps in the benchmark) and the
128x64x64 D3Q19 sphere packing (10000 steps): the oracle checks every output
of shorter runs on the full lattices (FP32 and both layouts), and the FP32
velocity (both lattices) and gradient (D2Q9) at the full step counts.
Properties that hold at any step count are checked at the full T too: the
rest state is a fixed point when rho_in = rho_out, and the adjoint gradient
of an FP64 plan matches a central difference of its own forward sweep."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import autotune
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(name, T, precision=None, layout=None, tune=True):
    wl = W.WORKLOADS[name]
    inlet = lbm.LBM_INLET_PROFILE if wl.inlet == "profile" else lbm.LBM_INLET_CONST
    s = lbm.Solver(wl.q, wl.nx, wl.ny, wl.nz, precision=precision or wl.precision, n_steps=T, inlet_kind=inlet,
                   geometry=dict(kind=wl.geom_kind, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                                 target_porosity=wl.porosity), layout=layout)
    if tune:
        autotune.tune(s, cache=None)  # the benchmark's choice for this lattice, without the on-disk cache
    return wl, s


def inlet_of(wl, s):
    if wl.inlet == "profile":
        return wl.rho_out + W.inlet_profile(s.plan.n_in, seed=2000)
    return np.array([wl.rho_out + wl.delta_rho])


def oracle_inlet(wl, rin):
    if wl.inlet != "profile":
        return rin[0]
    return rin.reshape((wl.nz, wl.ny) if wl.q == 19 else (wl.ny,))


CASES = [("disks512x256", 200, 40, None), ("spheres128x64x64", 30, 10, "compact"),
         ("spheres128x64x64", 30, 10, "dense")]


@pytest.mark.parametrize("name,T_fwd,T_grad,layout", CASES, ids=[f"{c[0]}-{c[3] or 'auto'}" for c in CASES])
def test_fullsize_forward_and_gradient(name, T_fwd, T_grad, layout):
    wl, s = make(name, T_fwd, layout=layout)
    m = s.mask_field.cpu().numpy()
    rin = inlet_of(wl, s)
    f = s.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    _, u = s.macroscopic(f)
    want = O.forward(wl.q, m, oracle_inlet(wl, rin), wl.rho_out, wl.tau, T_fwd)
    _, u_w = O.macroscopic(wl.q, m, want)
    assert rel(u.cpu().numpy(), u_w) < 1e-4

    _, g = make(name, T_grad, layout=layout)
    ut = W.perturbation((g.plan.d, *m.shape), seed=2001, scale=1e-4)
    f = g.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    L, lam = g.loss_grad(f, dev(ut))
    g_in, g_tau = g.adjoint(dev(rin), dev([wl.tau]), wl.rho_out, lam)
    Lw, g_in_w, g_tau_w = O.gradient(wl.q, m, oracle_inlet(wl, rin), wl.rho_out, wl.tau, T_grad, ut,
                                     ckpt_stride=max(1, int(np.sqrt(T_grad))))
    assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
    assert rel(g_in.cpu().numpy(), np.ravel(g_in_w)) < 1e-3
    assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)


@pytest.mark.parametrize("name", ["disks512x256", "spheres128x64x64"])
def test_fullsize_rest_is_fixed_point_at_full_T(name):
    """rho_in = rho_out from rest: every step leaves the (shifted) state at
    exactly zero, over the benchmark's full step count."""
    wl, s = make(name, W.WORKLOADS[name].steps)
    rin = np.full(s.plan.n_in, wl.rho_out)
    f = s.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    assert torch.count_nonzero(f).item() == 0


@pytest.mark.parametrize("name,T", [("disks512x256", 20000), ("spheres128x64x64", 2000)])
def test_fullsize_fp64_gradient_matches_central_difference(name, T):
    """dL/d(head) of the adjoint sweep against (L(h + e) - L(h - e)) / 2e of
    the FP64 forward sweep, constant head, on the full lattice."""
    wl = W.WORKLOADS[name]
    s = lbm.Solver(wl.q, wl.nx, wl.ny, wl.nz, precision=8, n_steps=T, inlet_kind=lbm.LBM_INLET_CONST,
                   geometry=dict(kind=wl.geom_kind, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                                 target_porosity=wl.porosity))
    autotune.tune(s, cache=None)
    ut = W.perturbation((s.plan.d, *s.plan.shape), seed=2002, scale=1e-4)
    h, tau = 1e-3, dev([wl.tau])
    f = s.forward(dev([wl.rho_out + h]), tau, wl.rho_out)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, _ = s.adjoint(dev([wl.rho_out + h]), tau, wl.rho_out, lam)
    e = 1e-7
    Lp, _ = s.loss_grad(s.forward(dev([wl.rho_out + h + e]), tau, wl.rho_out), dev(ut))
    Lm, _ = s.loss_grad(s.forward(dev([wl.rho_out + h - e]), tau, wl.rho_out), dev(ut))
    fd = (Lp.item() - Lm.item()) / (2 * e)
    assert abs(g_in.item() - fd) <= 1e-5 * abs(fd)


# The benchmark lattices at their FULL step counts, FP32, in the benchmark's
# (autotuned) launch configuration, against the FP64 oracle run to the same
# T.  This is where FP32 drift over tens of thousands of steps would show:
# the bound is 1e-4 relative L2 on the (near-)steady velocity and 1e-3
# relative on the gradients.  The oracle takes a few minutes on the host cores.


def test_fullsize_fp32_d2q9_velocity_and_gradient_at_full_T():
    """512x256 D2Q9 FP32, T = 20000, the 256-entry profile: the velocity of
    f^T, then the loss, dL/drho_in and dL/dtau of one checkpointed gradient
    evaluation, against one oracle reverse sweep (sqrt(T) checkpoints; it
    also returns its f^T)."""
    name = "disks512x256"
    wl = W.WORKLOADS[name]
    _, s = make(name, wl.steps)
    m = s.mask_field.cpu().numpy()
    rin = inlet_of(wl, s)
    ut = W.perturbation((s.plan.d, *m.shape), seed=2003, scale=1e-4)
    f = s.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    _, u = s.macroscopic(f)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([wl.tau]), wl.rho_out, lam)
    Lw, g_in_w, g_tau_w, fT_w = O.gradient(wl.q, m, oracle_inlet(wl, rin), wl.rho_out, wl.tau, wl.steps, ut,
                                           ckpt_stride=int(np.ceil(np.sqrt(wl.steps))), return_fT=True)
    _, u_w = O.macroscopic(wl.q, m, fT_w)
    assert rel(u.cpu().numpy(), u_w) < 1e-4
    assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
    assert rel(g_in.cpu().numpy(), np.ravel(g_in_w)) < 1e-3
    assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)


def test_fullsize_fp32_d3q19_velocity_at_full_T():
    """128x64x64 D3Q19 FP32 duct, T = 10000, fluid-only layout (the
    benchmark's), constant head: the velocity of f^T against the oracle."""
    name = "spheres128x64x64"
    wl = W.WORKLOADS[name]
    _, s = make(name, wl.steps, layout="compact")
    m = s.mask_field.cpu().numpy()
    rin = inlet_of(wl, s)
    f = s.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    _, u = s.macroscopic(f)
    want = O.forward(wl.q, m, oracle_inlet(wl, rin), wl.rho_out, wl.tau, wl.steps)
    _, u_w = O.macroscopic(wl.q, m, want)
    assert rel(u.cpu().numpy(), u_w) < 1e-4
