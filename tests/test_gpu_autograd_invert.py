"""torch.autograd wiring of the adjoint, and the inversion driver, on the GPU."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import autograd as A
from paper_2310_00810_gb300 import invert as I
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("profile", [False, True])
def test_autograd_backward_matches_oracle(profile):
    nx, ny, T = 96, 28, 60
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=51, r_min=3, r_max=6, target_porosity=0.72)
    s = lbm.Solver(9, nx, ny, precision=8, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE if profile else 0, geometry=g)
    m = s.mask_field.cpu().numpy()
    rin0 = 1.0 + (W.inlet_profile(ny, seed=52) if profile else np.array([1.1e-3]))
    ut = W.perturbation((2, ny, nx), seed=53, scale=1e-3)
    rho_in = dev(rin0).requires_grad_(True)
    tau = dev([0.85]).requires_grad_(True)
    loss = A.lbm_loss(rho_in, tau, s, 1.0, dev(ut))
    (3.0 * loss).sum().backward()
    Lw, g_in, g_tau = O.gradient(9, m, rin0 if profile else rin0[0], 1.0, 0.85, T, ut, ckpt_stride=8)
    assert abs(loss.item() - Lw) <= 1e-10 * Lw
    np.testing.assert_allclose(rho_in.grad.cpu().numpy(), 3.0 * np.ravel(g_in), rtol=1e-9, atol=0)
    assert abs(tau.grad.item() - 3.0 * g_tau) <= 1e-9 * abs(g_tau)


def test_autograd_gradcheck_fp64():
    """torch's own finite-difference check of the hand-written backward."""
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=54, r_min=2, r_max=4, target_porosity=0.75)
    s = lbm.Solver(9, 40, 16, precision=8, n_steps=25, geometry=g)
    ut = dev(W.perturbation((2, 16, 40), seed=55, scale=1e-3))
    rho_in = dev([1.0015]).requires_grad_(True)
    tau = dev([0.9]).requires_grad_(True)
    fn = lambda r, t: A.lbm_loss(r, t, s, 1.0, ut)
    assert torch.autograd.gradcheck(fn, (rho_in, tau), eps=1e-6, atol=1e-12, rtol=1e-4)


def test_inversion_recovers_constant_head():
    """Single-parameter inversion (the paper's constant inlet pressure cases):
    from delta = 0 to 1e-3 relative error on delta."""
    nx, ny, T = 128, 48, 600
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=56, r_min=3, r_max=7, target_porosity=0.7)
    s = lbm.Solver(9, nx, ny, precision=4, n_steps=T, geometry=g)
    truth = 1.3e-3
    f = s.forward(dev([1.0 + truth]), dev([0.8]), 1.0)
    _, ut = s.macroscopic(f)
    inv = I.Inversion(s, ut, 1.0, theta0=0.0, tau0=0.8, lr=0.1)
    res = inv.run(max_iters=300, tol=1e-3, truth_delta=truth)
    assert res.converged, (res.iterations, res.rel_err_inlet)
    assert abs(res.rho_in[0] - 1.0 - truth) <= 1e-3 * truth


def test_inversion_profile_reduces_error():
    """Multi-parameter (profile) inversion with Adam lowers the profile error (slowly: the profile is
    ill-conditioned, as the paper also reports for its profile case)."""
    nx, ny, T = 96, 24, 500
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=57, r_min=3, r_max=5, target_porosity=0.72)
    s = lbm.Solver(9, nx, ny, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=g)
    truth = W.inlet_profile(ny, seed=58)
    f = s.forward(dev(1.0 + truth), dev([0.8]), 1.0)
    _, ut = s.macroscopic(f)
    inv = I.Inversion(s, ut, 1.0, tau0=0.8, lr=0.05)
    res = inv.run(max_iters=150, tol=1e-3, truth_delta=truth)
    assert res.err_history[-1][0] < 0.9 * res.err_history[0][0]


def test_lbfgs_inverts_profile_to_1e3():
    """The same profile problem with L-BFGS reaches 1e-3 relative error."""
    nx, ny, T = 96, 24, 500
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=57, r_min=3, r_max=5, target_porosity=0.72)
    s = lbm.Solver(9, nx, ny, precision=8, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=g)
    truth = W.inlet_profile(ny, seed=58)
    f = s.forward(dev(1.0 + truth), dev([0.8]), 1.0)
    _, ut = s.macroscopic(f)
    inv = I.Inversion(s, ut, 1.0, tau0=0.8)
    res = inv.run_lbfgs(max_evals=120, tol=1e-3, truth_delta=truth)
    assert res.converged, (res.iterations, res.rel_err_inlet)


def test_lbfgs_joint_head_and_tau():
    """Joint constant head + tau (the 3D case's parameters, here on a small
    D3Q19 duct): the identifiable ratio delta / nu is recovered."""
    g = dict(kind=lbm.LBM_GEOM_SPHERES, seed=59, r_min=3, r_max=3, target_porosity=0.6, inlet_buffer=4)
    s = lbm.Solver(19, 48, 20, 20, precision=8, n_steps=300, geometry=g)
    d_true, tau_true = 1e-3, 0.8
    f = s.forward(dev([1.0 + d_true]), dev([tau_true]), 1.0)
    _, ut = s.macroscopic(f)
    inv = I.Inversion(s, ut, 1.0, theta0=0.5, tau0=1.0, invert_tau=True)
    res = inv.run_lbfgs(max_evals=80, tol=1e-3, truth_delta=d_true, truth_tau=tau_true)
    ratio = (res.rho_in[0] - 1.0) / ((res.tau - 0.5) / 3.0)
    assert abs(ratio / (d_true / ((tau_true - 0.5) / 3.0)) - 1.0) < 1e-2
    assert res.loss_history[-1] < 1e-3 * res.loss_history[0]
