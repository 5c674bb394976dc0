"""Cubic-spline inlet profiles on the GPU (lbm_spline_profile / lbm_spline_grad)
against the spline oracle, the chain rule through a whole gradient
evaluation, and an L-BFGS inversion of the knot values."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import spline_oracle as S
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


@pytest.mark.parametrize("q,nx,ny,nz,ky,kz", [(9, 40, 64, 1, 8, 1), (9, 16, 37, 1, 37, 1), (19, 24, 20, 12, 5, 3),
                                              (19, 16, 9, 7, 1, 7)])
def test_profile_and_gradient_match_the_oracle(q, nx, ny, nz, ky, kz):
    s = lbm.Solver(q, nx, ny, nz, precision=8, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=dict(kind=0))
    by, bz = lbm.lbm_spline_basis(ky, ny), lbm.lbm_spline_basis(kz, nz)
    r = np.random.Generator(np.random.PCG64(ky * 100 + kz))
    c = r.normal(0, 1e-3, (kz, ky))
    rho = torch.zeros(ny * nz, dtype=torch.float64, device="cuda")
    s.run(lambda: lbm.lbm_spline_profile(s.plan, dev(by), dev(bz), dev(c), 1.0, rho))
    np.testing.assert_allclose(rho.cpu().numpy().reshape(nz, ny), S.profile(c, ny, nz, 1.0), rtol=0, atol=1e-15)
    g = r.normal(size=(nz, ny))
    gc = torch.zeros(ky * kz, dtype=torch.float64, device="cuda")
    s.run(lambda: lbm.lbm_spline_grad(s.plan, dev(by), dev(bz), dev(g), gc))
    np.testing.assert_allclose(gc.cpu().numpy().reshape(kz, ky), S.grad(g, ky, kz, ny, nz), rtol=1e-13, atol=1e-13)


def test_rejects_a_constant_head_plan_and_too_many_knots():
    s = lbm.Solver(9, 16, 8, precision=8, inlet_kind=lbm.LBM_INLET_CONST, geometry=dict(kind=0))
    by, bz = dev(lbm.lbm_spline_basis(4, 8)), dev(np.ones((1, 1)))
    rho = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_spline_profile(s.plan, by, bz, dev(np.zeros(4)), 1.0, rho)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    s = lbm.Solver(9, 16, 8, precision=8, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=dict(kind=0))
    with pytest.raises(lbm.LBMError):
        lbm.lbm_spline_profile(s.plan, dev(np.zeros((8, 9))), bz, dev(np.zeros(9)), 1.0, rho)


def test_knot_gradient_through_a_whole_evaluation():
    """dL/dc = B^T dL/drho_in: the GPU chain (spline profile, forward, loss,
    adjoint, spline gradient) against the oracle's gradient and B^T."""
    q, nx, ny, T, ky = 9, 80, 33, 60, 6
    s = lbm.Solver(q, nx, ny, precision=8, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE,
                   geometry=dict(kind=1, seed=81, r_min=3, r_max=5, target_porosity=0.75))
    m = s.mask_field.cpu().numpy()
    by, bz = dev(lbm.lbm_spline_basis(ky, ny)), dev(np.ones((1, 1)))
    c = np.array([1.0, 1.4, 0.7, 1.2, 0.9, 1.1]) * 1e-3
    rho = torch.zeros(ny, dtype=torch.float64, device="cuda")
    ut = W.perturbation((2,) + m.shape, seed=82, scale=1e-3)
    tau = dev([0.8])
    s.run(lambda: lbm.lbm_spline_profile(s.plan, by, bz, dev(c), 1.0, rho))
    f = s.forward(rho, tau, 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, _ = s.adjoint(rho, tau, 1.0, lam)
    gc = torch.zeros(ky, dtype=torch.float64, device="cuda")
    s.run(lambda: lbm.lbm_spline_grad(s.plan, by, bz, g_in, gc))
    rin = S.profile(c[None, :], ny, 1, 1.0)[0]
    Lw, gw, _ = O.gradient(q, m, rin, 1.0, 0.8, T, ut, ckpt_stride=8)
    want = S.grad(gw, ky, 1, ny, 1)[0]
    assert abs(L.item() - Lw) <= 1e-10 * Lw
    np.testing.assert_allclose(gc.cpu().numpy(), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_lbfgs_recovers_spline_knots():
    """A spline truth profile (8 knots) is recovered to 1e-3 relative error by
    inverting the 8 knot values instead of the 128 node densities."""
    q, nx, ny, T, ky = 9, 128, 128, 3000, 8
    s = lbm.Solver(q, nx, ny, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE,
                   geometry=dict(kind=1, seed=91, r_min=6, r_max=10, target_porosity=0.65))
    r = np.random.Generator(np.random.PCG64(92))
    c_true = 1e-3 * (1.0 + 0.4 * r.uniform(-1, 1, ky))
    by = lbm.lbm_spline_basis(ky, ny)
    delta_true = by @ c_true
    rho_true = dev(1.0 + delta_true)
    f = s.forward(rho_true, dev([0.8]), 1.0)
    _, u = s.macroscopic(f)
    inv = I.Inversion(s, u.contiguous(), 1.0, tau0=0.8, spline=(ky, 1))
    res = inv.run_lbfgs(max_evals=60, tol=1e-3, truth_delta=delta_true)
    assert res.converged, res.err_history[-3:]
    assert inv.evaluations <= 40
    assert np.linalg.norm(res.rho_in - 1.0 - delta_true) / np.linalg.norm(delta_true) <= 1e-3
