"""The D2Q9 MRT collision (Eq. 16-18, lbm_set_collision) on the GPU against
the oracle: one step from a random state, the gradient through a whole sweep,
both layouts and precisions, and the BGK special case.  Tolerances as in the
main parity tests."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RATES = (1.64, 1.54, 1.9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


@pytest.fixture(autouse=True)
def _oracle_bgk():
    yield
    O.set_collision(O.COLL_BGK)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


GEOM = dict(kind=1, seed=61, r_min=3, r_max=6, target_porosity=0.72)


def test_set_collision_checks_its_arguments():
    s = lbm.Solver(9, 32, 16, precision=8, geometry=dict(kind=0))
    assert lbm.lbm_get_collision(s.plan)[0] == lbm.LBM_COLLISION_BGK
    s.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    mode, rates = lbm.lbm_get_collision(s.plan)
    assert mode == lbm.LBM_COLLISION_MRT and np.allclose(rates, RATES, rtol=1e-6)
    for bad in ((2.5, 1.0, 1.0), (1.0, 0.0, 1.0)):
        with pytest.raises(lbm.LBMError) as e:
            s.set_collision(lbm.LBM_COLLISION_MRT, *bad)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    s3 = lbm.Solver(19, 16, 8, 8, precision=8, geometry=dict(kind=0))
    with pytest.raises(lbm.LBMError) as e:
        s3.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("layout", ["dense", "compact"])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_steps_from_random_state(precision, layout, nsteps):
    nx, ny = 150, 37
    s = lbm.Solver(9, nx, ny, precision=precision, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=GEOM, layout=layout)
    s.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    m = s.mask_field.cpu().numpy()
    fs = W.perturbation((9,) + m.shape, seed=62, scale=2e-3)
    fs[:, m.astype(bool)] = 0
    rin = 1.0 + 1e-3 + W.perturbation((ny,), seed=63, scale=5e-4)
    tau = 0.7
    got = s.step(dev(rin), dev([tau]), 0.9995, dev(fs, s.plan.dtype), nsteps).cpu().numpy()
    w = O.lattice(9)[1].reshape(9, 1, 1)
    f = fs + w
    with O.collision(O.COLL_MRT, *RATES):
        for _ in range(nsteps):
            f = O.step(9, m, f, rin, 0.9995, tau)
    fl = ~m.astype(bool)
    assert rel(got[:, fl], (f - w)[:, fl]) < (1e-11 if precision == 8 else 2e-5)


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("layout", ["dense", "compact"])
@pytest.mark.parametrize("stride", [0, 7])
def test_gradient_matches_oracle(precision, layout, stride):
    nx, ny, T = 140, 33, 40
    s = lbm.Solver(9, nx, ny, precision=precision, n_steps=T, ckpt_stride=stride,
                   inlet_kind=lbm.LBM_INLET_PROFILE, geometry=GEOM, layout=layout)
    s.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    m = s.mask_field.cpu().numpy()
    rin = 1.0 + W.inlet_profile(ny, seed=64)
    tau = 0.7
    ut = W.perturbation((2,) + m.shape, seed=65, scale=1e-3)
    f = s.forward(dev(rin), dev([tau]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([tau]), 1.0, lam)
    with O.collision(O.COLL_MRT, *RATES):
        Lw, g_in_w, g_tau_w = O.gradient(9, m, rin, 1.0, tau, T, ut, ckpt_stride=5)
    _, g_bgk, t_bgk = O.gradient(9, m, rin, 1.0, tau, T, ut, ckpt_stride=5)
    g = g_in.cpu().numpy()
    if precision == 8:
        assert abs(L.item() - Lw) <= 1e-10 * abs(Lw)
        assert rel(g, g_in_w) < 1e-9
        assert abs(g_tau.item() - g_tau_w) <= 1e-9 * abs(g_tau_w)
    else:
        assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
        assert rel(g, g_in_w) < 1e-3
        assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)
    # the operator acts: the result is far from BGK's
    assert abs(g_tau.item() - t_bgk) > 10 * abs(g_tau.item() - g_tau_w)


def test_equal_rates_are_bgk_and_the_kernel_choice_is_restored():
    """S = I / tau on the GPU gives BGK's forward state to rounding; setting
    BGK back restores the TMA family's result bit for bit."""
    nx, ny, T, tau = 128, 40, 50, 0.8
    s = lbm.Solver(9, nx, ny, precision=8, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=GEOM,
                   layout="dense")
    lbm.lbm_plan_set_kernels(s.plan, step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA)
    rin = dev(1.0 + W.inlet_profile(ny, seed=66))
    bgk = s.forward(rin, dev([tau]), 1.0).clone()
    s.set_collision(lbm.LBM_COLLISION_MRT, 1 / tau, 1 / tau, 1 / tau)
    mrt = s.forward(rin, dev([tau]), 1.0).clone()
    s.set_collision(lbm.LBM_COLLISION_BGK)
    back = s.forward(rin, dev([tau]), 1.0)
    fl = torch.as_tensor(~s.mask_field.cpu().numpy().astype(bool), device="cuda")
    assert rel(mrt[:, fl].cpu().numpy(), bgk[:, fl].cpu().numpy()) < 1e-12
    assert torch.equal(bgk[:, fl], back[:, fl])
