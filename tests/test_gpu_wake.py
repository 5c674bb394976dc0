"""The cylinder-wake options on the GPU (fluid-only layout): periodic top and
bottom and the velocity inlet, with BGK and MRT, against the oracle; the
exact uniform-flow fixed point; and a viscosity inversion from a downstream
velocity snapshot (section 3.4)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import invert as I
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
def _oracle_defaults():
    yield
    O.set_periodic_y(False)
    O.set_velocity_inlet(None)
    O.set_velocity_ramp(0)
    O.set_time(1)
    O.set_collision(O.COLL_BGK)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def cylinder(nx, ny, cx, cy, d):
    y, x = np.mgrid[0:ny, 0:nx]
    return (((x - cx) ** 2 + (y - cy) ** 2) <= (d / 2) ** 2).astype(np.uint8)


def wake_solver(m, precision, T, stride=0, mrt=True, u_in=(0.05, 0.0)):
    ny, nx = m.shape
    s = lbm.Solver(9, nx, ny, precision=precision, n_steps=T, ckpt_stride=stride, geometry=torch.as_tensor(m),
                   periodic_y=True)
    assert s.layout == "compact"
    s.set_velocity_inlet(u_in)
    if mrt:
        s.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    return s


def test_options_are_checked():
    s = wake_solver(np.zeros((8, 16), np.uint8), 8, 4)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_set_periodic_y(s.plan, True)  # after the geometry
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as e:
        s.set_velocity_inlet((0.05, 0.0, 0.01))  # u_z on a D2Q9 plan
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    s.set_velocity_inlet((0.05, 0.0))
    s.set_layout("dense")
    with pytest.raises(lbm.LBMError) as e:
        s.forward(dev([1.0]), dev([0.8]), 1.0)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("mrt", [False, True])
def test_uniform_flow_is_a_fixed_point(mrt):
    nx, ny, u = 48, 16, (0.06, 0.0)
    m = np.zeros((ny, nx), np.uint8)
    s = wake_solver(m, 8, 1, mrt=mrt, u_in=u)
    feq = O.equilibrium(9, np.ones(m.shape), np.stack([np.full(m.shape, u[0]), np.zeros(m.shape)]))
    fs = feq - O.lattice(9)[1].reshape(9, 1, 1)
    got = s.step(dev([1.0]), dev([0.7]), 1.0, dev(fs), 5).cpu().numpy()
    np.testing.assert_allclose(got, fs, rtol=0, atol=1e-15)


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("mrt", [False, True])
@pytest.mark.parametrize("stride", [0, 7])
def test_wake_gradient_matches_oracle(precision, mrt, stride):
    nx, ny, T, tau = 96, 40, 60, 0.62
    m = cylinder(nx, ny, 20, 19.5, 8)
    m[0, 20] = 1  # a solid node on y = 0 makes the wrap visible in the link words
    s = wake_solver(m, precision, T, stride, mrt)
    roi = np.zeros(m.shape, np.uint8)
    roi[8:32, 40:80] = 1
    ut = W.perturbation((2,) + m.shape, seed=71, scale=1e-3)
    f = s.forward(dev([1.0]), dev([tau]), 1.0)
    L, lam = s.loss_grad(f, dev(ut), dev(roi, torch.uint8))
    g_in, g_tau = s.adjoint(dev([1.0]), dev([tau]), 1.0, lam)
    _, u = s.macroscopic(f)
    if mrt:
        O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0)):
        Lw, _, g_tau_w, fT = O.gradient(9, m, 1.0, 1.0, tau, T, ut, roi=roi, ckpt_stride=5, return_fT=True)
    _, uw = O.macroscopic(9, m, fT)
    links = s.link.cpu().numpy().view(np.uint32).reshape(m.shape)
    with O.wake_options(periodic_y=True):
        assert np.array_equal(links, O.links(9, m))
    if precision == 8:
        assert rel(u.cpu().numpy(), uw) < 1e-11
        assert abs(L.item() - Lw) <= 1e-10 * abs(Lw)
        assert abs(g_tau.item() - g_tau_w) <= 1e-9 * abs(g_tau_w)
    else:
        assert rel(u.cpu().numpy(), uw) < 1e-4
        assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
        assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)
    assert g_in.item() == 0.0  # the velocity inlet does not use rho_in


def test_viscosity_inversion_from_a_downstream_snapshot():
    """Section 3.4's inversion on a small wake (160 x 64, D = 8, u_in = 0.08,
    MRT, T = 2000): from nu = 0.06 to the truth nu = 0.02 by L-BFGS on tau,
    against the velocity snapshot in a rectangle downstream of the cylinder."""
    nx, ny, T = 160, 64, 2000
    m = cylinder(nx, ny, 32, 31.5, 8)
    s = wake_solver(m, 8, T, u_in=(0.08, 0.0))
    nu_true = 0.02
    f = s.forward(dev([1.0]), dev([0.5 + 3 * nu_true]), 1.0)
    _, ut = s.macroscopic(f)
    roi = torch.zeros(m.shape, dtype=torch.uint8, device="cuda")
    roi[:, 48:] = 1
    tau_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    rin = dev([1.0])

    def evaluate(x):
        tau_t.fill_(0.5 + 0.1 * float(x[0]))
        fT = s.forward(rin, tau_t, 1.0)
        L, lam = s.loss_grad(fT, ut, roi)
        _, g_tau = s.adjoint(rin, tau_t, 1.0, lam)
        return L.item(), np.array([g_tau.item() * 0.1])

    res = I.lbfgs(evaluate, np.array([3 * 0.06 / 0.1]), max_evals=40, lower={0: 0.05},
                  errors=lambda x: (abs(0.1 * x[0] / 3 - nu_true) / nu_true, None), done=lambda e: e[0] < 1e-3)
    assert res.converged and res.evaluations <= 25, res.errs


def test_snapshot_series_gradient_matches_the_oracle():
    """A loss over three snapshots (steps 40, 50, 60) equals the sum of the
    oracle's single-snapshot losses, and so does its gradient."""
    nx, ny, tau = 96, 40, 0.62
    m = cylinder(nx, ny, 20, 19.5, 8)
    times = (40, 50, 60)
    targets = [W.perturbation((2,) + m.shape, seed=80 + k, scale=1e-3) for k in range(3)]
    roi = np.zeros(m.shape, np.uint8)
    roi[8:32, 40:80] = 1
    series = I.SnapshotSeries(lambda t: wake_solver(m, 8, t), times, [dev(u) for u in targets],
                              dev(roi, torch.uint8))
    L, g_in, g_tau = series.loss_and_grad(dev([1.0]), dev([tau]), 1.0)
    O.set_collision(O.COLL_MRT, *RATES)
    Lw = gw = 0.0
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0)):
        for t, ut in zip(times, targets):
            l, _, g = O.gradient(9, m, 1.0, 1.0, tau, t, ut, roi=roi, ckpt_stride=5)
            Lw, gw = Lw + l, gw + g
    assert abs(L.item() - Lw) <= 1e-10 * Lw
    assert abs(g_tau.item() - gw) <= 1e-9 * abs(gw)
    assert g_in.item() == 0.0


def test_velocity_inlet_in_a_walled_channel():
    """Without periodicity (walls at y = -1/2, ny - 1/2): the solver moves to
    the fluid-only layout when the inlet is set, and matches the oracle."""
    nx, ny, T = 64, 24, 30
    m = cylinder(nx, ny, 20, 11.5, 6)
    s = lbm.Solver(9, nx, ny, precision=8, n_steps=T, geometry=torch.as_tensor(m), layout="dense")
    s.set_velocity_inlet((0.04, 0.0))
    assert s.layout == "compact"
    _, u = s.macroscopic(s.forward(dev([1.0]), dev([0.7]), 1.0))
    with O.wake_options(periodic_y=False, velocity_inlet=(0.04, 0.0)):
        _, uw = O.macroscopic(9, m, O.forward(9, m, 1.0, 1.0, 0.7, T))
    assert rel(u.cpu().numpy(), uw) < 1e-11


# ------------------------------------- gradual start and a loss over a time window


@pytest.mark.parametrize("precision", [8, 4])
def test_ramped_wake_forward_and_gradient_match_the_oracle(precision):
    m = cylinder(64, 24, 16, 12.3, 6)
    T, R, tau = 60, 40, 0.7
    s = wake_solver(m, precision, T, stride=7)
    s.set_velocity_ramp(R)
    ut = W.perturbation((2,) + m.shape, seed=41, scale=2e-3)
    roi = np.zeros(m.shape, np.uint8)
    roi[:, 30:] = 1
    f = s.forward(dev([1.0]), dev([tau]), 1.0)
    _, u = s.macroscopic(f)
    L, lam = s.loss_grad(f, dev(ut), dev(roi, torch.uint8))
    _, g_tau = s.adjoint(dev([1.0]), dev([tau]), 1.0, lam)
    O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=R):
        _, uw = O.macroscopic(9, m, O.forward(9, m, 1.0, 1.0, tau, T))
        Lw, _, gw = O.gradient(9, m, 1.0, 1.0, tau, T, ut, roi=roi, ckpt_stride=7)
    tol_u, tol_g = (1e-11, 1e-9) if precision == 8 else (1e-4, 1e-3)
    assert rel(u.cpu().numpy(), uw) < tol_u
    assert abs(L.item() - Lw) <= tol_u * abs(Lw)
    assert abs(g_tau.item() - gw) <= tol_g * abs(gw)
    # the ramp changes the flow (a check that it is applied at all)
    s0 = wake_solver(m, precision, T, stride=7)
    _, u0 = s0.macroscopic(s0.forward(dev([1.0]), dev([tau]), 1.0))
    assert rel(u0.cpu().numpy(), uw) > 1e-2


WINDOW = [(True, 8), (True, 4), (False, 8), (False, 4)]


@pytest.mark.parametrize("wake,precision", WINDOW, ids=[f"{'wake' if w else 'pressure'}-fp{8 * p}" for w, p in WINDOW])
def test_window_loss_gradient_matches_the_oracle(wake, precision):
    """One reverse sweep of lbm_adjoint_window against the oracle's window
    gradient: observations inside segments, on a segment boundary and at T."""
    T, stride, tau = 48, 7, 0.75
    obs = [14, 21, 33, 48]
    if wake:
        m = cylinder(64, 24, 16, 12.3, 6)
        s = wake_solver(m, precision, T, stride=stride)
        s.set_velocity_ramp(30)
        rin = np.array([1.0])
        opts = dict(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=30)
        O.set_collision(O.COLL_MRT, *RATES)
    else:
        g = dict(kind=lbm.LBM_GEOM_DISKS, seed=12, r_min=3, r_max=5, target_porosity=0.75, inlet_buffer=4)
        s = lbm.Solver(9, 72, 32, precision=precision, n_steps=T, ckpt_stride=stride,
                       inlet_kind=lbm.LBM_INLET_PROFILE, geometry=g, layout="dense")
        m = s.mask_field.cpu().numpy()
        rin = 1.0 + W.inlet_profile(32, seed=13)
        opts = {}
    ut = W.perturbation((len(obs), 2) + m.shape, seed=42, scale=2e-3)
    roi = np.ones(m.shape, np.uint8)
    roi[:, :10] = 0
    f = s.forward(dev(rin), dev([tau]), 1.0)
    L, g_in, g_tau = s.adjoint_window(dev(rin), dev([tau]), 1.0, f, obs, dev(ut), dev(roi, torch.uint8))
    assert s.status() == lbm.LBM_OK
    with O.wake_options(**opts):
        Lw, gw, gtw = O.gradient_window(9, m, rin if rin.size > 1 else rin[0], 1.0, tau, T, obs, ut, roi=roi,
                                        ckpt_stride=stride)
    tol_l, tol_g = (1e-11, 1e-9) if precision == 8 else (1e-4, 1e-3)
    assert abs(L.item() - Lw) <= tol_l * abs(Lw)
    assert abs(g_tau.item() - gtw) <= tol_g * abs(gtw)
    if not wake:
        assert rel(g_in.cpu().numpy(), gw) < tol_g


@pytest.mark.parametrize("layout", ["dense", "compact"])
def test_window_with_one_observation_at_T_is_the_adjoint_bit_for_bit(layout):
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=14, r_min=3, r_max=5, target_porosity=0.75, inlet_buffer=4)
    s = lbm.Solver(9, 72, 32, precision=4, n_steps=30, ckpt_stride=6, inlet_kind=lbm.LBM_INLET_PROFILE,
                   geometry=g, layout=layout)
    rin = dev(1.0 + W.inlet_profile(32, seed=15))
    ut = dev(W.perturbation((1, 2, 32, 72), seed=16, scale=2e-3))
    f = s.forward(rin, dev([0.8]), 1.0)
    L, lam = s.loss_grad(f, ut[0])
    g_in, g_tau = s.adjoint(rin, dev([0.8]), 1.0, lam)
    Lw, g_in_w, g_tau_w = s.adjoint_window(rin, dev([0.8]), 1.0, f, [30], ut)
    assert Lw.item() == L.item()
    assert torch.equal(g_in_w, g_in) and torch.equal(g_tau_w, g_tau)


def test_window_rejects_steps_outside_the_sweep():
    s = wake_solver(cylinder(32, 16, 8, 8.3, 4), 8, 10)
    f = s.forward(dev([1.0]), dev([0.8]), 1.0)
    ut = dev(np.zeros((1, 2, 16, 32)))
    for bad in ([0], [11]):
        with pytest.raises(lbm.LBMError) as e:
            s.adjoint_window(dev([1.0]), dev([0.8]), 1.0, f, bad, ut)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG
