"""In-place (AA-pattern) streaming in the fluid-only layout: the forward
sweep, lbm_step and the reverse sweep on one state buffer (and one lambda
buffer), against the two-buffer pull of the same plan and against the FP64
oracle, on D2Q9 and D3Q19, FP32 and FP64, pressure (Eq. 6, constant head and
profile) and wake boundaries (periodic y, velocity inlet with its ramp,
MRT), odd and even T and checkpoint strides, with and without the
overlapped recompute; the window loss; and the workspace and option checks.

Each node runs the same arithmetic in both schedules (only the addresses of
its loads and stores differ), so the two schedules agree bit for bit."""
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


def _set(s, aa, overlap=1):
    s.set_kernels(aa=aa, overlap=overlap)
    assert lbm.lbm_plan_get_kernels(s.plan)["aa"] == aa


def _porous(q, precision, T, stride, profile, seed=3):
    if q == 9:
        g = dict(kind=lbm.LBM_GEOM_DISKS, seed=seed, r_min=3, r_max=6, target_porosity=0.7, inlet_buffer=4)
        s = lbm.Solver(9, 150, 37, precision=precision, n_steps=T, ckpt_stride=stride, geometry=g,
                       inlet_kind=lbm.LBM_INLET_PROFILE if profile else lbm.LBM_INLET_CONST, layout="compact")
    else:
        g = dict(kind=lbm.LBM_GEOM_SPHERES, seed=seed, r_min=3, r_max=3, target_porosity=0.7, inlet_buffer=3)
        s = lbm.Solver(19, 44, 18, 14, precision=precision, n_steps=T, ckpt_stride=stride, geometry=g,
                       inlet_kind=lbm.LBM_INLET_PROFILE if profile else lbm.LBM_INLET_CONST, layout="compact")
    assert s.layout == "compact"
    return s


def _inlet(s, seed):
    n_in = s.plan.n_in
    return 1.0 + (W.inlet_profile(n_in, seed=seed) if n_in > 1 else np.array([2e-3]))


def _gradient(s, rin, tau, ut):
    f = s.forward(dev(rin), dev([tau]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([tau]), 1.0, lam)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_OK
    return f, L, g_in, g_tau


CASES = [  # q, precision, T, stride, profile
    (9, 4, 41, 6, True), (9, 4, 40, 7, False), (9, 8, 33, 5, True), (9, 8, 32, 0, False),
    (19, 4, 25, 4, True), (19, 4, 24, 5, False), (19, 8, 21, 6, True),
]


@pytest.mark.parametrize("q,precision,T,stride,profile", CASES)
@pytest.mark.parametrize("overlap", [1, 0])
def test_in_place_gradient_equals_the_two_buffer_pull(q, precision, T, stride, profile, overlap):
    s = _porous(q, precision, T, stride, profile)
    rin = _inlet(s, 5)
    ut = W.perturbation((s.plan.d, *s.plan.shape), seed=6, scale=1e-4)
    _set(s, 0, overlap)
    ref = _gradient(s, rin, 0.8, ut)
    _set(s, 1, overlap)
    got = _gradient(s, rin, 0.8, ut)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


@pytest.mark.parametrize("q,precision,T,stride,profile", [CASES[0], CASES[1], CASES[4], CASES[6]])
def test_in_place_gradient_matches_the_oracle(q, precision, T, stride, profile):
    s = _porous(q, precision, T, stride, profile)
    _set(s, 1)
    m = s.mask_field.cpu().numpy()
    rin = _inlet(s, 5)
    ut = W.perturbation((s.plan.d, *s.plan.shape), seed=6, scale=1e-4)
    f, L, g_in, g_tau = _gradient(s, rin, 0.8, ut)
    k = stride if stride else int(np.ceil(np.sqrt(T)))
    r = rin if rin.size > 1 else rin[0]
    Lw, gw, gtw, fw = O.gradient(q, m, r, 1.0, 0.8, T, ut, ckpt_stride=k, return_fT=True)
    _, u = s.macroscopic(f)
    _, uw = O.macroscopic(q, m, fw)
    tol_u, tol_g = (1e-11, 1e-9) if precision == 8 else (1e-4, 1e-3)
    assert rel(u.cpu().numpy(), uw) < tol_u
    assert abs(L.item() - Lw) <= tol_u * abs(Lw)
    assert rel(g_in.cpu().numpy(), gw) < tol_g
    assert abs(g_tau.item() - gtw) <= tol_g * abs(gtw)


@pytest.mark.parametrize("q,precision", [(9, 4), (19, 8)])
@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_in_place_step_equals_the_two_buffer_pull(q, precision, n):
    s = _porous(q, precision, 1, 0, True)
    rin = dev(_inlet(s, 7))
    f0 = W.perturbation((q, *s.plan.shape), seed=8, scale=2e-3)
    f0[:, s.mask_field.cpu().numpy() == 1] = 0.0
    f0 = dev(f0, s.plan.dtype)
    _set(s, 0)
    ref = s.step(rin, dev([0.75]), 1.0, f0, n)
    _set(s, 1)
    got = s.step(rin, dev([0.75]), 1.0, f0, n)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def _cylinder(nx, ny, cx, cy, d):
    y, x = np.mgrid[0:ny, 0:nx]
    return (((x - cx) ** 2 + (y - cy) ** 2) <= (d / 2) ** 2).astype(np.uint8)


@pytest.mark.parametrize("precision", [4, 8])
def test_in_place_wake_with_ramp_and_window(precision):
    """Periodic y, velocity inlet with its gradual start, MRT: forward,
    adjoint and the window loss, in place against the two-buffer pull and
    against the oracle's window gradient."""
    m = _cylinder(64, 24, 16, 12.3, 6)
    T, stride, tau, R = 47, 7, 0.75, 30
    obs = [13, 21, 34, 47]
    s = lbm.Solver(9, 64, 24, precision=precision, n_steps=T, ckpt_stride=stride, geometry=torch.as_tensor(m),
                   periodic_y=True)
    s.set_velocity_inlet((0.05, 0.0))
    s.set_velocity_ramp(R)
    s.set_collision(lbm.LBM_COLLISION_MRT, *RATES)
    ut = W.perturbation((len(obs), 2) + m.shape, seed=42, scale=2e-3)
    roi = np.ones(m.shape, np.uint8)
    roi[:, :10] = 0
    out = []
    for aa in (0, 1):
        _set(s, aa)
        f = s.forward(dev([1.0]), dev([tau]), 1.0)
        L, lam = s.loss_grad(f, dev(ut[-1]), dev(roi, torch.uint8))
        _, g_tau = s.adjoint(dev([1.0]), dev([tau]), 1.0, lam)
        Lw, _, gw = s.adjoint_window(dev([1.0]), dev([tau]), 1.0, f, obs, dev(ut), dev(roi, torch.uint8))
        torch.cuda.synchronize()
        out.append((f, L, g_tau, Lw, gw))
    for a, b in zip(out[1], out[0]):
        assert torch.equal(a, b)
    O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=R):
        Lo, _, go = O.gradient_window(9, m, 1.0, 1.0, tau, T, obs, ut, roi=roi, ckpt_stride=stride)
    tol_l, tol_g = (1e-11, 1e-9) if precision == 8 else (1e-4, 1e-3)
    assert abs(out[1][3].item() - Lo) <= tol_l * abs(Lo)
    assert abs(out[1][4].item() - go) <= tol_g * abs(go)


def test_in_place_workspace_holds_two_states_fewer():
    s = _porous(19, 4, 30, 0, False)
    p = s.plan
    _set(s, 0)
    two = lbm.lbm_workspace_size(p)
    _set(s, 1)
    one = lbm.lbm_workspace_size(p)
    state = -(-p.q * s.n_fluid * p.precision // 256) * 256
    assert two - one == 2 * state
    # a solver sized for the in-place schedule grows its workspace back when it is cleared
    s.ws = torch.zeros(one, dtype=torch.uint8, device="cuda")
    _set(s, 0)
    assert s.ws.numel() == two


def test_in_place_needs_a_forward_of_the_same_schedule():
    s = _porous(9, 4, 20, 0, False)
    _set(s, 1)
    f = s.forward(dev([1.002]), dev([0.8]), 1.0)
    _, lam = s.loss_grad(f, dev(np.zeros((2, *s.plan.shape))))
    lbm.lbm_plan_set_kernels(s.plan, aa=0)  # the checkpoints are in the in-place layouts
    with pytest.raises(lbm.LBMError) as e:
        s.adjoint(dev([1.002]), dev([0.8]), 1.0, lam)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG


def test_in_place_refuses_the_extrapolated_wall_velocity():
    s = _porous(9, 4, 10, 0, False)
    _set(s, 1)
    lbm.lbm_set_abb_velocity(s.plan, lbm.LBM_ABB_U_EXTRAP)
    with pytest.raises(lbm.LBMError) as e:
        s.forward(dev([1.002]), dev([0.8]), 1.0)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


def test_in_place_is_ignored_by_the_dense_layout():
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=4, r_min=3, r_max=6, target_porosity=0.7, inlet_buffer=4)
    s = lbm.Solver(9, 128, 32, precision=4, n_steps=30, geometry=g, layout="dense")
    _set(s, 0)
    size = lbm.lbm_workspace_size(s.plan)
    ref = s.forward(dev([1.002]), dev([0.8]), 1.0)
    _set(s, 1)
    assert lbm.lbm_workspace_size(s.plan) == size
    got = s.forward(dev([1.002]), dev([0.8]), 1.0)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
