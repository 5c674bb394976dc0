"""Parity of the two optional terms with the oracle, through the C ABI: Eq. 6
with the wall velocity extrapolated to the pressure plane (lbm_set_abb_velocity)
and the density-probe loss (lbm_probe_loss_grad).  Tolerances are those of the
main parity tests: FP64 to rounding, FP32 1e-4 on velocity and 1e-3 on
gradients."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


@pytest.fixture(autouse=True)
def _oracle_node_velocity():
    yield
    O.set_abb_velocity(O.UW_NODE)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _case(q):
    """Packings with solid nodes right behind the inlet / outlet in a few rows
    (those rows keep the node velocity) and just beyond them (strong x
    gradients where the extrapolation matters)."""
    if q == 9:
        nx, ny, nz = 96, 29, 1
        m, _ = O.geometry(9, nx, ny, kind=O.GEOM_DISKS, seed=51, r_min=3, r_max=6, porosity=0.75, buffer=3)
        m = m.copy()
        m[3, 1] = m[10, nx - 2] = m[20, 2] = m[21, 2] = 1
    else:
        nx, ny, nz = 48, 11, 9
        m, _ = O.geometry(19, nx, ny, nz, kind=O.GEOM_SPHERES, seed=51, r_min=2, r_max=2, porosity=0.8, buffer=3)
        m = m.copy()
        m[2, 3, 1] = m[4, 5, nx - 2] = m[6, 6, 2] = 1
    return nx, ny, nz, m


def _solver(q, m, precision, T, stride, layout, profile):
    nz, ny, nx = (1,) + m.shape if q == 9 else m.shape
    return lbm.Solver(q, nx, ny, nz, precision=precision, n_steps=T, ckpt_stride=stride,
                      inlet_kind=lbm.LBM_INLET_PROFILE if profile else lbm.LBM_INLET_CONST,
                      geometry=torch.as_tensor(m), layout=layout)


def test_set_abb_velocity_checks_and_reports():
    s = _solver(9, np.zeros((8, 16), np.uint8), 8, 4, 0, "dense", False)
    assert lbm.lbm_get_abb_velocity(s.plan) == lbm.LBM_ABB_U_NODE
    s.set_abb_velocity(lbm.LBM_ABB_U_EXTRAP)
    assert lbm.lbm_get_abb_velocity(s.plan) == lbm.LBM_ABB_U_EXTRAP
    with pytest.raises(lbm.LBMError) as e:
        s.set_abb_velocity(2)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_get_abb_velocity(s.plan) == lbm.LBM_ABB_U_EXTRAP


@pytest.mark.parametrize("q,T", [(9, 40), (19, 12)])
@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("layout", ["dense", "compact"])
@pytest.mark.parametrize("stride", [0, 3])
def test_extrapolated_abb_gradient_matches_oracle(q, T, precision, layout, stride):
    nx, ny, nz, m = _case(q)
    profile = q == 9
    s = _solver(q, m, precision, T, stride, layout, profile)
    s.set_abb_velocity(lbm.LBM_ABB_U_EXTRAP)
    n_in = ny * nz if profile else 1
    rin = 1.0 + (W.inlet_profile(n_in, seed=42) if profile else np.array([1.2e-3]))
    tau = 0.85
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + m.shape, seed=43, scale=1e-3)
    f = s.forward(dev(rin), dev([tau]), 1.0)
    _, u = s.macroscopic(f)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([tau]), 1.0, lam)
    rin_o = rin.reshape((nz, ny) if q == 19 else (ny,)) if profile else rin[0]
    with O.abb_velocity(O.UW_EXTRAP):
        Lw, g_in_w, g_tau_w, fT = O.gradient(q, m, rin_o, 1.0, tau, T, ut, ckpt_stride=5, return_fT=True)
    _, uw = O.macroscopic(q, m, fT)
    _, g_node, _ = O.gradient(q, m, rin_o, 1.0, tau, T, ut, ckpt_stride=5)
    g = g_in.cpu().numpy()
    if precision == 8:
        assert rel(u.cpu().numpy(), uw) < 1e-11
        assert abs(L.item() - Lw) <= 1e-10 * abs(Lw)
        assert rel(g, np.ravel(g_in_w)) < 1e-9
        assert abs(g_tau.item() - g_tau_w) <= 1e-9 * abs(g_tau_w)
    else:
        assert rel(u.cpu().numpy(), uw) < 1e-4
        assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
        assert rel(g, np.ravel(g_in_w)) < 1e-3
        assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)
    # the setting acts: the result is much closer to the extrapolated oracle than to the node-velocity one
    assert rel(g, np.ravel(g_in_w)) < 0.5 * rel(g, np.ravel(g_node))


def test_extrapolated_abb_overrides_the_kernel_choice():
    """The dense layout runs the one-node-per-thread kernels whatever family
    was chosen (TMA / register-vector / persistent), and switching back to the
    node velocity restores the chosen family's result."""
    q, T = 9, 30
    nx, ny, nz, m = _case(q)
    m = m[:, :64].copy()  # nx = 64: every kernel family applies
    s = _solver(q, m, 4, T, 0, "dense", True)
    lbm.lbm_plan_set_kernels(s.plan, step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA)
    rin = 1.0 + W.inlet_profile(ny, seed=44)
    node = s.forward(dev(rin), dev([0.8]), 1.0).clone()
    s.set_abb_velocity(lbm.LBM_ABB_U_EXTRAP)
    ext = s.forward(dev(rin), dev([0.8]), 1.0).clone()
    s.set_abb_velocity(lbm.LBM_ABB_U_NODE)
    back = s.forward(dev(rin), dev([0.8]), 1.0)
    with O.abb_velocity(O.UW_EXTRAP):
        want = O.forward(q, m, rin, 1.0, 0.8, T)
    _, u = s.macroscopic(ext)
    _, uw = O.macroscopic(q, m, want)
    assert rel(u.cpu().numpy(), uw) < 1e-4
    fl = torch.as_tensor(~m.astype(bool), device="cuda")  # solid entries are not written
    assert torch.equal(node[:, fl], back[:, fl]) and not torch.equal(node[:, fl], ext[:, fl])


# ------------------------------------------------------------- density probes


def _probes(m, n, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    fluid = np.flatnonzero(m.reshape(-1) == 0)
    nodes = r.choice(fluid, size=n, replace=False).astype(np.int64)
    return nodes, 1.0 + r.normal(0, 5e-4, n)


@pytest.mark.parametrize("q", [9, 19])
def test_probe_seed_matches_oracle(q):
    nx, ny, nz, m = _case(q)
    s = _solver(q, m, 8, 1, 0, "dense", False)
    fs = W.perturbation((q,) + m.shape, seed=61, scale=2e-3)
    fs[:, m.astype(bool)] = 0
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + m.shape, seed=62, scale=3e-3)
    nodes, rt = _probes(m, 40, 63)
    nodes[-1] = nodes[0]  # a repeated probe: both seeds add
    L, lam = s.loss_grad(dev(fs), dev(ut))
    s.probe_loss_grad(dev(fs), dev(nodes, torch.int64), dev(rt), 7.0, L, lam)
    f = fs + O.lattice(q)[1].reshape((q,) + (1,) * m.ndim)
    Lv, lamv = O.loss(q, m, f, ut)
    Lp, lamp = O.probe_loss(q, m, f, nodes, rt, 7.0)
    assert abs(L.item() - (Lv + Lp)) <= 1e-12 * (Lv + Lp)
    assert rel(lam.cpu().numpy(), lamv + lamp) < 1e-12


@pytest.mark.parametrize("q,T", [(9, 40), (19, 12)])
@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("layout", ["dense", "compact"])
def test_gradient_with_probes_matches_oracle(q, T, precision, layout):
    nx, ny, nz, m = _case(q)
    s = _solver(q, m, precision, T, 0, layout, False)
    rin, tau = 1.0 + 1.2e-3, 0.85
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + m.shape, seed=71, scale=1e-3)
    nodes, rt = _probes(m, 25, 72)
    w = 40.0
    f = s.forward(dev([rin]), dev([tau]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    s.probe_loss_grad(f, dev(nodes, torch.int64), dev(rt), w, L, lam)
    g_in, g_tau = s.adjoint(dev([rin]), dev([tau]), 1.0, lam)
    Lw, g_in_w, g_tau_w = O.gradient(q, m, rin, 1.0, tau, T, ut, ckpt_stride=5, probes=(nodes, rt, w))
    _, g_in_v, _ = O.gradient(q, m, rin, 1.0, tau, T, ut, ckpt_stride=5)
    tol = 1e-9 if precision == 8 else 1e-3
    assert abs(L.item() - Lw) <= (1e-10 if precision == 8 else 1e-4) * abs(Lw)
    assert abs(g_in.item() - g_in_w) <= tol * abs(g_in_w)
    assert abs(g_tau.item() - g_tau_w) <= tol * abs(g_tau_w)
    assert abs(g_in_w - g_in_v) > 10 * tol * abs(g_in_w)  # the probes change the gradient


def test_probe_out_of_range_is_latched_and_skipped():
    q = 9
    _, _, _, m = _case(q)
    s = _solver(q, m, 8, 1, 0, "dense", False)
    f = torch.zeros((q, *m.shape), dtype=torch.float64, device="cuda")
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(f)
    s.status()  # clear
    s.probe_loss_grad(f, dev([m.size], torch.int64), dev([1.5]), 1.0, L, lam)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_ERR_INVALID_ARG
    assert L.item() == 0.0 and not torch.any(lam)
    # no probes: nothing added, nothing latched
    s.probe_loss_grad(f, None, None, 1.0, L, lam)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_OK and L.item() == 0.0
