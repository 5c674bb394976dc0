"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Geometry and link words must be bit-exact.  Floating point: FP64 plans must
agree with the oracle to rounding (relative L2 <= 1e-11 on populations and
velocities, 1e-9 on gradients accumulated over many steps); FP32 plans must
meet 1e-4 relative L2 on velocity and 1e-3 relative on gradients.  Populations
are compared on fluid nodes only (solid nodes carry no populations)."""
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def weights(q, nd):
    return O.lattice(q)[1].reshape((q,) + (1,) * nd)


def solver(q, nx, ny, nz=1, precision=8, T=1, stride=0, inlet=lbm.LBM_INLET_CONST, kind=lbm.LBM_LOSS_VEC,
           norm=lbm.LBM_NORM_SUM, geom=None):
    return lbm.Solver(q, nx, ny, nz, precision=precision, n_steps=T, ckpt_stride=stride, inlet_kind=inlet,
                      loss_kind=kind, loss_norm=norm, geometry=geom)


def oracle_geom(q, nx, ny, nz, g):
    kind = g.get("kind", 0)
    return O.geometry(q, nx, ny, nz, kind=kind, seed=g.get("seed", 0), r_min=g.get("r_min", 6),
                      r_max=g.get("r_max", 12), porosity=g.get("target_porosity", 1.0),
                      hydro_q8=g.get("hydro_q8", 256), buffer=g.get("inlet_buffer", 8),
                      max_rejections=g.get("max_rejections", 1_000_000), fill=g.get("fill_isolated", True))


# ------------------------------------------------------------------ geometry

GEOMS = [
    (9, 64, 32, 1, dict(kind=0)),
    (9, 200, 72, 1, dict(kind=1, seed=3, r_min=3, r_max=9, target_porosity=0.55)),
    (9, 150, 60, 1, dict(kind=1, seed=4, r_min=2, r_max=5, target_porosity=0.5, hydro_q8=230)),
    (9, 512, 256, 1, dict(kind=1, seed=1000, r_min=6, r_max=12, target_porosity=0.6)),
    (19, 40, 24, 20, dict(kind=2, seed=5, r_min=3, r_max=3, target_porosity=0.5, inlet_buffer=4)),
    (19, 128, 64, 64, dict(kind=2, seed=3000, r_min=6, r_max=6, target_porosity=0.45)),
    (19, 36, 20, 16, dict(kind=2, seed=6, r_min=3, r_max=3, target_porosity=0.1, inlet_buffer=4,
                          max_rejections=300)),  # unreachable target: stops on the no-progress streak
]


@pytest.mark.parametrize("case", GEOMS, ids=lambda c: f"q{c[0]}_{c[1]}x{c[2]}x{c[3]}_k{c[4]['kind']}")
def test_geometry_bit_exact(case):
    q, nx, ny, nz, g = case
    s = solver(q, nx, ny, nz, geom=g)
    want, info = oracle_geom(q, nx, ny, nz, g)
    got = s.mask_field.cpu().numpy()
    assert np.array_equal(got, want.reshape(got.shape))
    assert np.array_equal(s.info.cpu().numpy(), info)
    links = s.link.cpu().numpy().view(np.uint32).reshape(got.shape)
    assert np.array_equal(links, O.links(q, want).reshape(got.shape))
    assert s.porosity.item() == info[3] / (nx * ny * nz)


def test_user_mask_geometry():
    rng = np.random.default_rng(0)
    m = (rng.random((30, 50)) < 0.3).astype(np.uint8) * 7  # nonzero means solid
    s = solver(9, 50, 30, geom=torch.as_tensor(m))
    assert np.array_equal(s.mask_field.cpu().numpy(), (m > 0).astype(np.uint8))
    assert np.array_equal(s.link.cpu().numpy().view(np.uint32).reshape(m.shape), O.links(9, (m > 0).astype(np.uint8)))


# ---------------------------------------------------------------- one step

def _state_case(q, precision, seed):
    if q == 9:
        nx, ny, nz = 200, 37, 1
        g = dict(kind=1, seed=seed, r_min=3, r_max=7, target_porosity=0.7)
    else:
        nx, ny, nz = 150, 13, 11
        g = dict(kind=2, seed=seed, r_min=3, r_max=3, target_porosity=0.7)
    return nx, ny, nz, g


@pytest.fixture(params=["persist", "tma", "vec", "scalar", "compact"])
def kernel(request, monkeypatch):
    """Runs a test with each kernel family: the one-launch persistent sweeps,
    the TMA-staged per-step kernels, the vectorised register kernels and one
    node per thread (all in the dense layout), and the fluid-only layout."""
    monkeypatch.setenv("LBM_LAYOUT", "compact" if request.param == "compact" else "dense")
    if request.param == "persist":
        monkeypatch.setenv("LBM_PERSIST", "1")
    elif request.param == "tma":
        monkeypatch.setenv("LBM_PERSIST", "0")
        monkeypatch.setenv("LBM_TMA_MIN_TILES", "1")
    elif request.param == "vec":
        monkeypatch.setenv("LBM_PERSIST", "0")
        monkeypatch.setenv("LBM_TMA", "0")
    elif request.param == "scalar":
        monkeypatch.setenv("LBM_KERNEL", "scalar")
    return request.param


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("profile", [False, True])
@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("nx", [200, 150, 141])
def test_steps_from_random_state(q, precision, profile, nsteps, nx, kernel):
    """lbm_step on a perturbed state vs the oracle's step (collide then stream).
    nx = 200 / 150 / 141 exercise 4-wide, 2-wide and scalar rows."""
    _, ny, nz, g = _state_case(q, precision, 11)
    s = solver(q, nx, ny, nz, precision=precision, inlet=lbm.LBM_INLET_PROFILE if profile else 0, geom=g)
    m = s.mask_field.cpu().numpy()
    shape = m.shape
    fs = W.perturbation((q,) + shape, seed=12, scale=2e-3)
    fs[:, m.astype(bool)] = 0
    n_in = ny * nz if profile else 1
    rin = 1.0 + 1e-3 + W.perturbation((n_in,), seed=13, scale=5e-4)
    rho_out, tau = 0.9995, 0.83
    got = s.step(dev(rin), dev([tau]), rho_out, dev(fs, s.plan.dtype), nsteps).cpu().numpy()
    f = fs + weights(q, len(shape))
    rin_o = rin.reshape((nz, ny) if q == 19 else (ny,)) if profile else rin[0]
    for _ in range(nsteps):
        f = O.step(q, m, f, rin_o, rho_out, tau)
    want = f - weights(q, len(shape))
    fl = ~m.astype(bool)
    tol = 1e-11 if precision == 8 else 2e-5
    assert rel(got[:, fl], want[:, fl]) < tol


# ---------------------------------------------------------- forward from rest

@pytest.mark.parametrize("q,precision,T", [(9, 8, 300), (9, 4, 300), (19, 8, 60), (19, 4, 60)])
def test_forward_from_rest(q, precision, T, kernel):
    nx, ny, nz, g = _state_case(q, precision, 21)
    s = solver(q, nx, ny, nz, precision=precision, T=T, inlet=lbm.LBM_INLET_PROFILE, geom=g)
    m = s.mask_field.cpu().numpy()
    n_in = ny * nz
    rin = 1.0 + W.inlet_profile(n_in, seed=22)
    tau = 0.8
    f = s.forward(dev(rin), dev([tau]), 1.0)
    rho, u = s.macroscopic(f)
    want_f = O.forward(q, m, rin.reshape((nz, ny) if q == 19 else (ny,)), 1.0, tau, T)
    want_rho, want_u = O.macroscopic(q, m, want_f)
    tol_u = 1e-11 if precision == 8 else 1e-4
    assert rel(u.cpu().numpy(), want_u) < tol_u
    fl = ~m.astype(bool)
    assert rel((rho.cpu().numpy() - 1.0)[fl], (want_rho - 1.0)[fl]) < (1e-10 if precision == 8 else 1e-4)
    assert np.all(u.cpu().numpy()[:, m.astype(bool)] == 0)


# ------------------------------------------------------------- loss + seed

@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("kind", [lbm.LBM_LOSS_VEC, lbm.LBM_LOSS_NORM])
@pytest.mark.parametrize("norm", [lbm.LBM_NORM_SUM, lbm.LBM_NORM_MEAN_FLUID])
@pytest.mark.parametrize("with_roi", [False, True])
def test_loss_and_seed(q, kind, norm, with_roi):
    nx, ny, nz, g = _state_case(q, 8, 31)
    s = solver(q, nx, ny, nz, precision=8, kind=kind, norm=norm, geom=g)
    m = s.mask_field.cpu().numpy()
    shape = m.shape
    fs = W.perturbation((q,) + shape, seed=32, scale=2e-3)
    fs[:, m.astype(bool)] = 0
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + shape, seed=33, scale=3e-3)
    roi = W.roi_band(shape, axis=len(shape) - 1, start=nx // 3) if with_roi else None
    L, lam = s.loss_grad(dev(fs), dev(ut), None if roi is None else dev(roi, torch.uint8))
    Lw, lamw = O.loss(q, m, fs + weights(q, len(shape)), ut, roi, kind, norm)
    assert abs(L.item() - Lw) <= 1e-12 * abs(Lw)
    assert rel(lam.cpu().numpy(), lamw) < 1e-12


def test_nonfinite_loss_is_latched():
    s = solver(9, 40, 20, precision=4, geom=dict(kind=0))
    f = torch.zeros((9, 20, 40), dtype=torch.float32, device="cuda")
    ut = torch.full((2, 20, 40), float("nan"), dtype=torch.float64, device="cuda")
    s.loss_grad(f, ut)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_ERR_NONFINITE
    assert s.status() == lbm.LBM_OK  # reading clears it


# --------------------------------------------------------------- gradients

@pytest.mark.parametrize("q,T", [(9, 40), (19, 12)])
@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("profile", [False, True])
@pytest.mark.parametrize("stride", [0, 1, 7])
@pytest.mark.parametrize("nx", [140, 138])
def test_gradient_matches_oracle(q, T, precision, profile, stride, nx, kernel):
    if q == 9:
        ny, nz, g = 33, 1, dict(kind=1, seed=41, r_min=3, r_max=6, target_porosity=0.72)
    else:
        ny, nz, g = 11, 9, dict(kind=2, seed=41, r_min=2, r_max=2, target_porosity=0.8, inlet_buffer=4)
    s = solver(q, nx, ny, nz, precision=precision, T=T, stride=stride,
               inlet=lbm.LBM_INLET_PROFILE if profile else 0, geom=g)
    m = s.mask_field.cpu().numpy()
    shape = m.shape
    n_in = ny * nz if profile else 1
    rin = 1.0 + (W.inlet_profile(n_in, seed=42) if profile else np.array([1.2e-3]))
    tau = 0.85
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + shape, seed=43, scale=1e-3)
    f = s.forward(dev(rin), dev([tau]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([tau]), 1.0, lam)
    rin_o = rin.reshape((nz, ny) if q == 19 else (ny,)) if profile else rin[0]
    Lw, g_in_w, g_tau_w = O.gradient(q, m, rin_o, 1.0, tau, T, ut, ckpt_stride=5)
    if precision == 8:
        assert abs(L.item() - Lw) <= 1e-10 * abs(Lw)
        assert rel(g_in.cpu().numpy(), np.ravel(g_in_w)) < 1e-9
        assert abs(g_tau.item() - g_tau_w) <= 1e-9 * abs(g_tau_w)
    else:
        assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
        assert rel(g_in.cpu().numpy(), np.ravel(g_in_w)) < 1e-3
        assert abs(g_tau.item() - g_tau_w) <= 1e-3 * abs(g_tau_w)


def test_channel64x32_fp64_end_to_end():
    """The 64x32 FP64 channel, 1000 steps, loss against the analytic
    Poiseuille profile, gradient with respect to a constant rho_in."""
    wl = W.WORKLOADS["channel64x32"]
    s = solver(9, wl.nx, wl.ny, precision=8, T=wl.steps, geom=dict(kind=0))
    m = s.mask_field.cpu().numpy()
    y = np.arange(wl.ny)
    nu = (wl.tau - 0.5) / 3.0
    G = wl.delta_rho / 3.0 / wl.nx
    ut = np.zeros((2, wl.ny, wl.nx))
    ut[0] = (G / (2 * nu) * (y + 0.5) * (wl.ny - 0.5 - y))[:, None]
    rin = np.array([wl.rho_out + wl.delta_rho])
    f = s.forward(dev(rin), dev([wl.tau]), wl.rho_out)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([wl.tau]), wl.rho_out, lam)
    Lw, g_in_w, g_tau_w = O.gradient(9, m, rin[0], wl.rho_out, wl.tau, wl.steps, ut, ckpt_stride=32)
    assert abs(L.item() - Lw) <= 1e-10 * Lw
    assert abs(g_in.item() - g_in_w) <= 1e-9 * abs(g_in_w)
    assert abs(g_tau.item() - g_tau_w) <= 1e-9 * abs(g_tau_w)


# ------------------------------------------------------- post-processing

def test_darcy_and_adam():
    s = solver(9, 96, 24, precision=8, T=1, geom=dict(kind=1, seed=9, r_min=3, r_max=5, target_porosity=0.75))
    m = s.mask_field.cpu().numpy()
    f = W.perturbation((9, 24, 96), seed=1, scale=1e-3)
    f[:, m.astype(bool)] = 0
    k, J = s.darcy(dev(f), dev([1.001]), dev([0.9]), 1.0, xs=40)
    kw, Jw = O.darcy(9, m, f + weights(9, 2), 1.001, 1.0, 0.9, xs=40)
    assert abs(J.item() - Jw) <= 1e-12 * abs(Jw) and abs(k.item() - kw) <= 1e-10 * abs(kw)

    n = 37
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(n)
    mm = np.zeros(n)
    vv = np.zeros(n)
    th_d, m_d, v_d = dev(theta), dev(mm), dev(vv)
    p_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    for t in range(1, 4):
        gp = rng.standard_normal(n)
        lbm.lbm_adam_step(th_d, m_d, v_d, dev(gp), p_d, 1.0, 1e-3, t, 0.02)
        O.adam(theta, gp * 1e-3, mm, vv, t, 0.02)
    assert np.allclose(th_d.cpu().numpy(), theta, rtol=1e-13, atol=1e-15)
    assert np.allclose(p_d.cpu().numpy(), 1.0 + 1e-3 * theta, rtol=1e-14)


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("layout", ["dense", "compact"])
def test_overlapped_reverse_sweep_is_bitwise_the_serial_one(q, layout):
    """Recomputing segment s - 1 on a second stream during the adjoint steps
    of segment s changes nothing: the adjoint launches and their reduction
    order are the same."""
    nx, ny, nz, g = _state_case(q, 4, 51)
    T = 23
    out = []
    for overlap in (0, 1):
        s = lbm.Solver(q, nx, ny, nz, precision=4, n_steps=T, ckpt_stride=4, inlet_kind=lbm.LBM_INLET_PROFILE,
                       geometry=g, layout=layout)
        lbm.lbm_plan_set_kernels(s.plan, overlap=overlap)
        rin = 1.0 + W.inlet_profile(ny * nz, seed=52)
        ut = W.perturbation((s.plan.d, *s.plan.shape), seed=53, scale=1e-3)
        f = s.forward(dev(rin), dev([0.8]), 1.0)
        L, lam = s.loss_grad(f, dev(ut))
        g_in, g_tau = s.adjoint(dev(rin), dev([0.8]), 1.0, lam)
        out.append((g_in.cpu().numpy(), g_tau.item()))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_compact_bind_checks_the_fluid_count_and_switches_back():
    """lbm_compact_bind rejects a fluid count that is not the link array's;
    switching a solver to the compact layout and back gives the same forward."""
    nx, ny, nz, g = _state_case(19, 4, 61)
    s = lbm.Solver(19, nx, ny, nz, precision=4, n_steps=20, geometry=g, layout="dense")
    nf = int(s.info[3].item())
    tables = torch.empty(lbm.lbm_compact_size(s.plan, nf + 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_compact_bind(s.plan, nf + 1, tables, s.stream)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    rin, tau = dev([1.001]), dev([0.8])
    f_dense = s.forward(rin, tau, 1.0).clone()
    s.set_layout("compact")
    assert s.layout == "compact"
    f_cmp = s.forward(rin, tau, 1.0).clone()
    s.set_layout("dense")
    f_back = s.forward(rin, tau, 1.0)
    fl = ~s.mask_field.bool()
    assert torch.allclose(f_dense[:, fl], f_cmp[:, fl], rtol=0, atol=1e-8)  # same arithmetic per node
    assert torch.equal(f_dense, f_back)
    assert torch.count_nonzero(f_cmp[:, ~fl]).item() == 0
