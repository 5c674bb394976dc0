"""Pins of the oracle's cylinder-wake options (section 3.4): periodic top and
bottom, and the velocity inlet (moving-wall bounce-back through x = -1/2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_00810_gb300 import workloads as W

RATES = (1.64, 1.54, 1.9)


@pytest.fixture(autouse=True)
def _defaults_afterwards():
    yield
    O.set_periodic_y(False)
    O.set_velocity_inlet(None)
    O.set_velocity_ramp(0)
    O.set_time(1)
    O.set_collision(O.COLL_BGK)


def _cylinder(nx=40, ny=20, cx=10, cy=9.5, r=3.2):
    y, x = np.mgrid[0:ny, 0:nx]
    return (((x - cx) ** 2 + (y - cy) ** 2) <= r * r).astype(np.uint8)


@pytest.mark.parametrize("mrt", [False, True])
def test_uniform_flow_is_an_exact_fixed_point(mrt):
    """With periodic y and no obstacle, the equilibrium state of uniform
    velocity u_in and rho = 1 is reproduced by the velocity inlet (its source
    turns f^eq_opp(i) into f^eq_i), by streaming and by Eq. 6 at the outlet
    with rho_out = 1."""
    nx, ny, u = 24, 10, (0.05, 0.0)
    m = np.zeros((ny, nx), np.uint8)
    f = O.equilibrium(9, np.ones((ny, nx)), np.stack([np.full((ny, nx), u[0]), np.zeros((ny, nx))]))
    if mrt:
        O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=u):
        g = O.step(9, m, f, 1.0, 1.0, 0.7)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-16)
    # with walls (not periodic) the no-slip walls change the flow
    with O.wake_options(periodic_y=False, velocity_inlet=u):
        assert np.abs(O.step(9, m, f, 1.0, 1.0, 0.7) - f).max() > 1e-4


def test_periodic_step_commutes_with_a_shift_in_y():
    m = _cylinder()
    r = np.random.Generator(np.random.PCG64(3))
    f = O.rest(9, m.shape) + r.normal(0, 1e-3, (9,) + m.shape)
    f[:, m.astype(bool)] = 0
    with O.wake_options(periodic_y=True, velocity_inlet=(0.04, 0.01)):
        g = O.step(9, m, f, 1.0, 1.0, 0.8)
        k = 7
        gs = O.step(9, np.roll(m, k, axis=0), np.roll(f, k, axis=1), 1.0, 1.0, 0.8)
    np.testing.assert_array_equal(gs, np.roll(g, k, axis=1))


def test_periodic_link_words_by_brute_force():
    m = _cylinder(cy=0.5)  # the cylinder straddles y = 0 / ny - 1
    with O.wake_options(periodic_y=True):
        link = O.links(9, m)
    c, _, _ = O.lattice(9)
    ny, nx = m.shape
    for y in range(ny):
        for x in range(nx):
            if m[y, x]:
                assert link[y, x] == 1 << 31
                continue
            want = 0
            for i in range(9):
                sx, sy = x - c[i][0], (y - c[i][1]) % ny
                if 0 <= sx < nx and m[sy, sx]:
                    want |= 1 << i
            assert link[y, x] == want, (y, x)


@pytest.mark.parametrize("mrt", [False, True])
def test_wake_adjoint_step_and_gradient_by_complex_step(mrt):
    m = _cylinder()
    rho_out, tau, T = 1.0, 0.62, 15
    h = 1e-30
    if mrt:
        O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0)):
        f = O.forward(9, m, 1.0, rho_out, tau, 10)
        lam = W.perturbation(f.shape, seed=8, scale=1.0)
        lam[:, m.astype(bool)] = 0
        lam_t, g_in, g_om = O.adjoint_step(9, m, f, lam, 1.0, rho_out, tau)
        df = W.perturbation(f.shape, seed=9, scale=1.0)
        df[:, m.astype(bool)] = 0
        jd = O.step(9, m, f + 1j * h * df, 1.0, rho_out, tau, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jd), np.sum(lam_t * df), rtol=1e-12, atol=0)
        jt = O.step(9, m, f, 1.0, rho_out, tau + 1j * h, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jt), -g_om / tau ** 2, rtol=1e-12, atol=0)
        assert g_in == 0.0  # the velocity inlet does not use rho_in
        ut = W.perturbation((2,) + m.shape, seed=16, scale=2e-3)
        L, gi, gt = O.gradient(9, m, 1.0, rho_out, tau, T, ut, ckpt_stride=4)
        d = O.loss(9, m, O.forward(9, m, 1.0, rho_out, tau + 1j * h, T, complex_step=True), ut, seed=False,
                   complex_step=True).imag / h
        assert np.isclose(gt, d, rtol=1e-11, atol=0) and gi == 0.0


# ------------------------------------------------ gradual start (velocity ramp)


@pytest.mark.parametrize("t", [1, 2, 5, 9, 10, 14])
def test_ramp_scales_the_inflow_source_by_sin_squared(t):
    """From rest (f* = w_i), the step producing f^t at the inlet nodes gives
    f_i = w_opp(i) + 6 w_i (c_i . u_in) r(t), r(t) = sin^2(pi t / (2 R)) for
    t < R and 1 after (R = 10 here): the increment over rest is the source
    times r(t), exactly."""
    import math

    nx, ny, R, u = 12, 6, 10, (0.05, 0.01)
    m = np.zeros((ny, nx), np.uint8)
    c, w, opp = O.lattice(9)
    f0 = O.rest(9, m.shape)
    with O.wake_options(periodic_y=True, velocity_inlet=u, ramp=R):
        O.set_time(t)
        g = O.step(9, m, f0, 1.0, 1.0, 0.8)
    r = math.sin(math.pi * t / (2 * R)) ** 2 if t < R else 1.0
    for i in range(9):
        if c[i][0] != 1:
            continue
        want = w[opp[i]] + 6.0 * w[i] * (c[i][0] * u[0] + c[i][1] * u[1]) * r
        np.testing.assert_allclose(g[i, :, 0], want, rtol=0, atol=1e-15)


def test_ramp_zero_is_the_impulsive_start_and_forward_counts_time_from_one():
    m = _cylinder()
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=0):
        a = O.forward(9, m, 1.0, 1.0, 0.7, 6)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=1):
        b = O.forward(9, m, 1.0, 1.0, 0.7, 6)  # r(t) = 1 from t = 1: the same run
    np.testing.assert_array_equal(a, b)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=8):
        f = O.rest(9, m.shape)
        for t in range(1, 7):
            O.set_time(t)
            f = O.step(9, m, f, 1.0, 1.0, 0.7)
        np.testing.assert_array_equal(O.forward(9, m, 1.0, 1.0, 0.7, 6), f)


@pytest.mark.parametrize("mrt", [False, True])
def test_ramped_gradient_matches_complex_step(mrt):
    """dL/dtau of a ramped wake sweep (the ramp does not depend on the
    parameters; the recompute must replay the same time levels) against the
    complex-step derivative of the forward and the loss."""
    m = _cylinder(nx=30, ny=12, cx=8, cy=5.5, r=2.5)
    T, tau, h = 24, 0.7, 1e-30
    ut = W.perturbation((2,) + m.shape, seed=4, scale=2e-3)
    roi = np.zeros(m.shape, np.uint8)
    roi[:, 15:] = 1
    if mrt:
        O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=16):
        L, g_in, g_tau = O.gradient(9, m, 1.0, 1.0, tau, T, ut, roi=roi, ckpt_stride=5)
        fc = O.forward(9, m, 1.0, 1.0, tau + 1j * h, T, complex_step=True)
        Lc = O.loss(9, m, fc, ut, roi, seed=False, complex_step=True)
    assert abs(Lc.real - L) <= 1e-13 * abs(L)
    assert abs(Lc.imag / h - g_tau) <= 1e-10 * abs(g_tau)


# ------------------------------------------------ loss over a time window


def _window_case(profile):
    if profile:
        m, _ = O.geometry(9, 24, 10, kind=O.GEOM_DISKS, seed=3, r_min=2, r_max=3, porosity=0.85, buffer=3)
        rin = 1.0 + W.inlet_profile(10, seed=5)
    else:
        m, rin = _cylinder(nx=30, ny=12, cx=8, cy=5.5, r=2.5), 1.0
    return m, rin


def test_window_with_one_observation_at_T_is_the_final_step_gradient():
    m, rin = _window_case(True)
    ut = W.perturbation((1, 2) + m.shape, seed=6, scale=2e-3)
    got = O.gradient_window(9, m, rin, 1.0, 0.8, 20, [20], ut, ckpt_stride=6)
    want = O.gradient(9, m, rin, 1.0, 0.8, 20, ut[0], ckpt_stride=6)
    assert got[0] == want[0] and np.array_equal(got[1], want[1]) and got[2] == want[2]


def test_window_gradient_is_the_sum_of_snapshot_gradients():
    """Linearity: the window's loss and gradient are the sums over its
    observations of final-step losses and gradients of sweeps ending there."""
    m, rin = _window_case(True)
    obs = [7, 12, 20]
    ut = W.perturbation((3, 2) + m.shape, seed=7, scale=2e-3)
    L, g_in, g_tau = O.gradient_window(9, m, rin, 1.0, 0.8, 20, obs, ut, ckpt_stride=4)
    parts = [O.gradient(9, m, rin, 1.0, 0.8, t, ut[k], ckpt_stride=4) for k, t in enumerate(obs)]
    assert abs(L - sum(p[0] for p in parts)) <= 1e-13 * abs(L)
    np.testing.assert_allclose(g_in, sum(p[1] for p in parts), rtol=1e-11, atol=0)
    assert abs(g_tau - sum(p[2] for p in parts)) <= 1e-11 * abs(g_tau)


@pytest.mark.parametrize("wake", [False, True])
def test_window_gradient_matches_complex_step(wake):
    """Against the complex-step derivative of sum_k L(f^{t_k}) formed by
    stepping complex states (no shared reverse code): dL/dtau, and for the
    pressure-driven case dL/d(head)."""
    m, rin = _window_case(not wake)
    T, tau, h, obs = 18, 0.75, 1e-30, [5, 11, 18]
    ut = W.perturbation((3, 2) + m.shape, seed=8, scale=2e-3)
    roi = np.ones(m.shape, np.uint8)
    roi[:, :4] = 0
    opts = dict(periodic_y=True, velocity_inlet=(0.05, 0.0), ramp=12) if wake else {}
    if wake:
        O.set_collision(O.COLL_MRT, *RATES)
    with O.wake_options(**opts):
        L, g_in, g_tau = O.gradient_window(9, m, rin, 1.0, tau, T, obs, ut, roi=roi, ckpt_stride=5)

        def window_loss(rho_in, tau_c):
            f = O.rest(9, m.shape).astype(np.complex128)
            total = 0j
            for t in range(1, T + 1):
                O.set_time(t)
                f = O.step(9, m, f, rho_in, 1.0, tau_c, complex_step=True)
                if t in obs:
                    total += O.loss(9, m, f, ut[obs.index(t)], roi, seed=False, complex_step=True)
            return total

        Lt = window_loss(np.asarray(rin, np.complex128), tau + 1j * h)
        assert abs(Lt.real - L) <= 1e-13 * abs(L)
        assert abs(Lt.imag / h - g_tau) <= 1e-10 * abs(g_tau)
        if not wake:
            Lh = window_loss(np.asarray(rin, np.complex128) + 1j * h, tau)
            assert abs(Lh.imag / h - np.sum(g_in)) <= 1e-10 * abs(np.sum(g_in))
