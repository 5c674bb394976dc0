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
