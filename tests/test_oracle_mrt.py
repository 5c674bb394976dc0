"""Pins of the oracle's D2Q9 MRT collision (Eq. 16-18) against the printed
moment matrix, the BGK special case and complex-step derivatives (CPU)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_00810_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mrt_matrix_d2q9.txt")
RATES = (1.64, 1.54, 1.9)  # s_e, s_eps, s_q


@pytest.fixture(autouse=True)
def _bgk_afterwards():
    yield
    O.set_collision(O.COLL_BGK)


def _printed_matrix():
    rows = [r for r in open(GOLDEN).read().splitlines() if r.strip() and not r.startswith("#")]
    M = np.array([[float(v) for v in r.split()] for r in rows])
    # the printed last row is |c_x c_y|; the orthogonal p_xy row is j_x * j_y elementwise
    M[8] = M[3] * M[5]
    return M


def _mask():
    m = np.zeros((7, 10), np.uint8)
    m[3, 5] = 1
    return m


def test_each_moment_relaxes_at_its_own_rate():
    """m* = m - s (m - m^eq) for every row of the printed matrix, with m^eq =
    M f^eq; rho and j are conserved."""
    r = np.random.Generator(np.random.PCG64(1))
    n = 50
    f = O.rest(9, (n,)) + r.normal(0, 2e-3, (9, n))
    tau = 0.7
    with O.collision(O.COLL_MRT, *RATES):
        fs = O.collide(9, f, tau)
    M = _printed_matrix()
    c, _, _ = O.lattice(9)
    rho = f.sum(0)
    u = (c[:, :2].T.astype(float) @ f) / rho
    feq = O.equilibrium(9, rho, u)
    m, ms, meq = M @ f, M @ fs, M @ feq
    s = np.array([0, RATES[0], RATES[1], 0, RATES[2], 0, RATES[2], 1 / tau, 1 / tau])
    np.testing.assert_allclose(ms, m - s[:, None] * (m - meq), rtol=0, atol=1e-14)
    np.testing.assert_allclose(ms[[0, 3, 5]], m[[0, 3, 5]], rtol=0, atol=1e-15)


def test_equal_rates_reduce_to_bgk():
    """S = I / tau is BGK: steps, losses and inlet gradients agree to
    rounding.  dL/dtau does not: under MRT only the two stress rates follow
    tau, the others are held at their set values."""
    m = _mask()
    tau = 0.8
    f = O.forward(9, m, 1.001, 1.0, tau, 10)
    bgk = O.step(9, m, f, 1.001, 1.0, tau)
    ut = W.perturbation((2,) + m.shape, seed=2, scale=1e-3)
    Lb, gb, tb = O.gradient(9, m, 1.001, 1.0, tau, 15, ut)
    with O.collision(O.COLL_MRT, 1 / tau, 1 / tau, 1 / tau):
        mrt = O.step(9, m, f, 1.001, 1.0, tau)
        Lm, gm, tm = O.gradient(9, m, 1.001, 1.0, tau, 15, ut)
    np.testing.assert_allclose(mrt, bgk, rtol=0, atol=1e-15)
    assert np.isclose(Lm, Lb, rtol=1e-12) and np.isclose(gm, gb, rtol=1e-10)
    assert not np.isclose(tm, tb, rtol=1e-3)
    # other rates change the result
    with O.collision(O.COLL_MRT, *RATES):
        assert not np.allclose(O.step(9, m, f, 1.001, 1.0, tau), bgk, rtol=0, atol=1e-12)


@pytest.mark.parametrize("profile", [False, True])
def test_mrt_adjoint_step_is_transpose_of_step(profile):
    m = _mask()
    rho_in = 1.0 + (0.001 + W.perturbation((7,), seed=5, scale=5e-4) if profile else 0.0012)
    rho_out, tau = 1.0, 0.75
    h = 1e-30
    with O.collision(O.COLL_MRT, *RATES):
        f = O.forward(9, m, rho_in, rho_out, tau, 12)
        lam = W.perturbation(f.shape, seed=8, scale=1.0)
        lam[:, m.astype(bool)] = 0
        lam_t, g_in, g_om = O.adjoint_step(9, m, f, lam, rho_in, rho_out, tau)
        df = W.perturbation(f.shape, seed=9, scale=1.0)
        df[:, m.astype(bool)] = 0
        jd = O.step(9, m, f + 1j * h * df, rho_in, rho_out, tau, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jd), np.sum(lam_t * df), rtol=1e-12, atol=0)
        dr = W.perturbation(np.shape(rho_in), seed=10, scale=1.0) if profile else 1.0
        jr = O.step(9, m, f, np.asarray(rho_in) + 1j * h * np.asarray(dr), rho_out, tau, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jr), np.sum(np.ravel(g_in) * np.ravel(dr)), rtol=1e-12, atol=0)
        jt = O.step(9, m, f, rho_in, rho_out, tau + 1j * h, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jt), -g_om / tau ** 2, rtol=1e-12, atol=0)


def test_mrt_gradient_matches_complex_step():
    m = _mask()
    T, rho_out, tau = 20, 1.0, 0.7
    rho_in = 1.0 + 0.001 + W.perturbation((7,), seed=15, scale=5e-4)
    ut = W.perturbation((2,) + m.shape, seed=16, scale=2e-3)
    h = 1e-30
    with O.collision(O.COLL_MRT, *RATES):
        L, g_in, g_tau = O.gradient(9, m, rho_in, rho_out, tau, T, ut, ckpt_stride=6)

        def loss_c(rin, t):
            return O.loss(9, m, O.forward(9, m, rin, rho_out, t, T, complex_step=True), ut, seed=False,
                          complex_step=True)

        for k in (0, 3, 6):
            e = np.zeros(7, np.complex128)
            e[k] = 1j * h
            assert np.isclose(g_in[k], loss_c(rho_in + e, tau).imag / h, rtol=1e-11, atol=0)
        assert np.isclose(g_tau, loss_c(rho_in, tau + 1j * h).imag / h, rtol=1e-11, atol=0)


def test_mrt_is_d2q9_only():
    m = np.zeros((4, 4, 5), np.uint8)
    with O.collision(O.COLL_MRT, *RATES):
        with pytest.raises(RuntimeError):
            O.step(19, m, O.rest(19, m.shape), 1.001, 1.0, 0.8)
