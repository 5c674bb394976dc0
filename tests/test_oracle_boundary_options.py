"""Pins of the oracle's two optional terms: the anti-bounce-back velocity
extrapolated to the pressure plane (Eq. 6 with u_w = u(x_b) + (u(x_b) - u(x_b + e)) / 2)
and the density-probe loss.

Each option is pinned away from the oracle's own formulas: the extrapolated
velocity by a flow whose velocity is linear in x (for which the extrapolation is
exact) and by the cases where it must reduce to the node velocity, the probe
term by a brute-force sum over the populations, and both reverse sweeps by
complex-step derivatives of the forward alone.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_00810_gb300 import workloads as W


@pytest.fixture(autouse=True)
def _node_velocity_afterwards():
    yield
    O.set_abb_velocity(O.UW_NODE)


def _mask(q):
    """Tiny lattices with a solid node right behind the inlet in one row (so
    that row keeps the node velocity) and one inside."""
    if q == 9:
        m = np.zeros((6, 8), np.uint8)
        m[2, 1] = 1
        m[4, 5] = 1
    else:
        m = np.zeros((5, 5, 6), np.uint8)
        m[1, 2, 1] = 1
        m[3, 2, 4] = 1
    return m


def _rho_in(q, m, profile, seed):
    ny, nz = m.shape[-2], (m.shape[0] if q == 19 else 1)
    if not profile:
        return 1.0015
    return 1.0 + 0.001 + W.perturbation((nz, ny) if q == 19 else (ny,), seed=seed, scale=5e-4)


def _eq_state(q, m, u):
    """Equilibrium populations at rho = 1 with velocity field u[D, ...]."""
    return O.equilibrium(q, np.ones(m.shape), u)


@pytest.mark.parametrize("q", [9, 19])
def test_linear_velocity_is_extrapolated_exactly_to_the_planes(q):
    """For u linear in x, u(-1/2) = u(0) - (u(1) - u(0)) / 2 exactly.  With tau = 1
    the post-collision state is f^eq, and Eq. 6's source 2 w_i rho_w (1 + 4.5 (c_i.u)^2
    - 1.5 u.u) is the even part f^eq_i + f^eq_opp(i) of the equilibrium at (rho_w, u_w):
    every Eq. 6 slot must equal -f^eq_opp(i)(x_b) + f^eq_i(rho_w, u_w(plane)) + f^eq_opp(i)(rho_w, u_w(plane))."""
    m = np.zeros((6, 8), np.uint8) if q == 9 else np.zeros((4, 4, 6), np.uint8)
    nx = m.shape[-1]
    d = 2 if q == 9 else 3
    x = np.arange(nx, dtype=np.float64)
    a, b = np.array([0.02, -0.01, 0.005][:d]), np.array([0.003, 0.002, -0.001][:d])
    u = (a.reshape((d,) + (1,) * m.ndim) + b.reshape((d,) + (1,) * m.ndim) * x).astype(np.float64)
    u = np.broadcast_to(u, (d,) + m.shape).copy()
    f = _eq_state(q, m, u)
    rin, rout = 1.002, 0.999
    c, w, opp = O.lattice(q)
    with O.abb_velocity(O.UW_EXTRAP):
        g = O.step(q, m, f, rin, rout, 1.0)
    for side, xb, rw, plane in ((+1, 0, rin, -0.5), (-1, nx - 1, rout, nx - 0.5)):
        uw = a + b * plane
        shape = (d,) + m.shape[:-1]
        fe = O.equilibrium(q, np.full(m.shape[:-1], rw), np.broadcast_to(uw.reshape((d,) + (1,) * (m.ndim - 1)), shape))
        for i in range(q):
            if c[i][0] != side:
                continue
            # links that also cross a wall plane bounce back; only rows whose
            # source stays inside the lattice in y (and z) take Eq. 6
            want = -f[opp[i]][..., xb] + fe[i] + fe[opp[i]]
            got = g[i][..., xb]
            if q == 9:
                ys = slice(max(0, c[i][1]), m.shape[0] + min(0, c[i][1]))
                sl = [ys]
            else:
                zs = slice(max(0, c[i][2]), m.shape[0] + min(0, c[i][2]))
                ys = slice(max(0, c[i][1]), m.shape[1] + min(0, c[i][1]))
                sl = [zs, ys]
            np.testing.assert_allclose(got[tuple(sl)], want[tuple(sl)], rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", [9, 19])
def test_extrapolation_reduces_to_the_node_velocity(q):
    """A state uniform in x (u(x_b + e) = u(x_b)) gives bit-identical steps in
    both modes; rows whose inward neighbour is solid keep the node velocity."""
    m = np.zeros((6, 8), np.uint8) if q == 9 else np.zeros((4, 4, 6), np.uint8)
    col = W.perturbation((q,) + m.shape[:-1] + (1,), seed=3, scale=1e-3)
    f = O.rest(q, m.shape) + np.broadcast_to(col, (q,) + m.shape)
    node = O.step(q, m, f, 1.001, 1.0, 0.8)
    with O.abb_velocity(O.UW_EXTRAP):
        ext = O.step(q, m, f, 1.001, 1.0, 0.8)
    assert np.array_equal(node, ext)

    m = _mask(q)
    f = O.rest(q, m.shape) + W.perturbation((q,) + m.shape, seed=4, scale=1e-3)
    node = O.step(q, m, f, 1.001, 1.0, 0.8)
    with O.abb_velocity(O.UW_EXTRAP):
        ext = O.step(q, m, f, 1.001, 1.0, 0.8)
    row = (slice(None), 2, 0) if q == 9 else (slice(None), 1, 2, 0)
    assert np.array_equal(node[row], ext[row])          # x = 1 is solid in that row
    assert not np.array_equal(node[..., 0], ext[..., 0])  # the other inlet rows change
    assert np.array_equal(node[..., 1:-1], ext[..., 1:-1])  # nothing changes inside


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("profile", [False, True])
def test_extrapolated_adjoint_step_is_transpose_of_step(q, profile):
    """Dot-product test of one reverse step with the extrapolated u_w, the
    forward Jacobian taken by complex step of the forward step alone."""
    m = _mask(q)
    rho_in = _rho_in(q, m, profile, 5)
    rho_out, tau = 1.0, 0.85
    with O.abb_velocity(O.UW_EXTRAP):
        f = O.forward(q, m, rho_in, rho_out, tau, 12)
        lam = W.perturbation(f.shape, seed=8, scale=1.0)
        lam[:, m.astype(bool)] = 0
        lam_t, g_in, g_om = O.adjoint_step(q, m, f, lam, rho_in, rho_out, tau)
        h = 1e-30
        df = W.perturbation(f.shape, seed=9, scale=1.0)
        df[:, m.astype(bool)] = 0
        jd = O.step(q, m, f + 1j * h * df, rho_in, rho_out, tau, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jd), np.sum(lam_t * df), rtol=1e-12, atol=0)
        dr = W.perturbation(np.shape(rho_in), seed=10, scale=1.0) if profile else 1.0
        jr = O.step(q, m, f, np.asarray(rho_in) + 1j * h * np.asarray(dr), rho_out, tau, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jr), np.sum(np.ravel(g_in) * np.ravel(dr)), rtol=1e-12, atol=0)
        jt = O.step(q, m, f, rho_in, rho_out, tau + 1j * h, complex_step=True).imag / h
        assert np.isclose(np.sum(lam * jt), -g_om / tau ** 2, rtol=1e-12, atol=0)
    # the extrapolation moves the adjoint at the inlet column and its neighbour only
    lam_node, _, _ = O.adjoint_step(q, m, f, lam, rho_in, rho_out, tau)
    diff = np.any(lam_node != lam_t, axis=tuple(range(m.ndim)))  # over Q and all but x
    assert diff[0] and diff[1] and diff[-1] and diff[-2] and not np.any(diff[2:-2])


@pytest.mark.parametrize("q,T", [(9, 16), (19, 8)])
def test_extrapolated_gradient_matches_complex_step(q, T):
    m = _mask(q)
    rho_in = _rho_in(q, m, True, 15)
    rho_out, tau = 1.0, 0.8
    d = 2 if q == 9 else 3
    ut = W.perturbation((d,) + m.shape, seed=16, scale=2e-3)
    with O.abb_velocity(O.UW_EXTRAP):
        L, g_in, g_tau = O.gradient(q, m, rho_in, rho_out, tau, T, ut, ckpt_stride=3)
        h = 1e-30

        def loss_c(rin, t):
            fT = O.forward(q, m, rin, rho_out, t, T, complex_step=True)
            return O.loss(q, m, fT, ut, seed=False, complex_step=True)

        flat = np.ravel(rho_in)
        for k in [0, 2, flat.size - 1]:
            e = np.zeros(flat.size, np.complex128)
            e[k] = 1j * h
            dk = loss_c((flat + e).reshape(np.shape(rho_in)), tau).imag / h
            assert np.isclose(np.ravel(g_in)[k], dk, rtol=1e-11, atol=0)
        assert np.isclose(g_tau, loss_c(rho_in, tau + 1j * h).imag / h, rtol=1e-11, atol=0)
        assert np.isclose(loss_c(rho_in, tau).real, L, rtol=1e-15)
    L0, g0, _ = O.gradient(q, m, rho_in, rho_out, tau, T, ut, ckpt_stride=3)
    assert not np.array_equal(g0, g_in)


# -------------------------------------------------------------- density probes


def _probes(m, n, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    fluid = np.flatnonzero(m.reshape(-1) == 0)
    nodes = r.choice(fluid, size=n, replace=False).astype(np.int64)
    nodes[-1] = nodes[0]  # a repeated probe counts twice
    return nodes, 1.0 + r.normal(0, 3e-4, n)


@pytest.mark.parametrize("q", [9, 19])
def test_probe_loss_by_brute_force_and_its_seed_by_complex_step(q):
    m = _mask(q)
    f = O.forward(q, m, 1.002, 1.0, 0.8, 10)
    nodes, rt = _probes(m, 5, 1)
    w = 3.0
    L, lam = O.probe_loss(q, m, f, nodes, rt, w)
    rho = f.reshape(q, -1).sum(0)
    assert np.isclose(L, w * np.sum((rho[nodes] - rt) ** 2), rtol=1e-13, atol=0)
    h = 1e-30
    for s in range(3):
        v = W.perturbation(f.shape, seed=20 + s, scale=1.0)
        Lc, _ = O.probe_loss(q, m, f + 1j * h * v, nodes, rt, w, complex_step=True)
        assert np.isclose(np.sum(lam * v), Lc.imag / h, rtol=1e-12, atol=0)
    # solid probes contribute nothing
    solid = np.flatnonzero(m.reshape(-1))[:1].astype(np.int64)
    Ls, lams = O.probe_loss(q, m, f, solid, np.array([0.5]), w)
    assert Ls == 0 and not lams.any()


@pytest.mark.parametrize("uw", [O.UW_NODE, O.UW_EXTRAP])
def test_gradient_with_probes_matches_complex_step(uw):
    q, T = 19, 8
    m = _mask(q)
    ut = W.perturbation((3,) + m.shape, seed=31, scale=2e-3)
    nodes, rt = _probes(m, 6, 2)
    rho_in, rho_out, tau = 1.0012, 1.0, 0.85
    with O.abb_velocity(uw):
        L, g_in, g_tau = O.gradient(q, m, rho_in, rho_out, tau, T, ut, probes=(nodes, rt, 50.0))
        Lv, gv, _ = O.gradient(q, m, rho_in, rho_out, tau, T, ut)
        h = 1e-30

        def loss_c(rin, t):
            fT = O.forward(q, m, rin, rho_out, t, T, complex_step=True)
            lv = O.loss(q, m, fT, ut, seed=False, complex_step=True)
            lp, _ = O.probe_loss(q, m, fT, nodes, rt, 50.0, complex_step=True)
            return lv + lp

        assert np.isclose(g_in, loss_c(rho_in + 1j * h, tau).imag / h, rtol=1e-11, atol=0)
        assert np.isclose(g_tau, loss_c(rho_in, tau + 1j * h).imag / h, rtol=1e-11, atol=0)
        assert np.isclose(L, loss_c(rho_in, tau).real, rtol=1e-14)
    assert L > Lv and g_in != gv
