"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form,
an invariant, a special case that reduces to a textbook result or a library
routine, a value the paper prints, or a brute-force restatement on a tiny
input.  Each is chosen so that a plausible slip (a dropped term, a wrong sign
or index, a transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_00810_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# --------------------------------------------------------------- RNG, lattice


def test_splitmix64_published_values():
    want = [int(v, 16) for v in _golden("splitmix64_seed0.txt")]
    assert O.splitmix64(0, len(want)) == want


@pytest.mark.parametrize("q", [9, 19])
def test_lattice_isotropy(q):
    """Weights and velocities satisfy the lattice isotropy conditions up to
    fourth order with c_s^2 = 1/3 (the reading of Eq. 9-10)."""
    c, w, opp = O.lattice(q)
    d = 2 if q == 9 else 3
    c = c[:, :d].astype(np.float64)
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), cs2 * np.eye(d), atol=1e-16)
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    I = np.eye(d)
    iso4 = cs2 * cs2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                        + np.einsum("ad,bc->abcd", I, I))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)
    for i in range(q):
        assert np.array_equal(c[opp[i]], -c[i])
    assert np.array_equal(c[0], np.zeros(d))


def test_d2q9_order_reproduces_eq18():
    """The oracle's D2Q9 ordering regenerates the paper's MRT matrix (Eq. 18)
    from the polynomial form of each moment row.  The last printed row
    (0 0 0 0 0 1 1 1 1) is |c_x c_y|; the orthogonal p_xy row is c_x c_y,
    so that row is a misprint and is checked in its printed form."""
    M = np.array([[float(v) for v in r.split()] for r in _golden("mrt_matrix_d2q9.txt")])
    c, _, _ = O.lattice(9)
    cx, cy = c[:, 0].astype(float), c[:, 1].astype(float)
    c2 = cx * cx + cy * cy
    rows = [np.ones(9), -4 + 3 * c2, 4 - 10.5 * c2 + 4.5 * c2 * c2, cx, (-5 + 3 * c2) * cx, cy,
            (-5 + 3 * c2) * cy, cx * cx - cy * cy, np.abs(cx * cy)]
    assert np.array_equal(np.array(rows), M)
    # rows 0..7 are mutually orthogonal (Gram-Schmidt construction)
    G = M[:8] @ M[:8].T
    assert np.array_equal(G, np.diag(np.diag(G)))


# ------------------------------------------------------------ collision (Eq. 4-5)


@pytest.mark.parametrize("q", [9, 19])
def test_equilibrium_moments(q):
    """Eq. 5 reproduces the textbook equilibrium moments: sum f^eq = rho,
    sum f^eq c = rho u, sum f^eq c c = rho c_s^2 I + rho u u."""
    d = 2 if q == 9 else 3
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.1 * rng.standard_normal(50)
    u = 0.05 * rng.standard_normal((d, 50))
    fe = O.equilibrium(q, rho, u)
    c, _, _ = O.lattice(q)
    c = c[:, :d].astype(float)
    assert np.allclose(fe.sum(0), rho, rtol=1e-14, atol=0)
    assert np.allclose(np.einsum("ia,in->an", c, fe), rho * u, rtol=1e-12, atol=1e-16)
    P = np.einsum("ia,ib,in->abn", c, c, fe)
    want = rho * (np.eye(d)[:, :, None] / 3.0 + np.einsum("an,bn->abn", u, u))
    assert np.allclose(P, want, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.7])
def test_bgk_conserves_and_relaxes(q, tau):
    """BGK (Eq. 4) conserves rho and rho u per node, leaves f^eq fixed, and
    scales the non-equilibrium part by exactly (1 - 1/tau)."""
    d = 2 if q == 9 else 3
    c, w, _ = O.lattice(q)
    c = c[:, :d].astype(float)
    f = w[:, None] * (1.0 + 0.2 * W.perturbation((q, 40), seed=7, scale=1.0))
    g = O.collide(q, f, tau)
    assert np.allclose(g.sum(0), f.sum(0), rtol=2e-15, atol=0)
    assert np.allclose(c.T @ g, c.T @ f, rtol=0, atol=2e-15)
    rho = f.sum(0)
    u = (c.T @ f) / rho
    fe = O.equilibrium(q, rho, u)
    assert np.allclose(g - fe, (1.0 - 1.0 / tau) * (f - fe), rtol=0, atol=1e-15)
    assert np.allclose(O.collide(q, fe, tau), fe, rtol=0, atol=2e-15)


# ------------------------------------------------ streaming, bounce-back, Eq. 6


def _closed_box(q, nx, ny, nz=1):
    m = np.zeros((ny, nx) if q == 9 else (nz, ny, nx), np.uint8)
    m[..., 0] = 1
    m[..., -1] = 1
    return m


@pytest.mark.parametrize("q", [9, 19])
def test_closed_box_conserves_mass(q):
    """With solid columns at both ends every boundary link bounces back, so
    the total mass over fluid nodes is invariant (Eq. 3 + halfway BB)."""
    m = _closed_box(q, 12, 9, 7) if q == 19 else _closed_box(q, 24, 17)
    m[(m.shape[0] // 2,) + (slice(4, 6),) * (m.ndim - 1)] = 1  # an internal grain
    c, w, _ = O.lattice(q)
    f = w.reshape((q,) + (1,) * m.ndim) * (1.0 + 0.3 * W.perturbation((q,) + m.shape, seed=3, scale=1.0))
    f[:, m.astype(bool)] = 0.0
    fl = ~m.astype(bool)
    m0 = f[:, fl].sum()
    g = O.forward(q, m, 1.0, 1.0, 0.8, 400 if q == 9 else 150, f0=f)
    assert abs(g[:, fl].sum() - m0) / m0 < 1e-13


@pytest.mark.parametrize("q", [9, 19])
def test_streaming_is_signed_permutation(q):
    """With 1/tau = 0 (no collision) and rho_w = 0, one step only moves
    values: interior links copy f_i(x - c_i) (pull in the direction of c_i),
    halfway bounce-back copies f_opp(i)(x), anti-bounce-back negates it."""
    shape = (7, 6, 5) if q == 19 else (6, 9)
    nx = shape[-1]
    m = np.zeros(shape, np.uint8)
    m[(1,) * (len(shape) - 1) + (4,)] = 1
    rng = np.random.default_rng(11)
    f = rng.integers(1, 1000, size=(q,) + shape).astype(np.float64)
    f[:, m.astype(bool)] = 0
    g = O.step(q, m, f, 0.0, 0.0, math.inf)
    c, _, opp = O.lattice(q)
    d = 2 if q == 9 else 3
    dims = shape[::-1]  # (nx, ny[, nz])
    n_abb = 0
    for idx in np.ndindex(*shape):
        if m[idx]:
            continue
        pos = idx[::-1]  # (x, y[, z])
        for i in range(q):
            src = [pos[a] - c[i][a] for a in range(d)]
            wall = any(src[a] < 0 or src[a] >= dims[a] for a in range(1, d))
            if wall:
                want = f[(opp[i],) + idx]
            elif src[0] < 0 or src[0] >= nx:
                want = -f[(opp[i],) + idx]
                n_abb += 1
            else:
                sidx = tuple(src[::-1])
                want = f[(opp[i],) + idx] if m[sidx] else f[(i,) + sidx]
            assert g[(i,) + idx] == want
    assert n_abb > 0


@pytest.mark.parametrize("q", [9, 19])
def test_rest_is_exact_fixed_point(q):
    """rho_in = rho_out = 1 from rest: f stays at w_i (Eq. 5 at u = 0, and
    Eq. 6 gives -w + 2 w = w), up to the rounding of sum_i w_i."""
    if q == 9:
        m, _ = O.geometry(9, 96, 48, kind=O.GEOM_DISKS, seed=5, r_min=4, r_max=7, porosity=0.7)
    else:
        m, _ = O.geometry(19, 32, 16, 16, kind=O.GEOM_SPHERES, seed=5, r_min=3, r_max=3, porosity=0.7)
    f = O.forward(q, m, 1.0, 1.0, 0.8, 30)
    w = O.lattice(q)[1].reshape((q,) + (1,) * m.ndim)
    fl = ~m.astype(bool)
    assert np.abs(f[:, fl] - np.broadcast_to(w, f.shape)[:, fl]).max() < 1e-15


def _steady_channel(ny, tau, L=8, tol=1e-12, chunk=2000, max_steps=200000):
    nx = L * ny
    m, _ = O.geometry(9, nx, ny)
    f, prev, steps = None, None, 0
    while steps < max_steps:
        f = O.forward(9, m, 1.001, 1.0, tau, chunk, f0=f)
        steps += chunk
        rho, u = O.macroscopic(9, m, f)
        if prev is not None and np.abs(u - prev).max() < tol:
            break
        prev = u
    return m, f, rho, u


def _poiseuille_error(ny, tau):
    m, f, rho, u = _steady_channel(ny, tau)
    nx = m.shape[1]
    xs = nx // 2
    y = np.arange(ny)
    nu = (tau - 0.5) / 3.0
    # local pressure gradient at mid-channel: dp/dx = c_s^2 drho/dx
    G = -(rho[:, xs + 1].mean() - rho[:, xs - 1].mean()) / 2.0 / 3.0
    ua = G / (2.0 * rho[:, xs].mean() * nu) * (y + 0.5) * (ny - 0.5 - y)
    return np.linalg.norm(u[0][:, xs] - ua) / np.linalg.norm(ua), (m, f, rho, u)


@pytest.mark.slow
def test_poiseuille_second_order_and_exact_tau():
    """Steady pressure-driven channel (walls at y = -1/2 and ny - 1/2):
    the mid-channel profile is the analytic Poiseuille parabola
    u(y) = G/(2 rho nu) (y + 1/2)(ny - 1/2 - y), nu = (tau - 1/2)/3 (Eq. 9),
    with second-order convergence, and BGK with halfway bounce-back is exact
    for Poiseuille flow at tau = 1/2 + sqrt(3/16)."""
    e8, _ = _poiseuille_error(8, 0.8)
    e16, (m, f, rho, u) = _poiseuille_error(16, 0.8)
    assert e16 < 5e-3
    assert 3.5 < e8 / e16 < 4.5
    e_magic, _ = _poiseuille_error(8, 0.5 + math.sqrt(3.0 / 16.0))
    assert e_magic < 1e-5 and e_magic < e8 / 100

    # mass: the steady column flux sum_y rho u_x is the same at every x
    J = (rho * u[0]).sum(0)
    assert (J.max() - J.min()) / J.mean() < 1e-7
    # pressure is uniform across the channel away from the ends
    nx = m.shape[1]
    assert np.ptp(rho[:, nx // 2]) < 1e-12
    # Eq. 6 imposes rho_in / rho_out at the planes x = -1/2 and nx - 1/2:
    # the bulk density line extrapolates to them within 1% of the drop
    xr = np.arange(nx // 4, 3 * nx // 4)
    p = np.polyfit(xr, rho.mean(0)[xr], 1)
    assert abs(np.polyval(p, -0.5) - 1.001) < 1e-5
    assert abs(np.polyval(p, nx - 0.5) - 1.0) < 1e-5

    # Darcy (Eq. 12) for a 2D channel of width H = ny: k = H^2 / 12
    k, _ = O.darcy(9, m, f, 1.001, 1.0, 0.8)
    assert abs(k - 16 * 16 / 12.0) / (16 * 16 / 12.0) < 0.02


def test_solid_nodes_report_zero():
    m, _ = O.geometry(9, 64, 32, kind=O.GEOM_DISKS, seed=2, r_min=4, r_max=6, porosity=0.75)
    f = O.forward(9, m, 1.001, 1.0, 0.8, 50)
    rho, u = O.macroscopic(9, m, f)
    s = m.astype(bool)
    assert np.all(u[:, s] == 0) and np.all(rho[s] == 0)
    assert np.all(rho[~s] > 0.99)


# ------------------------------------------------------------------- gradients


def _tiny(q):
    if q == 9:
        m = np.zeros((6, 8), np.uint8)
        m[3, 4] = 1
    else:
        m = np.zeros((5, 5, 6), np.uint8)
        m[2, 2, 3] = 1
    return m


def _tiny_target(q, m, seed):
    d = 2 if q == 9 else 3
    return W.perturbation((d,) + m.shape, seed=seed, scale=2e-3)


@pytest.mark.parametrize("kind", [O.LOSS_VEC, O.LOSS_NORM])
@pytest.mark.parametrize("norm", [O.NORM_SUM, O.NORM_MEAN_FLUID])
@pytest.mark.parametrize("q", [9, 19])
def test_loss_seed_matches_complex_step(q, kind, norm):
    """lam^T = dL/df^T against complex-step derivatives of the loss itself."""
    m = _tiny(q)
    f = O.forward(q, m, 1.002, 1.0, 0.8, 15)
    ut = _tiny_target(q, m, 21)
    roi = np.ones(m.shape, np.uint8)
    roi[..., :2] = 0
    L, lam = O.loss(q, m, f, ut, roi, kind, norm)
    h = 1e-30
    for s in range(3):
        v = W.perturbation(f.shape, seed=40 + s, scale=1.0)
        Lc = O.loss(q, m, f + 1j * h * v, ut, roi, kind, norm, seed=False, complex_step=True)
        assert abs(Lc.real - L) <= 1e-15 * abs(L)
        assert np.isclose(Lc.imag / h, np.sum(lam * v), rtol=1e-12, atol=0)


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("profile", [False, True])
def test_adjoint_step_is_transpose_of_step(q, profile):
    """Dot-product test of one reverse step: <lam, J df> = <J^T lam, df>,
    with J df taken by complex step of the forward step alone; likewise for
    the rho_in and tau directions."""
    m = _tiny(q)
    ny, nz = m.shape[-2], (m.shape[0] if q == 19 else 1)
    rho_in = 1.0 + (0.001 + W.perturbation((nz, ny) if q == 19 else (ny,), seed=5, scale=5e-4) if profile else 0.001)
    rho_out, tau = 1.0, 0.85
    f = O.forward(q, m, rho_in, rho_out, tau, 12)
    lam = W.perturbation(f.shape, seed=8, scale=1.0)
    lam[:, m.astype(bool)] = 0
    lam_t, g_in, g_om = O.adjoint_step(q, m, f, lam, rho_in, rho_out, tau)
    h = 1e-30
    df = W.perturbation(f.shape, seed=9, scale=1.0)
    df[:, m.astype(bool)] = 0
    jd = O.step(q, m, f + 1j * h * df, rho_in, rho_out, tau, complex_step=True).imag / h
    assert np.isclose(np.sum(lam * jd), np.sum(lam_t * df), rtol=1e-12, atol=0)
    # rho_in direction
    dr = W.perturbation(np.shape(rho_in), seed=10, scale=1.0) if profile else 1.0
    jr = O.step(q, m, f, np.asarray(rho_in) + 1j * h * np.asarray(dr), rho_out, tau, complex_step=True).imag / h
    assert np.isclose(np.sum(lam * jr), np.sum(np.ravel(g_in) * np.ravel(dr)), rtol=1e-12, atol=0)
    # tau direction: dL/dtau = -dL/domega / tau^2
    jt = O.step(q, m, f, rho_in, rho_out, tau + 1j * h, complex_step=True).imag / h
    assert np.isclose(np.sum(lam * jt), -g_om / tau ** 2, rtol=1e-12, atol=0)
    # solid nodes carry no adjoint
    assert np.all(lam_t[:, m.astype(bool)] == 0)


@pytest.mark.parametrize("q,T", [(9, 20), (19, 10)])
@pytest.mark.parametrize("profile", [False, True])
def test_gradient_matches_complex_step(q, T, profile):
    """Full reverse sweep against complex-step derivatives of forward + loss
    on tiny lattices (D2Q9 8x6 and D3Q19 6x5x5, one solid node each)."""
    m = _tiny(q)
    ny, nz = m.shape[-2], (m.shape[0] if q == 19 else 1)
    rho_in = 1.0 + (0.001 + W.perturbation((nz, ny) if q == 19 else (ny,), seed=15, scale=5e-4) if profile else 0.0015)
    rho_out, tau = 1.0, 0.8
    ut = _tiny_target(q, m, 16)
    L, g_in, g_tau = O.gradient(q, m, rho_in, rho_out, tau, T, ut)
    h = 1e-30

    def loss_c(rin, t):
        fT = O.forward(q, m, rin, rho_out, t, T, complex_step=True)
        return O.loss(q, m, fT, ut, seed=False, complex_step=True)

    if profile:
        flat = np.ravel(rho_in)
        for k in [0, flat.size // 2, flat.size - 1]:
            e = np.zeros(flat.size, np.complex128)
            e[k] = 1j * h
            d = loss_c((flat + e).reshape(np.shape(rho_in)), tau).imag / h
            assert np.isclose(np.ravel(g_in)[k], d, rtol=1e-11, atol=0)
    else:
        d = loss_c(rho_in + 1j * h, tau).imag / h
        assert np.isclose(g_in, d, rtol=1e-11, atol=0)
    d = loss_c(rho_in, tau + 1j * h).imag / h
    assert np.isclose(g_tau, d, rtol=1e-11, atol=0)
    assert np.isclose(loss_c(rho_in, tau).real, L, rtol=1e-15)


def test_gradient_matches_central_differences():
    q, T = 9, 30
    m = _tiny(q)
    ut = _tiny_target(q, m, 30)
    rho_in, rho_out, tau = 1.0012, 1.0, 0.9
    _, g_in, g_tau = O.gradient(q, m, rho_in, rho_out, tau, T, ut)

    def L(rin, t):
        return O.loss(q, m, O.forward(q, m, rin, rho_out, t, T), ut, seed=False)

    h = 1e-6 * rho_in
    fd = (L(rho_in + h, tau) - L(rho_in - h, tau)) / (2 * h)
    assert np.isclose(g_in, fd, rtol=1e-6)
    h = 1e-6 * tau
    fd = (L(rho_in, tau + h) - L(rho_in, tau - h)) / (2 * h)
    assert np.isclose(g_tau, fd, rtol=1e-6)


@pytest.mark.parametrize("stride", [1, 3, 7, 50])
def test_checkpointing_changes_nothing(stride):
    q, T = 9, 23
    m = _tiny(q)
    ut = _tiny_target(q, m, 31)
    rin = 1.0 + 0.001 + W.perturbation((6,), seed=32, scale=3e-4)
    full = O.gradient(q, m, rin, 1.0, 0.8, T, ut, ckpt_stride=0)
    ck = O.gradient(q, m, rin, 1.0, 0.8, T, ut, ckpt_stride=stride)
    assert full[0] == ck[0] and np.array_equal(full[1], ck[1]) and full[2] == ck[2]


def test_gradient_vanishes_at_the_truth():
    """A target made by a forward solve at theta*: L = 0 and grad = 0 exactly."""
    m, _ = O.geometry(9, 48, 24, kind=O.GEOM_DISKS, seed=12, r_min=3, r_max=5, porosity=0.75)
    rin = 1.0 + W.inlet_profile(24, seed=2)
    fT = O.forward(9, m, rin, 1.0, 0.8, 60)
    _, ut = O.macroscopic(9, m, fT)
    L, g_in, g_tau = O.gradient(9, m, rin, 1.0, 0.8, 60, ut, ckpt_stride=8)
    assert L == 0.0 and np.all(g_in == 0.0) and g_tau == 0.0


# ------------------------------------------------------------------ optimiser


def test_adam_constant_gradient_steps():
    """With a constant gradient g Adam's bias-corrected moments are exactly
    g and g^2, so every step moves theta by -lr g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    theta = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 0.02, 1e-8
    for t in range(1, 6):
        before = theta.copy()
        O.adam(theta, g, m, v, t, lr, eps=eps)
        assert np.allclose(theta - before, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)


# ------------------------------------------------------------------- geometry


def _sm64(state):
    M = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & M
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return state, z ^ (z >> 31)


def _py_geometry(d, nx, ny, nz, kind, seed, rmin, rmax, porosity, hydro, buf, max_rej):
    """Brute-force restatement of the geometry recipe (placement only)."""
    N = nx * ny * nz
    mask = np.zeros((nz, ny, nx), np.uint8)
    s = seed
    placed = []
    solid = 0
    target = int(porosity * N)
    rej = 0
    while N - solid > target and rej < max_rej:
        draws = []
        for n in ([256 * nx, 256 * ny] + ([256 * nz] if d == 3 else []) + [256 * (rmax - rmin) + 1]):
            s, z = _sm64(s)
            draws.append(((z >> 32) * n) >> 32)
        cx, cy = draws[0], draws[1]
        cz = draws[2] if d == 3 else 0
        r = 256 * rmin + draws[-1]
        ok = cx - r > 256 * (buf - 1) and cx + r < 256 * (nx - buf)
        if ok and kind == 1:
            ok = all((cx - a) ** 2 + (cy - b) ** 2 >= (r + rr + 256) ** 2 for a, b, rr in placed)
        if not ok:
            rej += 1
            continue
        placed.append((cx, cy, r))
        rv = (r * hydro) >> 8
        before = solid
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if (256 * x - cx) ** 2 + (256 * y - cy) ** 2 + ((256 * z - cz) ** 2 if d == 3 else 0) <= rv * rv:
                        if not mask[z, y, x]:
                            mask[z, y, x] = 1
                            solid += 1
        rej = 0 if solid > before else rej + 1
    return mask, len(placed)


@pytest.mark.parametrize("case", [
    (9, 40, 24, 1, 1, 77, 3, 5, 0.72, 256),
    (9, 40, 24, 1, 1, 78, 3, 5, 0.8, 230),
    (19, 20, 10, 10, 2, 79, 3, 3, 0.6, 256),
    (19, 20, 10, 10, 2, 80, 3, 3, 0.2, 256),  # unreachable target: stops on the no-progress streak
])
def test_geometry_matches_bruteforce(case):
    q, nx, ny, nz, kind, seed, rmin, rmax, por, hydro = case
    mask, info = O.geometry(q, nx, ny, nz, kind=kind, seed=seed, r_min=rmin, r_max=rmax, porosity=por,
                            hydro_q8=hydro, buffer=4, max_rejections=2000, fill=False)
    want, count = _py_geometry(2 if q == 9 else 3, nx, ny, nz, kind, seed, rmin, rmax, por, hydro, 4, 2000)
    assert np.array_equal(mask.reshape(want.shape), want)
    assert info[0] == count and info[1] == want.sum() and info[2] == 0


@pytest.mark.parametrize("q", [9, 19])
def test_flood_fill_matches_scipy_label(q):
    ndimage = pytest.importorskip("scipy.ndimage")
    if q == 9:
        args = dict(q=9, nx=96, ny=48, nz=1, kind=O.GEOM_DISKS, seed=17, r_min=3, r_max=8, porosity=0.55)
    else:
        args = dict(q=19, nx=32, ny=20, nz=20, kind=O.GEOM_SPHERES, seed=18, r_min=3, r_max=3, porosity=0.45,
                    buffer=3)
    raw, info0 = O.geometry(**args, fill=False)
    filled, info = O.geometry(**args, fill=True)
    fluid = raw == 0
    lab, _ = ndimage.label(fluid, structure=ndimage.generate_binary_structure(fluid.ndim, 1))
    keep = set(np.unique(lab[..., 0])) - {0}
    want = (~np.isin(lab, list(keep))).astype(np.uint8)
    assert np.array_equal(filled, want)
    assert info[2] == int(want.sum() - raw.sum())
    assert info[3] == int((want == 0).sum())


@pytest.mark.parametrize("q", [9, 19])
def test_link_words_bruteforce(q):
    if q == 9:
        m, _ = O.geometry(9, 30, 14, kind=O.GEOM_DISKS, seed=4, r_min=2, r_max=4, porosity=0.7, buffer=3)
    else:
        m, _ = O.geometry(19, 14, 8, 7, kind=O.GEOM_SPHERES, seed=4, r_min=2, r_max=2, porosity=0.75, buffer=3)
    link = O.links(q, m)
    c, _, _ = O.lattice(q)
    m3 = m.reshape((-1,) + m.shape[-2:]) if q == 19 else m[None]
    l3 = link.reshape(m3.shape)
    nz, ny, nx = m3.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if m3[z, y, x]:
                    assert l3[z, y, x] == (1 << 31)
                    continue
                want = 0
                for i in range(q):
                    sx, sy, sz = x - c[i][0], y - c[i][1], z - c[i][2]
                    if not (0 <= sy < ny and 0 <= sz < nz):
                        want |= 1 << i
                    elif 0 <= sx < nx and m3[sz, sy, sx]:
                        want |= 1 << i
                assert l3[z, y, x] == want


def test_disk_packing_config_properties():
    """The 512x256 disk packing (seed 1000): porosity 0.6 +- 0.005, buffer
    columns fluid, the same seed gives the same mask and another seed does not."""
    m, info = O.geometry(9, 512, 256, kind=O.GEOM_DISKS, seed=1000, r_min=6, r_max=12, porosity=0.6)
    por = 1.0 - m.mean()
    assert abs(por - 0.6) < 0.005
    assert not m[:, :8].any() and not m[:, -8:].any()
    m2, _ = O.geometry(9, 512, 256, kind=O.GEOM_DISKS, seed=1000, r_min=6, r_max=12, porosity=0.6)
    assert np.array_equal(m, m2)
    m3, _ = O.geometry(9, 512, 256, kind=O.GEOM_DISKS, seed=1001, r_min=6, r_max=12, porosity=0.6)
    assert not np.array_equal(m, m3)
    assert info[0] > 100


def test_thread_count_changes_nothing():
    """The OpenMP forward gives the same bits with 1 and 4 threads."""
    m, _ = O.geometry(9, 96, 48, kind=O.GEOM_DISKS, seed=8, r_min=3, r_max=6, porosity=0.7)
    O.set_threads(1)
    a = O.forward(9, m, 1.001, 1.0, 0.8, 40)
    O.set_threads(4)
    b = O.forward(9, m, 1.001, 1.0, 0.8, 40)
    O.set_threads(1)
    assert np.array_equal(a, b)


def test_thread_count_changes_nothing_in_gradient():
    """The OpenMP adjoint gives the same bits with 1 and 4 threads (constant head and profile)."""
    m, _ = O.geometry(9, 64, 32, kind=O.GEOM_DISKS, seed=5, r_min=3, r_max=5, porosity=0.7)
    rng = np.random.default_rng(3)
    ut = rng.normal(0, 1e-4, (2, 32, 64))
    for rin in (1.001, 1.0 + 1e-3 * rng.random(32)):
        out = []
        for th in (1, 4):
            O.set_threads(th)
            out.append(O.gradient(9, m, rin, 1.0, 0.8, 30, ut, ckpt_stride=6))
        O.set_threads(1)
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(np.asarray(a), np.asarray(b))
