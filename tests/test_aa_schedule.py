"""The in-place (AA-pattern) streaming schedule of the fluid-only kernels,
pinned on the CPU against the oracle's plain pull step.

The model below stores post-collision states g^t over the fluid nodes, in
one array, as the GPU kernels do: natural layout (slot (x, i) holds g_i(x))
for even t, swapped layout (g_i(x) at (x + c_i, opp(i)) where that node is
fluid, else at (x, i)) for odd t.  A step from the natural layout gathers
what each node receives through its neighbours and scatters its output
into the swapped layout; a step from the swapped layout reads and writes
each node's own slots.  Nodes are visited in a random order and every
update reads and writes the one array, so a schedule whose read and write
slots differed between nodes would give wrong populations here.  The
oracle's steps (f^{t+1} = stream(collide(f^t)), bounce-back at walls and
obstacles, the velocity inlet at u_in = 0 as plain bounce-back, periodic y)
give g^t = collide(f^t); the model must match them to rounding after every
step.  The same statement holds for the adjoint's lambda, whose layouts
stream the other way; its model is checked against the transpose of the
pull step built from the same neighbour table."""
import numpy as np
import pytest

from oracle import oracle as O


def _geometry(q, per_y, seed):
    rng = np.random.default_rng(seed)
    shape = (6, 7, 9) if q == 19 else (8, 11)
    m = (rng.random(shape) < 0.25).astype(np.uint8)
    m[..., :, -1] = 1  # no outlet links: every population that leaves comes back
    if not per_y:
        m[..., 0, :] = 1
        m[..., -1, :] = 1
    if q == 19:
        m[0] = 1
        m[-1] = 1
    return m


def _table(q, m, per_y):
    """pull[k, i]: compact index of x - c_i, or -1 where the population comes back."""
    c, _, _ = O.lattice(q)
    fluid = np.argwhere(m == 0)  # (z, y, x) or (y, x), node order
    index = -np.ones(m.shape, np.int64)
    index[tuple(fluid.T)] = np.arange(len(fluid))
    pull = -np.ones((len(fluid), q), np.int64)
    for k, node in enumerate(fluid):
        for i in range(q):
            if i == 0:
                pull[k, i] = k
                continue
            src = list(node)
            for a in range(len(node)):
                comp = len(node) - 1 - a  # array axis a holds component comp (x is last)
                src[a] = node[a] - c[i][comp]
            ny = m.shape[-2]
            if per_y:
                src[-2] %= ny
            if any(s < 0 or s >= m.shape[a] for a, s in enumerate(src)) or m[tuple(src)]:
                continue
            pull[k, i] = index[tuple(src)]
    return fluid, pull


def _collide_node(q, f, tau):
    return O.collide(q, f.reshape(q, 1), tau)[:, 0]


def _aa_forward(q, g0, pull, T, tau, rng):
    """T in-place steps from the natural state g0 [Q, nf]; returns the array after each step."""
    _, _, opp = O.lattice(q)
    nf = g0.shape[1]
    A = g0.copy()
    # where x + c_i lives: x + c_i = x - c_opp(i)
    push = pull[:, opp]
    out = []
    for t in range(1, T + 1):
        for k in rng.permutation(nf):
            if t % 2 == 1:  # natural -> swapped: gather, then scatter
                f = np.array([A[i, pull[k, i]] if pull[k, i] >= 0 else A[opp[i], k] for i in range(q)])
                g = _collide_node(q, f, tau)
                for i in range(q):
                    if push[k, i] >= 0:
                        A[opp[i], push[k, i]] = g[i]
                    else:
                        A[i, k] = g[i]
            else:  # swapped -> natural: own slots only
                f = np.array([A[opp[i], k] for i in range(q)])
                A[:, k] = _collide_node(q, f, tau)
        out.append(A.copy())
    return out


def _unswap(q, A, pull):
    """The natural layout of a swapped forward state."""
    _, _, opp = O.lattice(q)
    push = pull[:, opp]
    nf = A.shape[1]
    g = np.empty_like(A)
    for k in range(nf):
        for i in range(q):
            g[i, k] = A[opp[i], push[k, i]] if push[k, i] >= 0 else A[i, k]
    return g


@pytest.mark.parametrize("q,per_y", [(9, True), (9, False), (19, True), (19, False)])
def test_in_place_forward_schedule_matches_the_pull_step(q, per_y):
    m = _geometry(q, per_y, seed=3 + q)
    fluid, pull = _table(q, m, per_y)
    rng = np.random.default_rng(11)
    _, w, _ = O.lattice(q)
    f0 = w.reshape((q,) + (1,) * m.ndim) * (1.0 + 0.05 * rng.standard_normal((q, *m.shape)))
    f0[:, m == 1] = 0.0
    tau = 0.8
    sel = (slice(None),) + tuple(fluid.T)
    g0 = O.collide(q, f0, tau)[sel]
    T = 5
    states = _aa_forward(q, g0, pull, T, tau, rng)
    f = f0
    with O.wake_options(periodic_y=per_y, velocity_inlet=(0.0, 0.0, 0.0) if q == 19 else (0.0, 0.0)):
        for t in range(1, T + 1):
            f = O.step(q, m, f, 1.0, 1.0, tau)
            want = O.collide(q, f, tau)[sel]
            got = states[t - 1] if t % 2 == 0 else _unswap(q, states[t - 1], pull)
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-14, err_msg=f"step {t}")


def test_swapped_layout_puts_what_a_node_receives_in_its_own_slots():
    """In the swapped layout of g^t, slot (x, opp(i)) holds exactly the
    population x receives in direction i at step t + 1."""
    q = 9
    m = _geometry(q, True, seed=5)
    fluid, pull = _table(q, m, True)
    _, _, opp = O.lattice(q)
    rng = np.random.default_rng(2)
    g = rng.standard_normal((q, len(fluid)))
    push = pull[:, opp]
    A = np.full_like(g, np.nan)
    for k in range(len(fluid)):
        for i in range(q):
            if push[k, i] >= 0:
                A[opp[i], push[k, i]] = g[i, k]
            else:
                A[i, k] = g[i, k]
    assert not np.isnan(A).any()  # the scatter covers every slot once
    for k in range(len(fluid)):
        for i in range(q):
            want = g[i, pull[k, i]] if pull[k, i] >= 0 else g[opp[i], k]
            assert A[opp[i], k] == want


def test_in_place_adjoint_schedule_is_the_transpose_pull():
    """The reverse sweep's lambda layouts: a linear stand-in for the adjoint
    collision (a fixed Q x Q matrix B per node) run through the gather step
    (natural in, lambda_m(x) scattered to (x - c_m, opp(m))) and the local
    step (swapped in, own slots out) in random node order on one array
    equals the plain two-buffer transpose: lambda^t(x) = B mu(x) with
    mu_j(x) = lambda^{t+1}_j(x + c_j), or lambda^{t+1}_opp(j)(x) where the
    population came back."""
    q = 19
    m = _geometry(q, True, seed=8)
    fluid, pull = _table(q, m, True)
    _, _, opp = O.lattice(q)
    rng = np.random.default_rng(4)
    nf = len(fluid)
    B = rng.standard_normal((q, q))
    lam = rng.standard_normal((q, nf))
    push = pull[:, opp]

    def reference(l):
        mu = np.empty_like(l)
        for k in range(nf):
            for j in range(q):
                mu[j, k] = l[j, push[k, j]] if push[k, j] >= 0 else l[opp[j], k]
        return B @ mu

    A = lam.copy()
    want = lam.copy()
    for step in range(4):
        want = reference(want)
        for k in rng.permutation(nf):
            if step % 2 == 0:  # natural -> swapped
                mu = np.array([A[j, push[k, j]] if push[k, j] >= 0 else A[opp[j], k] for j in range(q)])
                out = B @ mu
                for mm in range(q):
                    if pull[k, mm] >= 0 and mm > 0:
                        A[opp[mm], pull[k, mm]] = out[mm]
                    else:
                        A[mm, k] = out[mm]
            else:  # swapped -> natural
                mu = np.array([A[opp[j], k] for j in range(q)])
                A[:, k] = B @ mu
        if step % 2 == 1:
            np.testing.assert_allclose(A, want, rtol=1e-12, atol=1e-12)
        else:  # swapped: lambda_m(x) sits at (x - c_m, opp(m)) where that node is fluid
            nat = np.empty_like(A)
            for k in range(nf):
                for mm in range(q):
                    nat[mm, k] = A[opp[mm], pull[k, mm]] if (mm > 0 and pull[k, mm] >= 0) else A[mm, k]
            np.testing.assert_allclose(nat, want, rtol=1e-12, atol=1e-12)
