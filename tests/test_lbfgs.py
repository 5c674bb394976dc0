"""The host L-BFGS driver of the inversions (invert.lbfgs) on closed-form
objectives (CPU): exact line steps on a quadratic, the bound that keeps tau
above 1/2, and recovery from non-finite trial points."""
import numpy as np

from paper_2310_00810_gb300 import invert as I


def _quadratic(A, b):
    def ev(x):
        return 0.5 * x @ A @ x - b @ x, A @ x - b
    return ev


def test_quadratic_converges_in_a_few_iterations():
    r = np.random.Generator(np.random.PCG64(1))
    n = 6
    Q = r.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = r.normal(size=n)
    xs = np.linalg.solve(A, b)
    res = I.lbfgs(_quadratic(A, b), np.zeros(n), max_evals=60,
                  errors=lambda x: (np.linalg.norm(x - xs) / np.linalg.norm(xs), None),
                  done=lambda e: e[0] < 1e-10)
    assert res.converged and res.iterations <= n + 2
    assert all(l1 <= l0 + 1e-12 for l0, l1 in zip(res.losses, res.losses[1:]))


def test_bound_keeps_the_stiff_coordinate_valid():
    """A stretched valley along the second coordinate (as probes make along
    tau) invites a huge secant step; beyond x1 < 0 the 'lattice' is unstable
    (NaN).  The bound stops the step at x1 = 0.05 and the run still converges."""
    def ev(x):
        if x[1] < 0:
            return np.nan, np.full(2, np.nan)
        a, e = 1e4, 1e-4
        return a * (x[0] - 1) ** 2 + e * (x[1] - 3) ** 2 + 50 * e * (x[0] - 1) * (x[1] - 3), \
            np.array([2 * a * (x[0] - 1) + 50 * e * (x[1] - 3), 2 * e * (x[1] - 3) + 50 * e * (x[0] - 1)])

    seen = []

    def errors(x):
        seen.append(x.copy())
        return abs(x[0] - 1), abs(x[1] - 3) / 3

    res = I.lbfgs(ev, np.array([0.0, 5.0]), max_evals=200, errors=errors, done=lambda e: max(e) < 1e-6,
                  lower={1: 0.05})
    assert res.converged
    assert all(np.isfinite(l) for l in res.losses)
    assert min(x[1] for x in seen) >= 0.05 - 1e-12


def test_non_finite_trials_are_halved_away():
    """A loss that is NaN outside |x| < 2 (no bound given): every accepted
    point stays finite and the minimum is found."""
    def ev(x):
        if np.any(np.abs(x) >= 2):
            return np.nan, np.full(x.shape, np.nan)
        return float(np.sum((x - 1.5) ** 2) + 0.1 * np.sum(x ** 4)), 2 * (x - 1.5) + 0.4 * x ** 3

    root = [z.real for z in np.roots([0.4, 0.0, 2.0, -3.0]) if abs(z.imag) < 1e-12][0]
    x_star = np.full(3, root)  # the real root of 2 (x - 1.5) + 0.4 x^3 = 0
    res = I.lbfgs(ev, np.array([-1.9, 0.0, 1.9]), max_evals=200,
                  errors=lambda x: (float(np.max(np.abs(x - x_star))), None), done=lambda e: e[0] < 1e-9)
    assert res.converged and all(np.isfinite(l) for l in res.losses)
