"""The host L-BFGS driver of the inversions (invert.lbfgs) on closed-form
objectives (CPU): exact line steps on a quadratic, the bound that keeps tau
above 1/2, and recovery from non-finite trial points."""
import numpy as np
import pytest

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


def _problem():
    r = np.random.Generator(np.random.PCG64(7))
    n = 5
    Q = r.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = r.normal(size=n)

    def ev(x):  # a quadratic plus a quartic term: several iterations, not exact after n
        return 0.5 * x @ A @ x - b @ x + 0.05 * np.sum(x ** 4), A @ x - b + 0.2 * x ** 3

    return ev, n


def test_iteration_log_writes_one_json_line_per_iteration(tmp_path):
    import json

    ev, n = _problem()
    path = str(tmp_path / "log.jsonl")
    res = I.lbfgs(ev, np.zeros(n), max_evals=30, errors=lambda x: (float(np.linalg.norm(x)), None),
                  callback=I.IterationLog(path))
    lines = [json.loads(l) for l in open(path)]
    assert [l["iteration"] for l in lines] == list(range(1, res.iterations + 1))
    assert lines[-1]["loss"] == res.losses[-1] and len(lines[-1]["x"]) == n


def test_checkpoint_resume_after_an_injected_failure_is_exact(tmp_path):
    """A run that fails (host-side injection) after 11 evaluations, resumed
    from its last checkpoint, ends at the same point, bit for bit, as a run
    that never failed."""
    ev, n = _problem()
    kw = dict(max_evals=60, errors=lambda x: (float(np.linalg.norm(ev(x)[1])), None), done=lambda e: e[0] < 1e-12)
    whole = I.lbfgs(ev, np.zeros(n), **kw)
    path = str(tmp_path / "ckpt.npz")
    try:
        I.lbfgs(I.inject_failures(ev, after=11), np.zeros(n), callback=I.Checkpoint(path), **kw)
        assert False, "the injected failure did not fire"
    except I.InjectedFailure:
        pass
    x, history, it, evals = I.Checkpoint.load(path)
    assert 0 < it and evals <= 11
    rest = I.lbfgs(ev, x, history=history, **kw)
    assert whole.converged and rest.converged
    assert np.array_equal(rest.x, whole.x)


def test_injection_reads_the_environment(monkeypatch):
    ev, n = _problem()
    assert I.inject_failures(ev) is ev
    monkeypatch.setenv("LBM_INJECT_FAIL_AFTER", "2")
    f = I.inject_failures(ev)
    f(np.zeros(n))
    f(np.zeros(n))
    try:
        f(np.zeros(n))
        assert False
    except I.InjectedFailure:
        pass


def test_adam_state_round_trip(tmp_path):
    """The Adam inversion's state (theta, moments, step count, derived rho_in
    and tau) saves and restores exactly; host-only, with a stand-in solver."""
    import types

    import torch

    plan = types.SimpleNamespace(n_in=6, ny=6, nz=1)
    solver = types.SimpleNamespace(plan=plan, device=torch.device("cpu"),
                                   new_state=lambda: torch.zeros((9, 6, 12), dtype=torch.float64))
    inv = I.Inversion(solver, torch.zeros((2, 6, 12), dtype=torch.float64), 1.0, theta0=0.3, tau0=0.9,
                      invert_tau=True)
    r = np.random.Generator(np.random.PCG64(1))
    for k in ("theta", "m", "v", "theta_tau", "m_tau", "v_tau", "rho_in", "tau"):
        getattr(inv, k).copy_(torch.as_tensor(r.normal(size=getattr(inv, k).shape)))
    inv.t = 17
    path = str(tmp_path / "adam.pt")
    inv.save(path)
    other = I.Inversion(solver, torch.zeros((2, 6, 12), dtype=torch.float64), 1.0)
    other.load(path)
    assert other.t == 17
    for k in ("theta", "m", "v", "theta_tau", "m_tau", "v_tau", "rho_in", "tau"):
        assert torch.equal(getattr(other, k), getattr(inv, k)), k


def test_lockstep_runs_equal_independent_runs():
    """lbfgs_lockstep over several problems takes, per problem, exactly the
    steps of an independent lbfgs run (same points, same evaluation count),
    whatever the other problems do (they stop at different rounds)."""
    rng = np.random.default_rng(7)
    probs = []
    for n in (3, 5, 8, 4):
        A = rng.standard_normal((n, n))
        H = A @ A.T + n * np.eye(n) * (0.2 + rng.random())
        b = rng.standard_normal(n)
        probs.append((H, b, np.linalg.solve(H, b)))

    def single(i):
        H, b, _ = probs[i]
        return lambda x: (0.5 * x @ H @ x - b @ x, H @ x - b)

    def errors(i):
        return lambda x: (float(np.linalg.norm(x - probs[i][2]) / np.linalg.norm(probs[i][2])), None)

    done = [lambda e: e[0] <= 1e-10] * len(probs)
    x0s = [np.zeros(len(p[1])) for p in probs]
    rounds = []

    def batch(req):
        rounds.append(sorted(req))
        return {i: single(i)(x) for i, x in req.items()}

    got = I.lbfgs_lockstep(batch, x0s, errors=[errors(i) for i in range(len(probs))], done=done, max_evals=200)
    for i in range(len(probs)):
        want = I.lbfgs(single(i), x0s[i], errors=errors(i), done=done[i], max_evals=200)
        assert got[i].converged and want.converged
        assert got[i].evaluations == want.evaluations
        assert np.array_equal(got[i].x, want.x)
        assert got[i].losses == want.losses
    assert len(rounds) == max(r.evaluations for r in got)
    assert len(rounds[-1]) < len(probs)  # the smaller problems finished earlier


def test_lockstep_reports_an_evaluation_failure():
    def batch(req):
        raise I.InjectedFailure("device lost")

    with pytest.raises(I.InjectedFailure):
        I.lbfgs_lockstep(batch, [np.zeros(2), np.zeros(3)], max_evals=10)
