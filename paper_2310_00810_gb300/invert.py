"""Gradient-based inversion of the inlet boundary condition (and tau) from an
observed velocity field: the optimisation loop of the paper (section 2.2 and
section 3), driven through the library's device kernels.

Two optimisers share the same gradient evaluation: Adam (the paper's, run by
the ``lbm_adam_step`` kernel, no host round trip per iteration) and L-BFGS
(``run_lbfgs``: two-loop recursion on the host over the short parameter
vector, with a secant step along each search direction).  In the Stokes
regime of these flows the velocity is nearly linear in the inlet density, so
the loss is nearly quadratic and L-BFGS needs far fewer gradient evaluations
than Adam's per-coordinate steps on a many-entry profile.

Each iteration is one gradient evaluation (``lbm_forward``, ``lbm_loss_grad``,
``lbm_adjoint``) followed by Adam updates (``lbm_adam_step``) of scaled
parameters, all enqueued on the solver's stream:
  inlet:  rho_in = rho_out + 1e-3 * theta          (theta ~ 1 for the 1e-3 heads)
  tau:    tau    = 0.5 + 0.1 * theta_tau            (so nu = theta_tau / 30)
The host reads back only the small parameter vector when it checks the stop
rule.  ``truth`` (optional) turns on the relative-error stop used for
time-to-target measurements: |delta - delta*| / |delta*| on delta = rho_in -
rho_out, and |nu - nu*| / |nu*| for tau.

Also here: the pure L-BFGS routine ``lbfgs`` (any evaluation function), its
lock-step form over many independent problems ``lbfgs_lockstep`` and the
batched inversion ``BatchInversion`` (one batched gradient evaluation serves
every instance's L-BFGS), the density-probe and spline-knot variants of the
inversion, ``SnapshotSeries``
(a loss over several observation times), and host-side recovery helpers:
``IterationLog`` (JSON lines), ``Checkpoint`` (exact resume), Adam state
``save``/``load`` and ``inject_failures`` (fault injection for tests).
"""
from __future__ import annotations

import dataclasses
import threading
import time

import numpy as np
import torch

from . import lbm

INLET_SCALE = 1e-3
TAU_OFFSET, TAU_SCALE = 0.5, 0.1
TAU_MIN_THETA = 0.05  # the L-BFGS steps keep tau >= 0.505


@dataclasses.dataclass
class InversionResult:
    iterations: int
    seconds: float
    converged: bool
    rho_in: np.ndarray
    tau: float
    rel_err_inlet: float | None
    rel_err_nu: float | None
    loss_history: list
    err_history: list


class IterationLog:
    """An lbfgs callback writing one JSON line per iteration (iteration,
    evaluations, seconds, loss, error record, and x when it is short)."""

    def __init__(self, path: str, max_x: int = 64):
        self.path, self.max_x = path, max_x

    def __call__(self, state: dict) -> None:
        import json

        rec = {k: state[k] for k in ("iteration", "evaluations", "seconds", "loss")}
        rec["error"] = None if state["error"] is None else [None if v is None else float(v) for v in state["error"]]
        if state["x"].size <= self.max_x:
            rec["x"] = [float(v) for v in state["x"]]
        with open(self.path, "a") as fh:
            fh.write(json.dumps(rec) + "\n")


class Checkpoint:
    """An lbfgs callback saving the resumable state (x and the curvature pairs)
    every `every` iterations to `path` (npz, written to a temporary file then
    renamed, so a crash never leaves a torn file); Checkpoint.load(path)
    returns (x, history, iteration, evaluations) for lbfgs(x0=x, history=history)."""

    def __init__(self, path: str, every: int = 1):
        self.path, self.every = path, every

    def __call__(self, state: dict) -> None:
        import os

        if state["iteration"] % self.every:
            return
        tmp = self.path + ".tmp.npz"
        n = state["x"].size
        pairs = lambda vs: np.array(vs, np.float64).reshape(len(vs), n) if vs else np.zeros((0, n))
        np.savez(tmp, x=state["x"], S=pairs(state["S"]), Y=pairs(state["Y"]), iteration=state["iteration"],
                 evaluations=state["evaluations"])
        os.replace(tmp, self.path)

    @staticmethod
    def load(path: str):
        with np.load(path) as z:
            return z["x"], (list(z["S"]), list(z["Y"])), int(z["iteration"]), int(z["evaluations"])


class InjectedFailure(RuntimeError):
    """Raised by a fault-injecting evaluation (LBM_INJECT_FAIL_AFTER)."""


def inject_failures(evaluate, after: int | None = None):
    """Host-side fault injection for recovery tests: the returned evaluation
    raises InjectedFailure on its call number `after` + 1 (default: the
    LBM_INJECT_FAIL_AFTER environment variable; unset, evaluate is returned
    unchanged).  Nothing is injected on the GPU."""
    import os

    if after is None:
        env = os.environ.get("LBM_INJECT_FAIL_AFTER")
        if env is None:
            return evaluate
        after = int(env)
    count = [0]

    def wrapped(x):
        count[0] += 1
        if count[0] > after:
            raise InjectedFailure(f"injected failure at evaluation {count[0]}")
        return evaluate(x)

    return wrapped


class SnapshotSeries:
    """A loss summed over velocity snapshots at steps t_1 < ... < t_K (the wake
    of section 3.4 observed over time rather than at one instant):
        L = sum_k L_k(u(t_k)),  L_k the plan's final-step loss against u_k on the ROI.
    Its gradient is the sum of the K single-snapshot gradients, each one
    checkpointed sweep of t_k steps through the library (cost sum_k t_k steps;
    the seeds are not injected into one shared reverse sweep).
    make_solver(t) returns a solver of t steps with the geometry and options
    of the problem; targets[k] is u_k (float64 [D, ...])."""

    def __init__(self, make_solver, times, targets, roi=None):
        if len(times) != len(targets) or not len(times):
            raise ValueError("one target per snapshot time")
        self.solvers = [make_solver(int(t)) for t in times]
        self.targets = [u.contiguous() for u in targets]
        self.roi = roi

    def loss_and_grad(self, rho_in, tau, rho_out: float):
        """(L, dL/drho_in, dL/dtau) as float64 tensors on the device."""
        L = g_in = g_tau = None
        for s, ut in zip(self.solvers, self.targets):
            f = s.forward(rho_in, tau, rho_out)
            l, lam = s.loss_grad(f, ut, self.roi)
            gi, gt = s.adjoint(rho_in, tau, rho_out, lam)
            L, g_in, g_tau = (l, gi, gt) if L is None else (L + l, g_in + gi, g_tau + gt)
        return L, g_in, g_tau


@dataclasses.dataclass
class LbfgsResult:
    x: np.ndarray
    iterations: int
    evaluations: int
    seconds: float
    converged: bool
    losses: list
    errs: list


def lbfgs(evaluate, x0, max_evals=400, memory=20, errors=None, done=None, lower=None, time_limit=None,
          callback=None, history=None):
    """Limited-memory BFGS (two-loop recursion) with a secant step along each
    direction, exact for a quadratic loss.  evaluate(x) -> (loss, gradient);
    errors(x) -> a record stored per iteration and done(record) -> stop;
    lower = {index: bound} keeps those coordinates above their bounds (the
    step is shortened to reach at most the bound).  A secant point is taken
    only if it lowers the loss, and a step whose loss is non-finite or larger
    is halved until it is not; a non-finite loss that halving cannot cure
    ends the run.
    callback(state) runs after every iteration with a dict of the iteration,
    evaluations, seconds, loss, error record, x and the curvature pairs S, Y;
    history = (S, Y) from such a state resumes a run at its x exactly."""
    t_start = time.perf_counter()
    x = np.array(x0, np.float64)
    f, g = evaluate(x)
    evals = 1
    S, Y, losses, errs = [], [], [f], []
    if history is not None:
        S, Y = [np.array(v, np.float64) for v in history[0]], [np.array(v, np.float64) for v in history[1]]
    converged = False
    it = 0
    while evals < max_evals:
        it += 1
        q = g.copy()
        alphas = []
        for sv, yv in reversed(list(zip(S, Y))):
            a = sv @ q / (yv @ sv)
            alphas.append(a)
            q -= a * yv
        gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]) if S else 1.0 / max(np.linalg.norm(g), 1e-300)
        r = gamma * q
        for (sv, yv), a in zip(zip(S, Y), reversed(alphas)):
            b = yv @ r / (yv @ sv)
            r += sv * (a - b)
        d = -r
        d0 = g @ d
        if d0 >= 0:  # not a descent direction: restart from steepest descent
            S, Y = [], []
            d = -g / max(np.linalg.norm(g), 1e-300)
            d0 = g @ d
        t_max = np.inf
        for i, lo in (lower or {}).items():
            if d[i] < 0:
                t_max = min(t_max, max((x[i] - lo) / -d[i], 0.0))
        t = min(1.0, t_max)
        f1, g1 = evaluate(x + t * d)
        evals += 1
        d1 = g1 @ d
        if np.isfinite(f1) and d1 > d0:  # secant step on the directional derivative
            t_new = min(-d0 / (d1 - d0) * t, t_max)
            if abs(t_new - t) > 1e-12 * t and evals < max_evals:
                f2, g2 = evaluate(x + t_new * d)
                evals += 1
                if np.isfinite(f2) and f2 <= f1:
                    t, f1, g1 = t_new, f2, g2
        while not (np.isfinite(f1) and f1 <= f + 1e-6 * abs(f)) and evals < max_evals and t > 1e-6:
            t *= 0.5
            f1, g1 = evaluate(x + t * d)
            evals += 1
        if not np.isfinite(f1):
            break
        sv, yv = t * d, g1 - g
        if yv @ sv > 0:
            S.append(sv)
            Y.append(yv)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        x, f, g = x + sv, f1, g1
        losses.append(f)
        e = errors(x) if errors is not None else None
        if e is not None:
            errs.append(e)
        if callback is not None:
            callback({"iteration": it, "evaluations": evals, "seconds": time.perf_counter() - t_start, "loss": f,
                      "error": e, "x": x.copy(), "S": [v.copy() for v in S], "Y": [v.copy() for v in Y]})
        if e is not None and done is not None and done(e):
            converged = True
            break
        if time_limit is not None and time.perf_counter() - t_start > time_limit:
            break
    return LbfgsResult(x, it, evals, time.perf_counter() - t_start, converged, losses, errs)



def lbfgs_lockstep(evaluate_batch, x0s, errors=None, done=None, **kw) -> list:
    """Independent L-BFGS runs (lbfgs, unchanged) over many problems in lock
    step: every round, each unfinished run has asked for one point, and a
    single call evaluate_batch({i: x_i}) -> {i: (loss_i, grad_i)} evaluates
    them all (one batched gradient evaluation of a batch of lattices).  Each
    run takes exactly the steps it would take alone with the same
    evaluations.  errors / done: one function per run (or None); the other
    keyword arguments go to every lbfgs (a time_limit is a shared deadline).
    Returns one LbfgsResult per problem."""
    n = len(x0s)
    cond = threading.Condition()
    pending: dict = {}
    answers: dict = {}
    running = set(range(n))
    failure: list = []
    outs: list = [None] * n

    def make_eval(i):
        def ev(x):
            with cond:
                pending[i] = np.array(x, np.float64)
                cond.notify_all()
                cond.wait_for(lambda: i in answers or failure)
                if failure:
                    raise RuntimeError("batched evaluation failed") from failure[0]
                return answers.pop(i)

        return ev

    def worker(i):
        try:
            outs[i] = lbfgs(make_eval(i), x0s[i], errors=None if errors is None else errors[i],
                            done=None if done is None else done[i], **kw)
        except BaseException as e:  # noqa: BLE001 - reported to the coordinator
            with cond:
                failure.append(e)
        finally:
            with cond:
                running.discard(i)
                cond.notify_all()

    threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(n)]
    for t in threads:
        t.start()
    while True:
        with cond:
            cond.wait_for(lambda: failure or all(i in pending for i in running))
            if failure or not running:
                break
            req = dict(pending)
            pending.clear()
        try:
            res = evaluate_batch(req)
        except BaseException as e:  # noqa: BLE001
            with cond:
                failure.append(e)
                cond.notify_all()
            break
        with cond:
            answers.update(res)
            cond.notify_all()
    for t in threads:
        t.join()
    if failure:
        raise failure[0]
    return outs


class BatchInversion:
    """L-BFGS inversions of every instance of a batch (lbm.Batch): the inlet
    density profile (or constant head) of each instance from its observed
    velocity field, with tau fixed per instance.  Each instance runs its own
    lbfgs on the scaled parameters (as Inversion.run_lbfgs), in lock step; a
    round is one batched forward + loss + checkpointed adjoint of all
    instances (instances that are done keep their last point)."""

    def __init__(self, batch, u_target, rho_out: float, tau, theta0=None):
        self.b, self.rho_out = batch, float(rho_out)
        self.u_target = u_target.contiguous()
        dev = batch.device
        self.tau = torch.as_tensor(np.broadcast_to(np.asarray(tau, np.float64), (batch.n,)).copy(), device=dev)
        self.n_in = [int(batch.view_inlet(batch.new_inlet(), i).numel()) for i in range(batch.n)]
        self.theta0 = [np.zeros(k) if theta0 is None else np.asarray(theta0[i], np.float64).copy()
                       for i, k in enumerate(self.n_in)]
        self.x = [t.copy() for t in self.theta0]
        self.rho_in = batch.new_inlet()
        self.f = batch.new_state()
        self.lam = batch.new_state()
        self.loss = torch.zeros(batch.n, dtype=torch.float64, device=dev)
        self.g_in = batch.new_inlet()
        self.g_tau = torch.zeros(batch.n, dtype=torch.float64, device=dev)
        self.rounds = 0

    def _evaluate(self, req: dict) -> dict:
        b = self.b
        for i, x in req.items():
            self.x[i] = x
        rho = np.zeros(int(b.inlet_off[-1]))
        for i in range(b.n):
            o = int(b.inlet_off[i])
            rho[o:o + self.n_in[i]] = self.rho_out + INLET_SCALE * self.x[i]
        with torch.cuda.stream(b.stream):
            self.rho_in.copy_(torch.from_numpy(rho), non_blocking=False)
        b.forward(self.rho_in, self.tau, self.rho_out, self.f)
        b.loss_grad(self.f, self.u_target, None, self.loss, self.lam)
        b.adjoint(self.rho_in, self.tau, self.rho_out, self.lam, self.g_in, self.g_tau)
        b.stream.synchronize()
        self.rounds += 1
        L = self.loss.cpu().numpy()
        g = self.g_in.cpu().numpy()
        out = {}
        for i in req:
            o = int(b.inlet_off[i])
            out[i] = (float(L[i]), g[o:o + self.n_in[i]] * INLET_SCALE)
        return out

    def run_lbfgs(self, truth_delta=None, tol: float = 1e-3, max_evals: int = 400, memory: int = 20,
                  time_limit: float | None = None) -> dict:
        """Every instance to `tol` relative error on delta (truth_delta: one
        array per instance) or max_evals / time_limit.  Returns the per-
        instance results, the rounds (batched evaluations) and the seconds."""
        n = self.b.n
        td = [None] * n if truth_delta is None else [np.asarray(t, np.float64) for t in truth_delta]
        errors = [None if td[i] is None else
                  (lambda x, t=td[i]: (float(np.linalg.norm(INLET_SCALE * x - t) / np.linalg.norm(t)), None))
                  for i in range(n)]
        done = [lambda e: e[0] <= tol] * n
        torch.cuda.synchronize(self.b.device)
        t0 = time.perf_counter()
        res = lbfgs_lockstep(self._evaluate, self.theta0, errors=errors, done=done, max_evals=max_evals,
                             memory=memory, time_limit=time_limit)
        secs = time.perf_counter() - t0
        return {"results": res, "rounds": self.rounds, "seconds": secs,
                "converged": all(r.converged for r in res),
                "rel_err": [r.errs[-1][0] if r.errs else None for r in res],
                "evaluations": [r.evaluations for r in res]}

class Inversion:
    """Adam inversion of the inlet density (constant head or profile) and,
    optionally, tau, against a target velocity field."""

    def __init__(self, solver: lbm.Solver, u_target, rho_out: float, theta0=None, tau0: float = 0.8,
                 invert_tau: bool = False, lr: float = 0.02, lr_tau: float = 0.01, roi=None, probes=None,
                 spline=None):
        p = solver.plan
        dev = solver.device
        # spline = (Ky, Kz): run_lbfgs inverts the knot values of a cubic-spline profile
        # (lbm_spline_profile / lbm_spline_grad) instead of one density per inlet node
        self.spline = None
        if spline is not None:
            ky, kz = int(spline[0]), int(spline[1])
            by, bz = lbm.lbm_spline_basis(ky, p.ny), lbm.lbm_spline_basis(kz, p.nz)
            self.spline = (torch.as_tensor(by, device=dev), torch.as_tensor(bz, device=dev), np.kron(bz, by))
            self.knots = torch.zeros(ky * kz, dtype=torch.float64, device=dev)
            self.g_knots = torch.zeros(ky * kz, dtype=torch.float64, device=dev)
        self.s, self.rho_out, self.invert_tau = solver, float(rho_out), invert_tau
        self.u_target = u_target.contiguous()
        self.roi = roi
        # probes = (node indices int64, observed densities float64, weight): the density-probe loss term
        self.probes = probes
        self.lr, self.lr_tau = lr, lr_tau
        t0 = np.zeros(p.n_in) if theta0 is None else np.broadcast_to(np.asarray(theta0, np.float64), (p.n_in,))
        self.theta = torch.tensor(np.array(t0), dtype=torch.float64, device=dev)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.rho_in = (self.rho_out + INLET_SCALE * self.theta).contiguous()
        th_tau = (tau0 - TAU_OFFSET) / TAU_SCALE
        self.theta_tau = torch.tensor([th_tau], dtype=torch.float64, device=dev)
        self.m_tau = torch.zeros_like(self.theta_tau)
        self.v_tau = torch.zeros_like(self.theta_tau)
        self.tau = torch.tensor([tau0], dtype=torch.float64, device=dev)
        self.f = solver.new_state()
        self.lam = solver.new_state()
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.g_in = torch.zeros(p.n_in, dtype=torch.float64, device=dev)
        self.g_tau = torch.zeros(1, dtype=torch.float64, device=dev)
        self.t = 0

    def state_dict(self) -> dict:
        """The Adam inversion's resumable state (host copies)."""
        keys = ("theta", "m", "v", "theta_tau", "m_tau", "v_tau", "rho_in", "tau")
        d = {k: getattr(self, k).detach().cpu().clone() for k in keys}
        d["t"] = self.t
        return d

    def load_state_dict(self, d: dict) -> None:
        for k in ("theta", "m", "v", "theta_tau", "m_tau", "v_tau", "rho_in", "tau"):
            getattr(self, k).copy_(d[k])
        self.t = int(d["t"])

    def save(self, path: str) -> None:
        """torch.save of state_dict(), through a temporary file and a rename."""
        import os

        torch.save(self.state_dict(), path + ".tmp")
        os.replace(path + ".tmp", path)

    def load(self, path: str) -> None:
        self.load_state_dict(torch.load(path, map_location="cpu"))

    def _loss_and_seed(self):
        s, p, st = self.s, self.s.plan, self.s.stream
        lbm.lbm_loss_grad(p, self.f, self.u_target, self.roi, self.loss, self.lam, s.ws, st)
        if self.probes is not None:
            nodes, rho_t, w = self.probes
            lbm.lbm_probe_loss_grad(p, self.f, nodes, rho_t, w, self.loss, self.lam, s.ws, st)

    def enqueue_iteration(self):
        """One gradient evaluation and the Adam updates, enqueued on the solver's stream."""
        s, p, st = self.s, self.s.plan, self.s.stream
        lbm.lbm_forward(p, self.rho_in, self.tau, self.rho_out, self.f, s.ws, st)
        self._loss_and_seed()
        lbm.lbm_adjoint(p, self.rho_in, self.tau, self.rho_out, self.lam, self.g_in, self.g_tau, s.ws, st)
        self.t += 1
        lbm.lbm_adam_step(self.theta, self.m, self.v, self.g_in, self.rho_in, self.rho_out, INLET_SCALE, self.t,
                          self.lr, stream=st)
        if self.invert_tau:
            lbm.lbm_adam_step(self.theta_tau, self.m_tau, self.v_tau, self.g_tau, self.tau, TAU_OFFSET, TAU_SCALE,
                              self.t, self.lr_tau, stream=st)

    def run(self, max_iters: int = 200, tol: float = 1e-3, truth_delta=None, truth_tau=None, check_every: int = 1,
            time_limit: float | None = None) -> InversionResult:
        """Iterate until the relative error on delta (and nu) is <= tol, or
        max_iters / time_limit is reached.  Without a truth, runs max_iters."""
        td = None if truth_delta is None else np.broadcast_to(np.asarray(truth_delta, np.float64), (self.s.plan.n_in,))
        nu_true = None if truth_tau is None else (truth_tau - 0.5) / 3.0
        losses, errs = [], []
        torch.cuda.synchronize(self.s.device)
        t_start = time.perf_counter()
        converged = False
        e_in = e_nu = None
        it = 0
        for it in range(1, max_iters + 1):
            self.enqueue_iteration()
            if td is None or it % check_every:
                continue
            rho = self.rho_in.cpu().numpy()  # synchronises the solver's stream
            losses.append(float(self.loss.cpu().item()))
            delta = rho - self.rho_out
            e_in = float(np.linalg.norm(delta - td) / np.linalg.norm(td))
            if nu_true is not None and self.invert_tau:
                e_nu = float(abs((self.tau.cpu().item() - 0.5) / 3.0 - nu_true) / nu_true)
            errs.append((e_in, e_nu))
            if e_in <= tol and (e_nu is None or e_nu <= tol):
                converged = True
                break
            if time_limit is not None and time.perf_counter() - t_start > time_limit:
                break
        torch.cuda.synchronize(self.s.device)
        secs = time.perf_counter() - t_start
        return InversionResult(it, secs, converged, self.rho_in.cpu().numpy(), float(self.tau.cpu().item()), e_in,
                               e_nu, losses, errs)

    # ------------------------------------------------------------- L-BFGS

    def _evaluate(self, x: np.ndarray):
        """Loss and gradient with respect to the scaled parameters x (one gradient evaluation)."""
        s, p, st = self.s, self.s.plan, self.s.stream
        n = self._n_par()
        tau = TAU_OFFSET + TAU_SCALE * x[n] if self.invert_tau else float(self.tau_fixed)
        with torch.cuda.stream(st):
            if self.spline is None:
                self.rho_in.copy_(torch.from_numpy(self.rho_out + INLET_SCALE * x[:n]), non_blocking=False)
            else:
                self.knots.copy_(torch.from_numpy(INLET_SCALE * x[:n]), non_blocking=False)
            self.tau.fill_(tau)
        if self.spline is not None:
            lbm.lbm_spline_profile(p, self.spline[0], self.spline[1], self.knots, self.rho_out, self.rho_in, st)
        lbm.lbm_forward(p, self.rho_in, self.tau, self.rho_out, self.f, s.ws, st)
        self._loss_and_seed()
        lbm.lbm_adjoint(p, self.rho_in, self.tau, self.rho_out, self.lam, self.g_in, self.g_tau, s.ws, st)
        if self.spline is not None:
            lbm.lbm_spline_grad(p, self.spline[0], self.spline[1], self.g_in, self.g_knots, st)
        st.synchronize()
        g = (self.g_in if self.spline is None else self.g_knots).cpu().numpy() * INLET_SCALE
        if self.invert_tau:
            g = np.concatenate([g, self.g_tau.cpu().numpy() * TAU_SCALE])
        return float(self.loss.cpu().item()), g

    def _n_par(self) -> int:
        return self.s.plan.n_in if self.spline is None else int(self.knots.numel())

    def _delta(self, x_in: np.ndarray) -> np.ndarray:
        """delta = rho_in - rho_out per inlet node for the inlet parameters x_in."""
        return INLET_SCALE * (x_in if self.spline is None else self.spline[2] @ x_in)

    def run_lbfgs(self, max_evals: int = 400, tol: float = 1e-3, truth_delta=None, truth_tau=None,
                  memory: int = 20, time_limit: float | None = None, callback=None,
                  resume=None) -> InversionResult:
        """L-BFGS on the scaled parameters until the relative error on delta
        (and nu) is <= tol, or max_evals gradient evaluations / time_limit.
        callback: an lbfgs callback (IterationLog, Checkpoint); resume = (x,
        history) from Checkpoint.load continues a run where it stopped."""
        p = self.s.plan
        n = self._n_par()
        self.tau_fixed = float(self.tau.cpu().item())
        x = self.theta.cpu().numpy().copy() if self.spline is None else np.zeros(n)
        if self.invert_tau:
            x = np.concatenate([x, self.theta_tau.cpu().numpy()])
        history = None
        if resume is not None:
            x, history = np.array(resume[0], np.float64), resume[1]
        td = None if truth_delta is None else np.broadcast_to(np.asarray(truth_delta, np.float64), (p.n_in,))
        nu_true = None if truth_tau is None else (truth_tau - 0.5) / 3.0

        def errors(xk):
            if td is None:
                return None
            e_in = float(np.linalg.norm(self._delta(xk[:n]) - td) / np.linalg.norm(td))
            e_nu = None
            if nu_true is not None and self.invert_tau:
                e_nu = float(abs(TAU_SCALE * xk[n] / 3.0 - nu_true) / nu_true)
            return e_in, e_nu

        def done(e):
            return e[0] <= tol and (e[1] is None or e[1] <= tol)

        torch.cuda.synchronize(self.s.device)
        r = lbfgs(inject_failures(self._evaluate), x, max_evals=max_evals, memory=memory, errors=errors, done=done,
                  lower=({n: TAU_MIN_THETA} if self.invert_tau else None), time_limit=time_limit, callback=callback,
                  history=history)
        x = r.x
        self.theta.copy_(torch.from_numpy(self._delta(x[:n]) / INLET_SCALE))
        if self.invert_tau:
            self.theta_tau.fill_(float(x[n]))
        self.evaluations = r.evaluations
        e_in, e_nu = r.errs[-1] if r.errs else (None, None)
        return InversionResult(r.iterations, r.seconds, r.converged, self.rho_out + self._delta(x[:n]),
                               TAU_OFFSET + TAU_SCALE * x[n] if self.invert_tau else self.tau_fixed, e_in, e_nu,
                               r.losses, r.errs)
