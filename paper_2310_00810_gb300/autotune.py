"""Autotuner for the state layout and kernel choice of a plan.

For a given lattice (size, Q, precision, geometry) it times, on the device,
the candidate kernel families of the stream-collide and adjoint steps in the
dense layout — TMA staging with 8- or 4-row tiles, register kernels with 4 or
2 nodes per thread, one node per thread — then programmatic dependent launch
on/off and the one-launch persistent sweeps, the overlapped reverse sweep (recompute on a second stream) on/off,
the segment recompute on a register family beside the adjoint, two stream-collide steps per launch
(D2Q9 FP32), then the fluid-only (compact) layout with two-buffer or in-place streaming, and keeps the
fastest.  Only the speed differs between candidates;
every family and layout computes the same step.  Results are cached in JSON
keyed by GPU name, Q, precision, lattice size and inlet kind.

Timing uses a short tuning plan bound to the solver's geometry (T_tune time
steps), with CUDA events around graph-replayed launch sequences.

``tune_batch`` does the same for a batch of lattices (lbm.Batch): it times a
whole gradient evaluation (forward, loss, checkpointed adjoint) of a short
copy of the batch (same sizes and geometries, T_tune steps) in the dense
layout (register kernels over row segments) and in the packed fluid-only
layout, and keeps the faster.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import lbm

_lock = threading.Lock()
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(p: lbm.Plan) -> str:
    name = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    return f"{name}|q{p.q}|p{p.precision}|{p.nx}x{p.ny}x{p.nz}|{p.inlet_kind}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, key, value):
    with _lock:
        db = _load(path)
        db[key] = value
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(db, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def step_candidates(p: lbm.Plan):
    """(name, step_family, vec, tma_rows) the plan's shape allows."""
    out = []
    if p.precision == 4 and p.nx % 4 == 0:
        out.append(("tma8", lbm.LBM_FAMILY_TMA, 4, 8))
        if p.q == 9:
            out.append(("tma4", lbm.LBM_FAMILY_TMA, 4, 4))
    if p.nx % 4 == 0 and p.precision == 4:
        out.append(("vec4", lbm.LBM_FAMILY_VEC, 4, 8))
    if p.nx % 2 == 0:
        out.append(("vec2", lbm.LBM_FAMILY_VEC, 2, 8))
    out.append(("scalar", lbm.LBM_FAMILY_SCALAR, 2, 8))
    return out


def _time(fn, repeats, stream):
    fn()  # warm: graph capture, first-touch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(repeats):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return best


def tune(solver: lbm.Solver, t_tune: int = 64, repeats: int = 3, cache: str | None = DEFAULT_CACHE,
         use_cache: bool = True, apply: bool = True) -> dict:
    """Choose and (by default) apply the fastest kernel configuration for the
    solver's plan.  Returns {"choice": {...}, "timings_us": {...}}."""
    p = solver.plan
    if getattr(solver, "periodic_y", False):
        # periodic link words wrap in y, which only the fluid-only kernels follow: no dense candidates
        return {"choice": lbm.lbm_plan_get_kernels(p), "layout": solver.layout, "timings_us": {},
                "us_per_time_step": None, "skipped": "periodic y runs in the fluid-only layout only"}
    key = _key(p)
    if use_cache and cache:
        hit = _load(cache).get(key)
        if hit:
            if apply:
                _apply(solver, hit)
            return dict(hit, cached=True)
    dev = solver.device
    tp = lbm.Solver(p.q, p.nx, p.ny, p.nz, precision=p.precision, n_steps=t_tune, ckpt_stride=8,
                    inlet_kind=p.inlet_kind, link=solver.link, mask=solver.mask, device=dev, layout="dense")
    tq = tp.plan
    rho_in = torch.full((tq.n_in,), 1.001, dtype=torch.float64, device=dev)
    tau = torch.tensor([0.8], dtype=torch.float64, device=dev)
    a = tp.new_state().zero_()
    b = tp.new_state().zero_()
    st = tp.stream
    timings = {}

    def time_step(choice):
        lbm.lbm_plan_set_kernels(tq, **choice)
        return _time(lambda: lbm.lbm_step(tq, rho_in, tau, 1.0, a, b, t_tune, tp.ws, st), repeats, st) / (t_tune + 1)

    best_step, best_t = None, float("inf")
    for name, fam, vec, rows in step_candidates(tq):
        choice = dict(step_family=fam, adjoint_family=lbm.LBM_FAMILY_AUTO, vec=vec, tma_rows=rows, pdl=1, persist=0)
        t = time_step(choice)
        timings[f"step:{name}"] = round(t * 1e6, 3)
        if t < best_t:
            best_step, best_t = (name, fam, vec, rows), t

    u_t = torch.zeros((tq.d, *tq.shape), dtype=torch.float64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    lam = tp.new_state()
    g_in = torch.zeros(tq.n_in, dtype=torch.float64, device=dev)
    g_tau = torch.zeros(1, dtype=torch.float64, device=dev)

    def time_sweeps(choice):
        lbm.lbm_plan_set_kernels(tq, **choice)

        def run():
            lbm.lbm_forward(tq, rho_in, tau, 1.0, a, tp.ws, st)
            lbm.lbm_loss_grad(tq, a, u_t, None, loss, lam, tp.ws, st)
            lbm.lbm_adjoint(tq, rho_in, tau, 1.0, lam, g_in, g_tau, tp.ws, st)

        return _time(run, repeats, st) / t_tune

    _, sfam, svec, srows = best_step
    best, best_t = None, float("inf")
    for name, fam, vec, rows in step_candidates(tq):
        choice = dict(step_family=sfam, adjoint_family=fam, vec=vec if fam != sfam else svec, tma_rows=srows,
                      pdl=1, persist=0, adjoint_tma_rows=rows if fam == lbm.LBM_FAMILY_TMA else 0)
        t = time_sweeps(choice)
        timings[f"sweep:step={best_step[0]},adjoint={name}"] = round(t * 1e6, 3)
        if t < best_t:
            best, best_t = choice, t
    for pdl in (0,):
        c = dict(best, pdl=pdl)
        t = time_sweeps(c)
        timings[f"sweep:best,pdl={pdl}"] = round(t * 1e6, 3)
        if t < best_t:
            best, best_t = c, t
    if tq.N * tq.q * tq.precision <= 24 * 2 ** 20 and p.nx % 4 == 0:
        c = dict(best, persist=1)
        t = time_sweeps(c)
        timings["sweep:best,persist=1"] = round(t * 1e6, 3)
        if t < best_t:
            best, best_t = c, t
    for ov in (0,):
        c = dict(best, overlap=ov)
        t = time_sweeps(c)
        timings[f"sweep:best,overlap={ov}"] = round(t * 1e6, 3)
        if t < best_t:
            best, best_t = c, t
    if not best.get("persist") and best.get("overlap", 1):
        # the segment recompute on a register family: its CTAs need no shared memory, so they can share the SMs
        # with the adjoint's TMA CTAs on the second stream
        for name, fam in (("vec", lbm.LBM_FAMILY_VEC), ("scalar", lbm.LBM_FAMILY_SCALAR)):
            c = dict(best, recompute_family=fam)
            t = time_sweeps(c)
            timings[f"sweep:best,recompute={name}"] = round(t * 1e6, 3)
            if t < best_t:
                best, best_t = c, t
    if tq.q == 9 and tq.precision == 4 and p.nx % 4 == 0 and not best.get("persist"):
        # two stream-collide steps per launch (temporal blocking), with either tile height
        for rows in (8, 4):
            c = dict(best, steps_per_launch=2, tma_rows=rows)
            t = time_sweeps(c)
            timings[f"sweep:best,steps_per_launch=2,rows={rows}"] = round(t * 1e6, 3)
            if t < best_t:
                best, best_t = c, t
    layout = "dense"
    tp.set_layout("compact")
    if tp.layout == "compact":
        for pdl in (1, 0):
            c = dict(best, pdl=pdl, persist=0, overlap=1, steps_per_launch=1, aa=0)
            t = time_sweeps(c)
            timings[f"sweep:compact,pdl={pdl}"] = round(t * 1e6, 3)
            if t < best_t:
                best, best_t, layout = c, t, "compact"
        if not solver_uw_extrap(solver):
            # in-place streaming (one state buffer; every other step reads no table)
            base = best if layout == "compact" else dict(best, persist=0, overlap=1, steps_per_launch=1)
            c = dict(base, aa=1)
            t = time_sweeps(c)
            timings["sweep:compact,in_place"] = round(t * 1e6, 3)
            if t < best_t:
                best, best_t, layout = c, t, "compact"
    result = {"choice": best, "layout": layout, "timings_us": timings, "us_per_time_step": round(best_t * 1e6, 3),
              "key": key}
    if cache:
        _store(cache, key, result)
    if apply:
        _apply(solver, result)
    tp.plan.close()
    return dict(result, cached=False)


def solver_uw_extrap(solver: lbm.Solver) -> bool:
    """Whether the plan's Eq. 6 takes the extrapolated wall velocity (the in-place schedule does not)."""
    return lbm.lbm_get_abb_velocity(solver.plan) == lbm.LBM_ABB_U_EXTRAP


def _apply(solver: lbm.Solver, result: dict) -> None:
    solver.set_layout(result.get("layout", "dense"))
    choice = dict(result["choice"])
    if solver_uw_extrap(solver):
        choice["aa"] = 0
    solver.set_kernels(**choice)


def _batch_key(b) -> str:
    import hashlib

    name = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    geo = hashlib.sha1(repr((b.sizes, b.geometries)).encode()).hexdigest()[:16]
    return f"{name}|batch|q{b.q}|p{b.precision}|n{b.n}|{geo}|{b.inlet_kind}"


def tune_batch(batch, t_tune: int = 64, repeats: int = 2, cache: str | None = DEFAULT_CACHE, use_cache: bool = True,
               apply: bool = True) -> dict:
    """Choose and (by default) apply the faster layout of a batch.  Returns
    {"layout": ..., "timings_us": {...}, "us_per_time_step": ...}."""
    key = _batch_key(batch)
    if use_cache and cache:
        hit = _load(cache).get(key)
        if hit:
            if apply:
                batch.set_layout(hit["layout"])
            return dict(hit, cached=True)
    dev = batch.device
    tb = lbm.Batch(batch.q, batch.sizes, precision=batch.precision, n_steps=t_tune, ckpt_stride=8,
                   inlet_kind=batch.inlet_kind, geometries=batch.geometries, device=dev)
    rho_in = tb.new_inlet().fill_(1.001)
    tau = torch.full((tb.n,), 0.8, dtype=torch.float64, device=dev)
    ut = tb.new_velocity()
    f, lam = tb.new_state(), tb.new_state()
    loss = torch.zeros(tb.n, dtype=torch.float64, device=dev)
    g_in, g_tau = tb.new_inlet(), torch.zeros(tb.n, dtype=torch.float64, device=dev)

    def run():
        tb.forward(rho_in, tau, 1.0, f)
        tb.loss_grad(f, ut, None, loss, lam)
        tb.adjoint(rho_in, tau, 1.0, lam, g_in, g_tau)

    timings = {}
    best, best_t = None, float("inf")
    for layout in ("dense", "compact"):
        tb.set_layout(layout)
        t = _time(run, repeats, tb.stream) / t_tune
        timings[f"batch:{layout}"] = round(t * 1e6, 3)
        if t < best_t:
            best, best_t = layout, t
    result = {"layout": best, "timings_us": timings, "us_per_time_step": round(best_t * 1e6, 3), "key": key}
    if cache:
        _store(cache, key, result)
    if apply:
        batch.set_layout(best)
    tb.close()
    return dict(result, cached=False)
