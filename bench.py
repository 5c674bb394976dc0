"""Benchmark of the AD-LBM hot path: forward + adjoint gradient evaluations.

One step = one gradient evaluation of the 512x256 D2Q9 FP32 disk packing
(porosity 0.6, 20000 time steps, 256-entry inlet density profile): the
forward sweep with sqrt(T) checkpoints, the loss and its seed, the
checkpointed reverse sweep (segment recompute + adjoint steps) and one Adam
update of the profile, all on the device.  The metric is fwd+adjoint MLUPS:
lattice nodes x time steps per second (each time step's forward and adjoint
update counted once), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the CPU oracle (plain FP64 C) is timed on the same
workload and metric, each step a bounded sample of time steps.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "disks512x256"
METRIC = "fwd+adjoint MLUPS (D2Q9 FP32 512x256 disks, 20000 steps, checkpointed adjoint)"
UNIT = "MLUPS"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-roofline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=250)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="override T (profiling runs only; the reported workload is T = 20000)")
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels", "unet"],
                    help="kernels: time the stream-collide and adjoint kernels alone on --lattice; "
                         "unet: training throughput of the learned initialiser")
    ap.add_argument("--unet-batch", type=int, default=16)
    ap.add_argument("--unet-engine", default="tcgen05", choices=["tcgen05", "mma_sync"],
                    help="--mode unet: the convolutions' GEMM engine")
    ap.add_argument("--lattice", default="disks8192x4096", help="workload name for --mode kernels")
    ap.add_argument("--layout", default=None, choices=[None, "dense", "compact"],
                    help="state layout for --mode kernels (default: compact for D3Q19, dense for D2Q9)")
    ap.add_argument("--launches", type=int, default=20)
    ap.add_argument("--aa", type=int, default=0, choices=[0, 1],
                    help="--mode kernels: the in-place (AA-pattern) schedule of the fluid-only layout")
    ap.add_argument("--no-invert", action="store_true", help="skip the time-to-1e-3 inversion leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched leg")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--no-batch-invert", action="store_true", help="skip the batched time-to-1e-3 leg")
    ap.add_argument("--batch-invert-instances", type=int, default=12,
                    help="instances of the batched time-to-1e-3 leg (the first of the 64-instance recipe)")
    ap.add_argument("--batch-invert-max-nx", type=int, default=384,
                    help="largest nx of the batched time-to-1e-3 leg's instances (1024: every size)")
    ap.add_argument("--no-c3", action="store_true", help="skip the 3D joint (head, tau) inversion leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initialiser leg")
    ap.add_argument("--no-wake", action="store_true", help="skip the cylinder-wake viscosity inversion leg")
    ap.add_argument("--learned-solves", type=int, default=2048, help="training solves of the learned initialiser")
    ap.add_argument("--learned-epochs", type=int, default=25)
    ap.add_argument("--learned-eval", type=int, default=3, help="held-out inversions (from the guess and from zero)")
    ap.add_argument("--invert-time-limit", type=float, default=180.0)
    return ap.parse_args()


def replica_seeds(rank: int) -> dict:
    """Seeds of rank `rank`'s independent replica (replicas differ in their
    inlet profiles and batched geometries; the lattice of the timed workload
    is the same on every rank)."""
    return {"profile": 2000 + rank, "batch": 4000 + 100 * rank}


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = [r for r in csv.reader(open(self.path)) if len(r) >= 9]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- the workload

def make_problem(device, rank, time_steps=None):
    import dataclasses

    import torch

    from paper_2310_00810_gb300 import lbm
    from paper_2310_00810_gb300 import workloads as W

    wl = W.WORKLOADS[WORKLOAD]
    if time_steps:
        wl = dataclasses.replace(wl, steps=time_steps)
    s = lbm.Solver(wl.q, wl.nx, wl.ny, precision=wl.precision, n_steps=wl.steps, inlet_kind=lbm.LBM_INLET_PROFILE,
                   geometry=dict(kind=lbm.LBM_GEOM_DISKS, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                                 target_porosity=wl.porosity), device=device)
    delta_true = W.inlet_profile(wl.ny, seed=replica_seeds(rank)["profile"])
    dv = lambda a: torch.as_tensor(np.asarray(a, np.float64), device=device)
    tau = dv([wl.tau])
    f = s.forward(dv(wl.rho_out + delta_true), tau, wl.rho_out)
    _, u_target = s.macroscopic(f)
    prob = dict(solver=s, wl=wl, tau=tau, u_target=u_target.contiguous(), delta_true=delta_true,
                theta=torch.zeros(wl.ny, dtype=torch.float64, device=device),
                m=torch.zeros(wl.ny, dtype=torch.float64, device=device),
                v=torch.zeros(wl.ny, dtype=torch.float64, device=device),
                rho_in=torch.full((wl.ny,), wl.rho_out, dtype=torch.float64, device=device),
                f=s.new_state(), lam=s.new_state(),
                loss=torch.zeros(1, dtype=torch.float64, device=device),
                g_in=torch.zeros(wl.ny, dtype=torch.float64, device=device),
                g_tau=torch.zeros(1, dtype=torch.float64, device=device), t=0)
    return prob


def issue_step(P, ev=None):
    """Enqueue one gradient evaluation + Adam update on the solver's stream."""
    from paper_2310_00810_gb300 import lbm

    s, wl = P["solver"], P["wl"]
    p = s.plan
    if ev is not None:
        ev[0].record(s.stream)
    lbm.lbm_forward(p, P["rho_in"], P["tau"], wl.rho_out, P["f"], s.ws, s.stream)
    if ev is not None:
        ev[1].record(s.stream)
    lbm.lbm_loss_grad(p, P["f"], P["u_target"], None, P["loss"], P["lam"], s.ws, s.stream)
    lbm.lbm_adjoint(p, P["rho_in"], P["tau"], wl.rho_out, P["lam"], P["g_in"], P["g_tau"], s.ws, s.stream)
    P["t"] += 1
    lbm.lbm_adam_step(P["theta"], P["m"], P["v"], P["g_in"], P["rho_in"], wl.rho_out, 1e-3, P["t"], 0.02,
                      stream=s.stream)
    if ev is not None:
        ev[2].record(s.stream)


def launches_per_step(wl, k):
    """Kernels of this library launched by one gradient evaluation."""
    T = wl.steps
    S = (T + k - 1) // k
    fwd = T  # T-1 stream-collide + 1 stream-only
    loss = 4  # count, weight, loss, final
    recompute = 0
    for sg in range(S):
        ln = min(k, T - sg * k)
        recompute += max(0, ln - 1) - (1 if sg == 0 and ln >= 2 else 0)
    adj = T + 1  # T adjoint steps + gradient finalise
    return fwd + loss + recompute + adj + 1  # + Adam


def fluid_nodes(P):
    return int(P["solver"].info[3].item())


def run_native(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2310_00810_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    P = make_problem(device, rank, args.time_steps)
    s, wl = P["solver"], P["wl"]
    from paper_2310_00810_gb300 import autotune

    tuned = autotune.tune(s)  # kernel family / tile shape for this lattice (cached per GPU and shape)
    N = wl.nodes
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    for _ in range(max(3, args.warmup)):
        issue_step(P)
    barrier()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(s.stream):
            flush.fill_(float(i))  # evict the previous step's lines from the 129 MB L2
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed launches
        issue_step(P, evs[i])
        torch.cuda.nvtx.range_pop()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    step_ms = [evs[i][0].elapsed_time(evs[i][2]) for i in range(args.steps)]
    fwd_ms = [evs[i][0].elapsed_time(evs[i][1]) for i in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), device)
    ms_per_step = total_ms / args.steps
    value = job_throughput(N * wl.steps * args.steps, world, total_ms * 1e-3) / 1e6

    # roofline of the dominant kernel: the fused stream-collide step, timed live
    # through the forward phase of every timed step (T launches per phase)
    nf = fluid_nodes(P)
    bytes_per_launch = 2 * wl.q * 4 * nf + 4 * N  # populations of fluid nodes + link words
    fwd_launch_s = statistics.mean(fwd_ms) * 1e-3 / wl.steps
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = bytes_per_launch / fwd_launch_s / 1e9
    roofline = {"bound": "hbm", "kernel": f"stream-collide step ({tuned['choice']})",
                "achieved": round(achieved, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "peak_source": "measured" if peaks else "fallback",
                "traffic": None, "bytes_per_launch": bytes_per_launch,
                "note": "512x256 state (9.4 MB read+write per step) is L2-resident; see roofline_hbm"}

    e2e = None if args.no_e2e else run_e2e(P, args, device, barrier, world)
    hbm = None
    if not args.no_hbm_roofline:
        hbm = {f"{name}/{layout}": kernel_rooflines(device, hbm_peak, name, 20, layout)
               for name, layout in (("disks8192x4096", "dense"), ("disks8192x4096", "compact"),
                                    ("spheres512x256x256", "compact"))}

    inversion = None if args.no_invert else time_to_target(P, args.invert_time_limit)
    batched = None if args.no_batch else batch_leg(device, args.batch_instances, rank)
    batched_inv = None if args.no_batch_invert else batch_invert_leg(device, args.batch_invert_instances, rank,
                                                                      args.invert_time_limit,
                                                                      max_nx=args.batch_invert_max_nx)
    c3 = None if args.no_c3 else c3_leg(device, args.invert_time_limit)
    learned = None if args.no_learned else learned_init_leg(device, args.learned_solves, args.learned_epochs,
                                                            args.learned_eval, args.invert_time_limit / 2)
    wake = None if args.no_wake else cylinder_wake_leg(device, args.invert_time_limit / 2)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps)
        cpu["single_thread"] = cpu_baseline(max(20, args.cpu_sample_steps // 4), threads=1)["value"]
        cpu["cpu_model"] = cpu_model()
        cpu["other_workloads"] = cpu_other_workloads(cpu["cores"])

    rel_err = float(np.linalg.norm((P["rho_in"].cpu().numpy() - wl.rho_out) - P["delta_true"]) /
                    np.linalg.norm(P["delta_true"]))
    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: D2Q9 BGK FP32 512x256, seeded disks r 6-12 porosity "
                                   f"{nf / N:.4f} (target 0.6), T={wl.steps}, tau 0.8, 256-entry inlet profile "
                                   f"(4 sine modes, amplitude 1e-3), sqrt(T) checkpoints, Adam lr 0.02",
                       "nodes": N, "fluid_nodes": nf, "time_steps": wl.steps,
                       "l2": "512 MB buffer written between timed steps (L2 flush); per-step state is L2-resident",
                       "parallelism": f"replicas x{world} (independent inversions, no collective)",
                       "kernels": tuned["choice"], "layout": tuned.get("layout", "dense"),
                       "autotune_us_per_time_step": tuned.get("us_per_time_step"),
                       "autotune_timings_us": tuned.get("timings_us")},
            "e2e": e2e, "gpu_launches": launches_per_step(wl, s.plan_k if hasattr(s, "plan_k") else
                                                          max(1, math.ceil(math.sqrt(wl.steps)))) * args.steps,
            "roofline": roofline, "roofline_hbm": hbm, "cpu_baseline": cpu, "clocks": clocks,
            "wall_s_timed_region": round(wall, 3),
            "inversion_progress": {"adam_steps": P["t"], "rel_err_delta": rel_err},
            "time_to_1e-3": inversion,
            "batched": batched,
            "batched_time_to_1e-3": batched_inv,
            "joint_inversion_3d": c3,
            "learned_initialiser": learned,
            "viscosity_inversion_wake": wake,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def time_to_target(P, time_limit):
    """Wall time for the single-instance inversion of the 256-entry inlet
    profile from delta = 0 to 1e-3 relative error (L-BFGS on the device
    gradients; each evaluation is one forward + checkpointed adjoint sweep)."""
    from paper_2310_00810_gb300 import invert as I

    s, wl = P["solver"], P["wl"]
    inv = I.Inversion(s, P["u_target"], wl.rho_out, tau0=wl.tau)
    res = inv.run_lbfgs(max_evals=2000, tol=1e-3, truth_delta=P["delta_true"], time_limit=time_limit)
    return {"seconds": round(res.seconds, 2), "converged": bool(res.converged), "iterations": res.iterations,
            "gradient_evaluations": inv.evaluations, "rel_err_delta": res.rel_err_inlet, "method": "L-BFGS",
            "start": "delta = 0 (no initial guess)", "time_limit_s": time_limit}


def carman_kozeny(porosity, d_p, shape_factor=180.0, sphericity=1.0):
    """Eq. 8: k_CK = Phi_s^2 eps^3 D_p^2 / (Phi_CK (1 - eps)^2)."""
    return sphericity ** 2 * porosity ** 3 * d_p ** 2 / (shape_factor * (1.0 - porosity) ** 2)


def c3_leg(device, time_limit):
    """The 3D joint inversion: D3Q19 FP32 128x64x64 Boolean-sphere packing
    (r = 6, porosity 0.45), T = 10000, constant head and tau recovered together
    from the steady velocity field (truth delta = 1e-3, tau = 0.8; start delta =
    0, tau = 1.0), by L-BFGS on the device gradients.  In the Stokes regime
    u ~ delta / nu, so the identifiable quantity is the ratio delta / nu (and
    the Darcy permeability); the individual errors are reported as well.
    Darcy k (Eq. 12) at the recovered parameters against Carman-Kozeny (Eq. 8,
    D_p = 12, Phi_CK = 180)."""
    import torch

    from paper_2310_00810_gb300 import autotune, lbm
    from paper_2310_00810_gb300 import invert as I
    from paper_2310_00810_gb300 import workloads as W

    wl = W.WORKLOADS["spheres128x64x64"]
    s = lbm.Solver(wl.q, wl.nx, wl.ny, wl.nz, precision=wl.precision, n_steps=wl.steps,
                   inlet_kind=lbm.LBM_INLET_CONST,
                   geometry=dict(kind=wl.geom_kind, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                                 target_porosity=wl.porosity), device=device)
    tuned = autotune.tune(s)
    nf = int(s.info[3].item())
    porosity = nf / wl.nodes
    dv = lambda a: torch.as_tensor(np.asarray(a, np.float64), device=device)
    delta_true, tau_true = 1e-3, wl.tau
    f = s.forward(dv([wl.rho_out + delta_true]), dv([tau_true]), wl.rho_out)
    _, u_target = s.macroscopic(f)
    k_true, _ = s.darcy(f, dv([wl.rho_out + delta_true]), dv([tau_true]), wl.rho_out)
    inv = I.Inversion(s, u_target.contiguous(), wl.rho_out, tau0=1.0, invert_tau=True)
    res = inv.run_lbfgs(max_evals=400, tol=1e-3, truth_delta=delta_true, truth_tau=tau_true, time_limit=time_limit)
    d_hat = float(res.rho_in[0]) - wl.rho_out
    nu_hat, nu_true = (res.tau - 0.5) / 3.0, (tau_true - 0.5) / 3.0
    ratio_err = abs(d_hat / nu_hat - delta_true / nu_true) / (delta_true / nu_true)
    f_hat = s.forward(dv([wl.rho_out + d_hat]), dv([res.tau]), wl.rho_out)
    k_hat, _ = s.darcy(f_hat, dv([wl.rho_out + d_hat]), dv([res.tau]), wl.rho_out)
    k_ck = carman_kozeny(porosity, 2.0 * wl.r_max)
    # the same inversion with density probes added to the loss: 16 fluid nodes on each of the
    # sections x = 16, 48, 80, 112 observe rho; weight w = 0.1 sum |u_t|^2 / sum (rho_p - rho_out)^2,
    # a tenth of the velocity term at the start (at rest), which a CPU oracle scan of weights on a
    # small duct found fastest (larger weights stretch the valley along tau)
    rho_field, _ = s.macroscopic(f)
    m = s.mask_field.cpu().numpy()
    nodes = []
    for xs in (16, 48, 80, 112):
        fl = np.flatnonzero(m[:, :, xs].reshape(-1) == 0)
        pick = fl[np.linspace(0, fl.size - 1, 16).astype(np.int64)]
        zz, yy = np.unravel_index(pick, m.shape[:2])
        nodes += list((zz * wl.ny + yy) * wl.nx + xs)
    nodes_t = torch.as_tensor(np.array(nodes, np.int64), device=device)
    rho_t = rho_field.reshape(-1)[nodes_t].contiguous()
    w_p = 0.1 * float((u_target ** 2).sum().item()) / float(((rho_t - wl.rho_out) ** 2).sum().item())
    inv_p = I.Inversion(s, u_target.contiguous(), wl.rho_out, tau0=1.0, invert_tau=True, probes=(nodes_t, rho_t, w_p))
    res_p = inv_p.run_lbfgs(max_evals=200, tol=1e-3, truth_delta=delta_true, truth_tau=tau_true,
                            time_limit=min(time_limit, 60.0))
    with_probes = {"probes": f"64 fluid nodes on x = 16, 48, 80, 112, weight {w_p:.4g}", "seconds": round(res_p.seconds, 2),
                   "converged": bool(res_p.converged), "gradient_evaluations": inv_p.evaluations,
                   "rel_err_delta": res_p.rel_err_inlet, "rel_err_nu": res_p.rel_err_nu,
                   "err_history_tail": [list(e) for e in res_p.err_history[-4:]]}
    out = {"workload": "spheres128x64x64: D3Q19 BGK FP32 128x64x64 duct, Boolean spheres r 6, "
                       f"porosity {porosity:.4f} (target 0.45), T={wl.steps}, constant head + tau",
           "kernels": tuned["choice"], "layout": tuned.get("layout", "dense"),
           "us_per_time_step": tuned.get("us_per_time_step"), "autotune_timings_us": tuned.get("timings_us"),
           "seconds": round(res.seconds, 2), "converged": bool(res.converged), "gradient_evaluations": inv.evaluations,
           "seconds_per_gradient_eval": round(res.seconds / max(1, inv.evaluations), 3),
           "rel_err_delta": res.rel_err_inlet, "rel_err_nu": res.rel_err_nu, "rel_err_delta_over_nu": ratio_err,
           "method": "L-BFGS on (delta / 1e-3, (tau - 0.5) / 0.1)", "start": "delta = 0, tau = 1.0",
           "darcy_k_truth": float(k_true.item()), "darcy_k_recovered": float(k_hat.item()),
           "darcy_k_rel_err": abs(float(k_hat.item()) - float(k_true.item())) / float(k_true.item()),
           "carman_kozeny_k": k_ck, "k_over_k_ck": float(k_true.item()) / k_ck, "time_limit_s": time_limit,
           "with_density_probes": with_probes}
    del s, inv, inv_p
    torch.cuda.empty_cache()
    return out


def cylinder_wake_leg(device, time_limit):
    """Section 3.4's viscosity inversion at Re 100 on the paper's 400 x 160
    channel: a cylinder of diameter 10 centred at (80, 81.3) (off the channel's
    mid-line by 1.8 nodes, which starts the shedding), periodic top and bottom,
    velocity inlet u_inf = 0.2 started with a sin^2 ramp over 1500 steps, Eq. 6
    outlet at rho = 1, D2Q9 MRT (free rates s_e 1.1, s_eps 1.1, s_q 1.2), FP32,
    fluid-only layout.  Truth nu = 0.02 (tau = 0.56), start nu = 0.06 (the
    paper's).  The loss sums |u - u_target|^2 over the 100 x 80 rectangle
    100 <= x < 200, 40 <= y < 120 at a window of observation steps, its
    gradient taken in one reverse sweep (lbm_adjoint_window).  Two stages:
    L-BFGS on the wake's onset window (steps 1600..2400, where the loss is
    smooth in nu), then on one shedding period of the periodic wake (steps
    7000..7300, whose loss oscillates in nu with the shedding phase) from the
    first stage's estimate.  The late window alone from nu = 0.06 is run too."""
    import torch

    from paper_2310_00810_gb300 import invert as I
    from paper_2310_00810_gb300 import lbm

    nx, ny, d, ramp, nu_true, nu0 = 400, 160, 10, 1500, 0.02, 0.06
    windows = {"onset": list(range(1600, 2401, 100)), "periodic": list(range(7000, 7301, 50))}
    yy, xx = np.mgrid[0:ny, 0:nx]
    m = torch.as_tensor((((xx - 80) ** 2 + (yy - 81.3) ** 2) <= (d / 2) ** 2).astype(np.uint8))
    roi = torch.zeros((ny, nx), dtype=torch.uint8, device=device)
    roi[40:120, 100:200] = 1
    rin = torch.ones(1, dtype=torch.float64, device=device)

    def solver(T):
        s = lbm.Solver(9, nx, ny, precision=4, n_steps=T, geometry=m, periodic_y=True, device=device)
        s.set_velocity_inlet((0.2, 0.0))
        s.set_velocity_ramp(ramp)
        s.set_collision(lbm.LBM_COLLISION_MRT, 1.1, 1.1, 1.2)
        return s

    tau_true = torch.tensor([0.5 + 3 * nu_true], dtype=torch.float64, device=device)
    stages = {}
    for name, obs in windows.items():
        u = []
        for t in obs:  # the observed fields: the forward model at the truth, read at each observation step
            st = solver(t)
            u.append(st.macroscopic(st.forward(rin, tau_true, 1.0))[1])
            st.plan.close()
        stages[name] = (solver(obs[-1]), obs, torch.stack(u).contiguous())

    def invert(name, start):
        s, obs, ut = stages[name]
        tau = torch.empty(1, dtype=torch.float64, device=device)

        def evaluate(x):  # x = nu / 0.01
            tau.fill_(0.5 + 0.03 * float(x[0]))
            f = s.forward(rin, tau, 1.0)
            L, _, g_tau = s.adjoint_window(rin, tau, 1.0, f, obs, ut, roi)
            return L.item(), np.array([g_tau.item() * 0.03])

        res = I.lbfgs(evaluate, np.array([start / 0.01]), max_evals=40, lower={0: 1.2}, time_limit=time_limit,
                      errors=lambda x: (abs(0.01 * x[0] - nu_true) / nu_true, None), done=lambda e: e[0] < 1e-3)
        nu = 0.01 * float(res.x[0])
        return nu, {"window_steps": [obs[0], obs[-1], obs[1] - obs[0]], "start_nu": start, "recovered_nu": nu,
                    "rel_err_nu": abs(nu - nu_true) / nu_true, "converged": bool(res.converged),
                    "gradient_evaluations": res.evaluations, "seconds": round(res.seconds, 2)}

    torch.cuda.synchronize(device)
    nu1, onset = invert("onset", nu0)
    nu2, periodic = invert("periodic", nu1)
    _, late_only = invert("periodic", nu0)
    out = {"workload": "cylinder400x160 Re 100: D2Q9 MRT FP32, D = 10, periodic y, u_inf = 0.2 (sin^2 ramp over "
                       "1500 steps), fluid-only layout", "truth_nu": nu_true, "start_nu": nu0, "recovered_nu": nu2,
           "rel_err_nu": abs(nu2 - nu_true) / nu_true, "converged": bool(periodic["converged"]),
           "gradient_evaluations": onset["gradient_evaluations"] + periodic["gradient_evaluations"],
           "seconds": round(onset["seconds"] + periodic["seconds"], 2),
           "method": "L-BFGS on nu / 0.01; windowed loss over the 100x80 downstream rectangle; onset window, "
                     "then the periodic window from its estimate",
           "stage_onset": onset, "stage_periodic": periodic, "periodic_window_only_from_start": late_only,
           "time_limit_s": time_limit}
    for s, _, _ in stages.values():
        s.plan.close()
    del stages
    torch.cuda.empty_cache()
    return out


def unet_flops_per_sample(base, H, W):
    """Multiply-add FLOPs (2 per MAC) of one forward pass of the U-Net."""
    c = [base << l for l in range(4)]
    f, prev = 0, 8
    for l in range(4):
        px = (H >> l) * (W >> l)
        f += 2 * px * 9 * (prev * c[l] + c[l] * c[l])
        prev = c[l]
    for l in (2, 1, 0):
        px = (H >> l) * (W >> l)
        f += 2 * px * c[l + 1] * c[l]  # transposed convolution: one tap per output pixel
        f += 2 * px * 9 * (2 * c[l] * c[l] + c[l] * c[l])
    return f + 2 * H * W * c[0]


def learned_init_leg(device, n_train, epochs, n_eval, time_limit):
    """The learned initialiser at 256x128: generate training solves with the
    library (batched forward, T = 10000, disks r 6-12, porosity U[0.5, 0.7],
    4-mode sine profiles), train the U-Net (base 32, BF16 kernels), then invert
    held-out packings by L-BFGS from the network's guess and from delta = 0."""
    import torch

    from paper_2310_00810_gb300 import unet as N

    nx, ny, T, base, batch = 256, 128, 10000, 32, 16
    t0 = time.perf_counter()
    data = N.generate(n_train, 5000, nx=nx, ny=ny, steps=T, chunk=64, device=device)
    torch.cuda.synchronize(device)
    t_gen = time.perf_counter() - t0
    net = N.UNet(base=base, height=ny, width=nx, batch=batch, seed=5)
    N.train(net, data, epochs=1, lr=1e-3)  # warm-up epoch (first launches, allocations)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    hist = N.train(net, data, epochs=epochs, lr=2e-3, seed=1, lr_final=1e-4)
    torch.cuda.synchronize(device)
    t_train = time.perf_counter() - t0
    samples = epochs * (n_train // batch) * batch
    flops = 3 * unet_flops_per_sample(base, ny, nx) * samples  # forward + two backward products
    seeds = [5000 + 20000 + i for i in range(n_eval)]
    rows = N.evaluate(net, seeds, nx=nx, ny=ny, steps=T, max_evals=600, time_limit=time_limit)
    # the same held-out inversions, all in one packed batch started from the network's guesses: the
    # learned initialiser with batching against the plain single-instance inversion from delta = 0
    batched = N.evaluate_batched(net, seeds, nx=nx, ny=ny, steps=T, max_evals=600, time_limit=time_limit)
    zero_single = float(np.mean([r["zero"]["seconds"] for r in rows]))
    mean = lambda key, f: float(np.mean([f(r[key]) for r in rows]))
    return {"workload": f"U-Net base {base}, input 2 velocity channels + mask at {nx}x{ny}, BF16 weights/activations, "
                        f"FP32 accumulation (mma.sync tensor cores); {n_train} training solves (D2Q9 FP32, T={T}, "
                        f"disks r 6-12, porosity U[0.5, 0.7], seeds 5000+j), {epochs} epochs, held-out seeds 25000+i",
            "generation_s": round(t_gen, 2), "solves_per_s": round(n_train / t_gen, 2),
            "train_s": round(t_train, 2), "train_samples_per_s": round(samples / t_train, 1),
            "train_tflops": round(flops / t_train / 1e12, 2), "final_train_loss": hist[-1],
            "prediction_rel_err": float(np.mean([r["prediction_rel_err"] for r in rows])),
            "lbfgs_from_unet": {"gradient_evaluations": mean("unet", lambda r: r["gradient_evaluations"]),
                                "seconds": mean("unet", lambda r: r["seconds"]),
                                "converged": all(r["unet"]["converged"] for r in rows)},
            "lbfgs_from_zero": {"gradient_evaluations": mean("zero", lambda r: r["gradient_evaluations"]),
                                "seconds": mean("zero", lambda r: r["seconds"]),
                                "converged": all(r["zero"]["converged"] for r in rows)},
            "held_out": rows,
            "batched_from_unet": batched,
            "seconds_per_instance_unet_batched": batched["seconds_per_instance"],
            "seconds_per_instance_zero_single": round(zero_single, 3),
            "speedup_unet_batched_vs_zero_single": round(zero_single / max(batched["seconds_per_instance"], 1e-9), 2)}


def batch_leg(device, count, rank, steps=2, layout=None):
    """The batched inversions: `count` independent D2Q9 FP32 lattices with
    nx = 32 U{4..32}, ny = nx / 2, seeded disks (porosity U[0.5, 0.7]),
    T = 5000, one gradient evaluation (forward + loss + checkpointed adjoint)
    of every instance per batch step, all instances in shared kernels.  The
    layout (dense register kernels or packed fluid-only) is the batch
    autotuner's unless given."""
    import torch

    from paper_2310_00810_gb300 import autotune, lbm
    from paper_2310_00810_gb300 import workloads as W

    T = 5000
    spec = W.batch_sizes(count, seed=replica_seeds(rank)["batch"])
    sizes = [(nx, ny, 1) for nx, ny, _, _ in spec]
    geoms = [dict(kind=lbm.LBM_GEOM_DISKS, seed=sd, r_min=6, r_max=12, target_porosity=por)
             for nx, ny, por, sd in spec]
    b = lbm.Batch(9, sizes, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometries=geoms,
                  device=device)
    tuned = autotune.tune_batch(b) if layout is None else None
    if layout is not None:
        b.set_layout(layout)
    rho_in = b.new_inlet()
    for i, (nx, ny, _, sd) in enumerate(spec):
        b.view_inlet(rho_in, i).copy_(torch.as_tensor(1.0 + W.inlet_profile(ny, seed=2000 + sd), device=device))
    tau = torch.full((b.n,), 0.8, dtype=torch.float64, device=device)
    f_true = b.forward(rho_in, tau, 1.0)
    torch.cuda.synchronize(device)
    ut = b.velocity(f_true)  # observed fields; the evaluation starts from delta = 0
    rho0 = torch.ones_like(rho_in)
    f = b.new_state()
    lam = b.new_state()
    loss = torch.zeros(b.n, dtype=torch.float64, device=device)
    g_in = b.new_inlet()
    g_tau = torch.zeros(b.n, dtype=torch.float64, device=device)

    def one():
        b.forward(rho0, tau, 1.0, f)
        b.loss_grad(f, ut, None, loss, lam)
        b.adjoint(rho0, tau, 1.0, lam, g_in, g_tau)

    one()
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(steps):
        one()
    e1.record(b.stream)
    torch.cuda.synchronize(device)
    sec = e0.elapsed_time(e1) * 1e-3 / steps
    nodes = sum(nx * ny for nx, ny, _ in sizes)
    fluid = int(b.info.view(b.n, 4)[:, 3].sum().item())
    # algorithmic population bytes of one gradient evaluation: forward 2Qs + recompute 2Qs + adjoint 3Qs per
    # fluid node and time step
    alg = 7 * 9 * 4 * fluid * T
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks))["hbm_gbs"] if os.path.exists(peaks) else 6800.0
    return {"instances": b.n, "nodes": nodes, "fluid_nodes": fluid, "time_steps": T, "layout": b.layout,
            "tuner": None if tuned is None else {"layout": tuned["layout"], "timings_us": tuned["timings_us"],
                                                 "cached": tuned.get("cached")},
            "seconds_per_gradient_eval": round(sec, 4),
            "aggregate_mlups": round(nodes * T / sec / 1e6, 1),
            "hbm_gbs_algorithmic": round(alg / sec / 1e9, 1), "hbm_frac": round(alg / sec / 1e9 / hbm_peak, 4),
            "gradient_evals_per_s_per_instance": round(1.0 / sec, 3),
            "gradient_evals_per_s_total": round(b.n / sec, 2),
            "sizes": f"nx in [{min(s[0] for s in sizes)}, {max(s[0] for s in sizes)}], ny = nx / 2"}


def batch_invert_leg(device, count, rank, time_limit, n_single=2, max_nx=1024):
    """Time to 1e-3 relative error on the inlet profiles of `count` batched
    instances (the first `count` of the 64-instance recipe with nx <= max_nx,
    T = 5000): one L-BFGS per instance in lock step over the autotuned packed
    batch, against the plain single-instance inversion (autotuned plan, L-BFGS
    from delta = 0) of `n_single` of the same instances, run one after
    another."""
    import torch

    from paper_2310_00810_gb300 import autotune, lbm
    from paper_2310_00810_gb300 import invert as I
    from paper_2310_00810_gb300 import workloads as W

    T = 5000
    spec = [x for x in W.batch_sizes(64, seed=replica_seeds(rank)["batch"]) if x[0] <= max_nx][:count]
    sizes = [(nx, ny, 1) for nx, ny, _, _ in spec]
    geoms = [dict(kind=lbm.LBM_GEOM_DISKS, seed=sd, r_min=6, r_max=12, target_porosity=por)
             for nx, ny, por, sd in spec]
    b = lbm.Batch(9, sizes, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometries=geoms,
                  device=device)
    tuned = autotune.tune_batch(b)
    truth = [W.inlet_profile(ny, seed=2000 + sd) for _, ny, _, sd in spec]
    rho_in = b.new_inlet()
    for i in range(b.n):
        b.view_inlet(rho_in, i).copy_(torch.as_tensor(1.0 + truth[i], device=device))
    tau = torch.full((b.n,), 0.8, dtype=torch.float64, device=device)
    ut = b.velocity(b.forward(rho_in, tau, 1.0))
    inv = I.BatchInversion(b, ut, 1.0, 0.8)
    r = inv.run_lbfgs(truth_delta=truth, tol=1e-3, max_evals=600, time_limit=time_limit)
    singles = []
    for i in range(min(n_single, count)):
        nx, ny, _ = sizes[i]
        s = lbm.Solver(9, nx, ny, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=geoms[i],
                       device=device)
        autotune.tune(s)
        _, u1 = s.macroscopic(s.forward(torch.as_tensor(1.0 + truth[i], device=device),
                                        torch.tensor([0.8], dtype=torch.float64, device=device), 1.0))
        si = I.Inversion(s, u1.contiguous(), 1.0, tau0=0.8)
        rs = si.run_lbfgs(max_evals=600, tol=1e-3, truth_delta=truth[i], time_limit=time_limit / 2)
        singles.append({"instance": i, "size": f"{nx}x{ny}", "seconds": round(rs.seconds, 2),
                        "gradient_evaluations": si.evaluations, "converged": bool(rs.converged),
                        "batched_evaluations": r["evaluations"][i]})
        del s, si
    single_per_instance = float(np.mean([x["seconds"] for x in singles])) if singles else None
    batched_per_instance = r["seconds"] / b.n
    out = {"instances": b.n, "selection": f"the first {b.n} instances of the 64-instance recipe with nx <= {max_nx}",
           "time_steps": T, "layout": tuned["layout"], "method": "L-BFGS per instance, lock step",
           "start": "delta = 0", "sizes": [f"{nx}x{ny}" for nx, ny, _ in sizes],
           "rounds": r["rounds"], "seconds": round(r["seconds"], 2), "converged": r["converged"],
           "converged_count": int(sum(1 for x in r["rel_err"] if x is not None and x <= 1e-3)),
           "evaluations": r["evaluations"], "max_rel_err": max(x for x in r["rel_err"] if x is not None),
           "seconds_per_instance_batched": round(batched_per_instance, 3),
           "single_instance": singles, "seconds_per_instance_single": single_per_instance,
           "speedup_per_instance": (round(single_per_instance / batched_per_instance, 2)
                                    if single_per_instance else None),
           "time_limit_s": time_limit}
    del b, inv
    torch.cuda.empty_cache()
    return out


def run_e2e(P, args, device, barrier, world):
    """Same metric through the public API with host buffers: every step copies
    the inputs (inlet profile, tau, target velocity) from pinned host memory
    and reads the loss and gradient back."""
    import torch

    from paper_2310_00810_gb300 import lbm

    s, wl = P["solver"], P["wl"]
    h_rho = P["rho_in"].cpu().pin_memory()
    h_tau = P["tau"].cpu().pin_memory()
    h_ut = P["u_target"].cpu().pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    h_g = torch.empty(wl.ny, dtype=torch.float64).pin_memory()
    d_rho, d_tau, d_ut = torch.empty_like(P["rho_in"]), torch.empty_like(P["tau"]), torch.empty_like(P["u_target"])
    K = max(10, args.steps)

    def one():
        with torch.cuda.stream(s.stream):
            d_rho.copy_(h_rho, non_blocking=True)
            d_tau.copy_(h_tau, non_blocking=True)
            d_ut.copy_(h_ut, non_blocking=True)
        lbm.lbm_forward(s.plan, d_rho, d_tau, wl.rho_out, P["f"], s.ws, s.stream)
        lbm.lbm_loss_grad(s.plan, P["f"], d_ut, None, P["loss"], P["lam"], s.ws, s.stream)
        lbm.lbm_adjoint(s.plan, d_rho, d_tau, wl.rho_out, P["lam"], P["g_in"], P["g_tau"], s.ws, s.stream)
        with torch.cuda.stream(s.stream):
            h_loss.copy_(P["loss"], non_blocking=True)
            h_g.copy_(P["g_in"], non_blocking=True)

    one()  # warm call: the sweeps' graphs do not depend on these buffers, so nothing is captured anew
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(K):
        one()
    e1.record(s.stream)
    barrier()
    ms = e0.elapsed_time(e1)
    bi = (h_rho.numel() + h_tau.numel() + h_ut.numel()) * 8
    bo = (h_loss.numel() + h_g.numel()) * 8
    val = world * wl.nodes * wl.steps * K / (ms * 1e-3) / 1e6
    return {"value": round(val, 1), "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "steps": K, "ms_per_step": round(ms / K, 3)}


# DRAM bytes (read + write) per launch on the roofline lattices, from one ncu capture of each kernel
# on a smaller lattice of the same recipe, scaled by the fluid nodes processed (traffic grows in
# proportion): dense TMA kernels from disks4096x2048 (x 4 nodes), compact kernels from
# disks4096x2048 (x 4.0001 fluid nodes) and spheres256x128x128 (x 8.0006 fluid nodes).
HBM_TRAFFIC = {
    ("disks8192x4096", "dense"): {"stream-collide": 4 * (343.118080e6 + 201.248512e6),
                                  "adjoint": 4 * (642.651648e6 + 217.033472e6)},
    ("disks8192x4096", "compact"): {"stream-collide": 20132542 / 5032998 * (343.8e6 + 144.4e6),
                                    "adjoint": 20132542 / 5032998 * (527.8e6 + 158.9e6)},
    ("spheres512x256x256", "compact"): {"stream-collide": 15090843 / 1886221 * (297.2e6 + 112.1e6),
                                        "adjoint": 15090843 / 1886221 * (463.7e6 + 130.9e6)},
}


def kernel_rooflines(device, hbm_peak, name, n_launch, layout=None, aa=0):
    """Stream-collide and adjoint kernels alone on workload `name` (a lattice
    larger than L2 for the HBM roofline) in the given state layout: CUDA
    events around n_launch back-to-back launches of each.  Algorithmic bytes
    count fluid nodes: 2 Q s per stream-collide update, 3 Q s per adjoint
    update, plus the 4-byte link word of every node.  aa = 1: the in-place
    schedule of the fluid-only layout (its gather and local steps alternate;
    the times are their average)."""
    import torch

    from paper_2310_00810_gb300 import lbm
    from paper_2310_00810_gb300 import workloads as W

    wl = W.WORKLOADS[name]
    s = lbm.Solver(wl.q, wl.nx, wl.ny, wl.nz, precision=wl.precision, n_steps=n_launch, ckpt_stride=n_launch,
                   geometry=dict(kind=wl.geom_kind, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                                 target_porosity=wl.porosity), device=device, layout=layout)
    nf, N, q, sz = int(s.info[3].item()), wl.nodes, wl.q, wl.precision
    if aa:
        s.set_kernels(**dict(lbm.lbm_plan_get_kernels(s.plan), aa=1))
    rho_in = torch.tensor([1.001], dtype=torch.float64, device=device)
    tau = torch.tensor([wl.tau], dtype=torch.float64, device=device)
    a = s.new_state().zero_()
    b = s.new_state().zero_()
    out = {}
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # stream-collide: lbm_step(n) = 1 collide-only + (n-1) stream-collide + 1 stream-only launches
    lbm.lbm_step(s.plan, rho_in, tau, 1.0, a, b, 4, s.ws, s.stream)
    e[0].record(s.stream)
    lbm.lbm_step(s.plan, rho_in, tau, 1.0, a, b, n_launch, s.ws, s.stream)
    e[1].record(s.stream)
    # adjoint: a forward sweep, the loss seed, then the reverse sweep (stride = T: one segment,
    # n_launch - 2 recompute launches and n_launch adjoint launches)
    u_t = torch.zeros((s.plan.d, *s.plan.shape), dtype=torch.float64, device=device)
    lbm.lbm_forward(s.plan, rho_in, tau, 1.0, a, s.ws, s.stream)
    loss = torch.zeros(1, dtype=torch.float64, device=device)
    lbm.lbm_loss_grad(s.plan, a, u_t, None, loss, b, s.ws, s.stream)
    g_in = torch.zeros(1, dtype=torch.float64, device=device)
    g_tau = torch.zeros(1, dtype=torch.float64, device=device)
    lbm.lbm_adjoint(s.plan, rho_in, tau, 1.0, b, g_in, g_tau, s.ws, s.stream)  # warm (graph capture)
    e[2].record(s.stream)
    lbm.lbm_adjoint(s.plan, rho_in, tau, 1.0, b, g_in, g_tau, s.ws, s.stream)
    e[3].record(s.stream)
    torch.cuda.synchronize(device)
    t_sc = e[0].elapsed_time(e[1]) * 1e-3 / (n_launch + 1)
    t_rev = e[2].elapsed_time(e[3]) * 1e-3
    t_adj = (t_rev - (n_launch - 2) * t_sc) / n_launch
    for kern, t, per in (("stream-collide", t_sc, 2 * q * sz), ("adjoint", t_adj, 3 * q * sz)):
        byts = per * nf + 4 * N
        ach = byts / t / 1e9
        tr = HBM_TRAFFIC.get((name, s.layout) + (("in place",) if aa and s.layout == "compact" else ()),
                             {}).get(kern)
        sched = ", in place" if aa and s.layout == "compact" else ""
        out[kern] = {"bound": "hbm", "kernel": f"{kern} on {name} ({s.layout} layout{sched})", "achieved": round(ach, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                     "frac_of_nominal_8tbs": round(ach / 8000.0, 4),
                     "traffic": round(tr) if tr else None, "bytes_per_launch": byts,
                     "us_per_launch": round(t * 1e6, 2), "fluid_nodes": nf, "nodes": N,
                     "glups_fluid": round(nf / t / 1e9, 2)}
    del a, b, s
    torch.cuda.empty_cache()
    return out


def cpu_baseline(sample_steps, threads=None):
    """The FP64 C oracle, as it stands, on a bounded sample of the workload:
    the full gradient (forward + checkpointed reverse sweep) over the first
    `sample_steps` time steps of the same 512x256 problem."""
    from oracle import oracle as O
    from paper_2310_00810_gb300 import workloads as W

    wl = W.WORKLOADS[WORKLOAD]
    m, _ = O.geometry(9, wl.nx, wl.ny, kind=O.GEOM_DISKS, seed=wl.seed, r_min=wl.r_min, r_max=wl.r_max,
                      porosity=wl.porosity)
    rin = wl.rho_out + W.inlet_profile(wl.ny, seed=2000)
    ut = np.zeros((2, wl.ny, wl.nx))
    cores = threads if threads else (os.cpu_count() or 1)
    O.set_threads(cores)
    t0 = time.perf_counter()
    O.gradient(9, m, rin, wl.rho_out, wl.tau, sample_steps, ut, ckpt_stride=max(1, int(math.sqrt(sample_steps))))
    dt = time.perf_counter() - t0
    O.set_threads(1)
    return {"value": round(wl.nodes * sample_steps / dt / 1e6, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{WORKLOAD} gradient over the first {sample_steps} of 20000 time steps "
                      f"({dt:.1f} s, FP64 C; per-node loops on {cores} OpenMP threads)"}


def cpu_model() -> str:
    """The host CPU as the kernel reports it (model name, or the Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    parts = {l.split(":", 1)[0].strip(): l.split(":", 1)[1].strip() for l in info.splitlines() if ":" in l}
    return f"Arm implementer {parts.get('CPU implementer', '?')} part {parts.get('CPU part', '?')}"


def cpu_other_workloads(threads):
    """The oracle's full gradient on the 64x32 FP64 channel (T = 1000) and on a
    bounded sample of the 128x64x64 D3Q19 packing (the first 10 of its 10000
    steps), on `threads` OpenMP threads: MLUPS as nodes x steps / s."""
    from oracle import oracle as O
    from paper_2310_00810_gb300 import workloads as W

    O.set_threads(threads)
    out = {}
    c1 = W.WORKLOADS["channel64x32"]
    m1, _ = O.geometry(9, c1.nx, c1.ny, kind=O.GEOM_CHANNEL)
    t0 = time.perf_counter()
    O.gradient(9, m1, 1.001, 1.0, c1.tau, c1.steps, np.zeros((2, c1.ny, c1.nx)), ckpt_stride=32)
    out["channel64x32_full_gradient_mlups"] = round(c1.nodes * c1.steps / (time.perf_counter() - t0) / 1e6, 3)
    c3 = W.WORKLOADS["spheres128x64x64"]
    m3, _ = O.geometry(19, c3.nx, c3.ny, c3.nz, kind=O.GEOM_SPHERES, seed=c3.seed, r_min=c3.r_min, r_max=c3.r_max,
                       porosity=c3.porosity)
    t0 = time.perf_counter()
    O.gradient(19, m3, 1.001, 1.0, c3.tau, 10, np.zeros((3, c3.nz, c3.ny, c3.nx)), ckpt_stride=3)
    out["spheres128x64x64_gradient_sample_mlups"] = round(c3.nodes * 10 / (time.perf_counter() - t0) / 1e6, 3)
    O.set_threads(1)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    K, Wm = args.steps, max(0, args.warmup)
    sample = max(4, min(args.cpu_sample_steps, 30))
    for _ in range(min(Wm, 1)):
        cpu_baseline(4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(K):
        vals.append(cpu_baseline(sample))
    wall = time.perf_counter() - t0
    from paper_2310_00810_gb300 import workloads as W

    wl = W.WORKLOADS[WORKLOAD]
    value = K * wl.nodes * sample / wall / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
           "steps": K, "warmup": Wm, "ms_per_step": round(wall / K * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD} (oracle sample: {sample} of 20000 time steps per step)"},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                            "sample": f"gradient over the first {sample} time steps of {WORKLOAD}, per step "
                                      f"(per-node loops on {vals[-1]['cores']} OpenMP threads)"},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_kernels(args):
    import torch

    from paper_2310_00810_gb300 import build

    build.build()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks))["hbm_gbs"] if os.path.exists(peaks) else 6800.0
    print(json.dumps({"mode": "kernels", "lattice": args.lattice,
                      "layout": args.layout,
                      "aa": args.aa,
                      "kernels": kernel_rooflines(device, hbm_peak, args.lattice, args.launches, args.layout,
                                                  args.aa)}),
          flush=True)


def run_unet(args):
    """Training throughput of the learned initialiser's kernels alone: Adam
    steps of the U-Net (base 32, 256x128, batch 16) on a fixed synthetic batch."""
    import torch

    from paper_2310_00810_gb300 import build
    from paper_2310_00810_gb300 import unet as N

    build.build()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    N.unet_set_engine(N.ENGINE_TCGEN05 if args.unet_engine == "tcgen05" else N.ENGINE_MMA_SYNC)
    B, H, W, base = args.unet_batch, 128, 256, 32
    net = N.UNet(base=base, height=H, width=W, batch=B, seed=1, device=device)
    r = np.random.Generator(np.random.PCG64(2))
    x = np.zeros((B, H, W, N.IN_CHANNELS), np.float32)
    x[..., :3] = r.normal(0, 1, (B, H, W, 3))
    xd = torch.as_tensor(x, device=device).to(torch.bfloat16).view(torch.int16).contiguous()
    t = torch.as_tensor(r.normal(1, 0.3, (B, H)).astype(np.float32), device=device)
    for _ in range(max(1, args.warmup)):
        net.train_step(xd, t, 1e-3)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    torch.cuda.nvtx.range_push("timed_step")
    for _ in range(args.steps):
        net.train_step(xd, t, 1e-3)
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize(device)
    dt = e0.elapsed_time(e1) * 1e-3
    flops = 3 * unet_flops_per_sample(base, H, W) * B * args.steps
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(peaks))["bf16_tflops"] if os.path.exists(peaks) else 1900.0
    print(json.dumps({"mode": "unet", "engine": args.unet_engine, "status": N.unet_get_status(),
                      "samples_per_s": round(B * args.steps / dt, 1),
                      "ms_per_step": round(dt / args.steps * 1e3, 3), "tflops": round(flops / dt / 1e12, 2),
                      "bf16_peak_tflops": peak, "frac": round(flops / dt / 1e12 / peak, 4),
                      "flops_per_sample_forward": unet_flops_per_sample(base, H, W)}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "kernels":
        run_kernels(args)
    elif args.mode == "unet":
        run_unet(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
