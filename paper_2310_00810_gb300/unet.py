"""Binding of ``include/unet.h`` (argument marshalling only) and the training
and inference code of the learned inlet-profile initialiser: training data from the library's own
forward solves, training with the library's forward/backward/Adam kernels,
and inference as the starting point of the gradient inversion.

The network (a 4-level U-Net, see the header) reads the observed steady
velocity field and the obstacle mask of a lattice and predicts the inlet
density profile delta(y) / 1e-3; the zero-initialised inversion is both the
fallback and the yardstick of its error (``evaluate``)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import time

import numpy as np
import torch

from . import lbm
from . import workloads as W

IN_CHANNELS = 8
VELOCITY_SCALE = 1e3  # the input channels carry u / 1e-3


class unet_desc(C.Structure):
    _fields_ = [("base", C.c_int32), ("height", C.c_int32), ("width", C.c_int32), ("batch", C.c_int32)]


def _ptr(t, dtype=None, numel=None):
    return lbm._ptr(t, dtype, numel)


def unet_param_layout(base: int):
    n_t = C.c_int32()
    n_p = C.c_int64()
    lbm._check(lbm.load().unet_param_layout(base, C.byref(n_t), C.byref(n_p), None, None), "unet_param_layout")
    offs = np.zeros(n_t.value, np.int64)
    cnts = np.zeros(n_t.value, np.int64)
    lbm._check(lbm.load().unet_param_layout(base, C.byref(n_t), C.byref(n_p), offs.ctypes.data_as(C.c_void_p),
                                            cnts.ctypes.data_as(C.c_void_p)), "unet_param_layout")
    return offs, cnts, n_p.value


def unet_workspace_size(desc: unet_desc) -> int:
    n = C.c_size_t()
    lbm._check(lbm.load().unet_workspace_size(C.byref(desc), C.byref(n)), "unet_workspace_size")
    return n.value


def unet_pack_input(desc, u, mask, scale, x, stream=None):
    lbm._check(lbm.load().unet_pack_input(C.byref(desc), _ptr(u, torch.float64), _ptr(mask, torch.uint8),
                                          float(scale), _ptr(x, torch.int16), lbm._stream(stream)), "unet_pack_input")


def unet_prepare_weights(desc, params, ws, stream=None):
    lbm._check(lbm.load().unet_prepare_weights(C.byref(desc), _ptr(params, torch.float32), _ptr(ws, torch.uint8),
                                               lbm._stream(stream)), "unet_prepare_weights")


def unet_forward(desc, x, out, ws, stream=None):
    lbm._check(lbm.load().unet_forward(C.byref(desc), _ptr(x, torch.int16), _ptr(out, torch.float32),
                                       _ptr(ws, torch.uint8), lbm._stream(stream)), "unet_forward")


def unet_backward(desc, x, target, loss, grad, ws, stream=None):
    lbm._check(lbm.load().unet_backward(C.byref(desc), _ptr(x, torch.int16), _ptr(target, torch.float32),
                                        _ptr(loss, torch.float32), _ptr(grad, torch.float32), _ptr(ws, torch.uint8),
                                        lbm._stream(stream)), "unet_backward")


ENGINE_MMA_SYNC, ENGINE_TCGEN05 = 0, 1


def unet_set_engine(engine: int) -> None:
    """The convolutions' GEMM engine (process-wide): ENGINE_TCGEN05 (default, where the shapes allow it) or
    ENGINE_MMA_SYNC."""
    lbm._check(lbm.load().unet_set_engine(engine), "unet_set_engine")


def unet_get_status() -> int:
    """LBM_OK, or LBM_ERR_TIMEOUT if a bounded wait of a tensor-core kernel gave up since the last call."""
    return lbm.load().unet_get_status()


def unet_adam(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    n = params.numel()
    lbm._check(lbm.load().unet_adam(n, _ptr(params, torch.float32), _ptr(m, torch.float32, n),
                                    _ptr(v, torch.float32, n), _ptr(grad, torch.float32, n), int(t), float(lr),
                                    float(beta1), float(beta2), float(eps), lbm._stream(stream)), "unet_adam")


def param_shapes(base: int):
    """Shapes in the order of unet_param_layout (3x3: [3,3,cin,cout]; transposed: [2,2,cin,cout])."""
    c = [base << l for l in range(4)]
    s, prev = [], IN_CHANNELS
    for l in range(4):
        s += [(3, 3, prev, c[l]), (c[l],), (3, 3, c[l], c[l]), (c[l],)]
        prev = c[l]
    for l in (2, 1, 0):
        s += [(2, 2, c[l + 1], c[l]), (c[l],), (3, 3, 2 * c[l], c[l]), (c[l],), (3, 3, c[l], c[l]), (c[l],)]
    s += [(c[0],), (1,)]
    return s


class UNet:
    """Parameters (FP32 masters), Adam state and workspace of one network on one device."""

    def __init__(self, base=32, height=128, width=256, batch=16, seed=0, device="cuda"):
        self.device = torch.device(device)
        self.desc = unet_desc(base, height, width, batch)
        self.offsets, self.counts, n = unet_param_layout(base)
        shapes = param_shapes(base)
        assert len(shapes) == len(self.offsets) and all(int(np.prod(s)) == c for s, c in zip(shapes, self.counts))
        rng = np.random.Generator(np.random.PCG64(seed))
        p = np.zeros(n, np.float32)
        for o, s in zip(self.offsets, shapes):
            if len(s) > 1:  # He-normal: fan-in = taps x input channels (one tap per output of a transposed conv)
                fan_in = (s[0] * s[1] if s[0] == 3 else 1) * s[2]
                p[o:o + int(np.prod(s))] = rng.normal(0.0, np.sqrt(2.0 / fan_in), int(np.prod(s)))
            elif s[0] == base and o == self.offsets[-2]:  # head weight
                p[o:o + s[0]] = rng.normal(0.0, np.sqrt(1.0 / s[0]), s[0])
        self.params = torch.tensor(p, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.ws = torch.empty(unet_workspace_size(self.desc), dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.out = torch.zeros((batch, height), dtype=torch.float32, device=self.device)
        self.t = 0

    def shapes(self):
        return param_shapes(self.desc.base)

    def tensors(self):
        """Views of the FP32 master parameters, shaped."""
        return [self.params[o:o + int(c)].view(s) for o, c, s in zip(self.offsets, self.counts, self.shapes())]

    def forward(self, x):
        unet_prepare_weights(self.desc, self.params, self.ws)
        unet_forward(self.desc, x, self.out, self.ws)
        return self.out

    def loss_and_grad(self, x, target):
        self.forward(x)
        unet_backward(self.desc, x, target, self.loss, self.grad, self.ws)
        return self.loss

    def train_step(self, x, target, lr):
        self.loss_and_grad(x, target)
        self.t += 1
        unet_adam(self.params, self.m, self.v, self.grad, self.t, lr)
        return self.loss


# ------------------------------------------------------------- data

@dataclasses.dataclass
class Dataset:
    x: torch.Tensor        # int16 (bf16 bits) [n][h][w][8]
    target: torch.Tensor   # float32 [n][h]: delta / 1e-3
    porosity: np.ndarray
    seeds: np.ndarray


def sample_recipe(seed: int):
    """Porosity U[0.5, 0.7] and disk radii 6-12 lu for one training solve (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return float(rng.uniform(0.5, 0.7))


def generate(n: int, seed0: int, nx: int = 256, ny: int = 128, steps: int = 10000, chunk: int = 64, tau: float = 0.8,
             device="cuda", r_min: int = 6, r_max: int = 12) -> Dataset:
    """n forward solves through the library (batched lattices), each a seeded
    disk packing with porosity U[0.5, 0.7] and a 4-mode sine inlet profile
    (seed + 2000 offset as the benchmark's profiles), run T steps from rest;
    returns the packed network inputs and the profile targets."""
    dev = torch.device(device)
    xs, ts, por, seeds = [], [], [], []
    desc = None
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        sd = [seed0 + c0 + i for i in range(m)]
        geoms = [dict(kind=lbm.LBM_GEOM_DISKS, seed=s, r_min=r_min, r_max=r_max, target_porosity=sample_recipe(s))
                 for s in sd]
        # the packed fluid-only batch (about twice the dense batch's speed on these packings)
        b = lbm.Batch(9, [(nx, ny, 1)] * m, precision=4, n_steps=steps, inlet_kind=lbm.LBM_INLET_PROFILE,
                      geometries=geoms, device=dev, layout="compact")
        rho_in = b.new_inlet()
        tgt = np.zeros((m, ny), np.float32)
        for i, s in enumerate(sd):
            d = W.inlet_profile(ny, seed=s + 2000)
            tgt[i] = d / 1e-3
            b.view_inlet(rho_in, i).copy_(torch.as_tensor(1.0 + d, device=dev))
        tau_t = torch.full((m,), tau, dtype=torch.float64, device=dev)
        f = b.forward(rho_in, tau_t, 1.0)
        u = _batch_velocity(b, f, dev)
        desc = unet_desc(8, ny, nx, m)
        x = torch.empty((m, ny, nx, IN_CHANNELS), dtype=torch.int16, device=dev)
        unet_pack_input(desc, u, b.mask[: m * nx * ny], VELOCITY_SCALE, x)
        torch.cuda.synchronize(dev)
        xs.append(x)
        ts.append(torch.as_tensor(tgt, device=dev))
        por.append(b.porosity.cpu().numpy())
        seeds += sd
        del b, f, u
    return Dataset(torch.cat(xs), torch.cat(ts), np.concatenate(por), np.array(seeds))


def _batch_velocity(b, f, dev):
    """Velocity fields [m][2][ny][nx] of a batch of equal-size D2Q9 lattices."""
    nx, ny, _ = b.sizes[0]
    out = torch.empty((b.n, 2, ny, nx), dtype=torch.float64, device=dev)
    for i in range(b.n):
        p = lbm.Plan(9, nx, ny, 1, b.precision, 1)
        o = int(b.node_off[i])
        lbm.lbm_bind_geometry(p, b.link[o:o + nx * ny])
        lbm.lbm_macroscopic(p, b.view_state(f, i).contiguous(), None, out[i])
    return out


def train(net: UNet, data: Dataset, epochs: int, lr: float = 1e-3, seed: int = 0, log=None, lr_final=None):
    """Adam over shuffled minibatches of the network's batch size, the learning
    rate decaying from lr to lr_final (cosine over the epochs; constant if
    lr_final is None); returns the loss history."""
    import math

    B = net.desc.batch
    n = (data.x.shape[0] // B) * B
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = []
    for ep in range(epochs):
        lr_ep = lr if lr_final is None or epochs < 2 else (
            lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * ep / (epochs - 1))))
        order = torch.as_tensor(rng.permutation(data.x.shape[0])[:n], device=data.x.device)
        tot = 0.0
        for i in range(0, n, B):
            idx = order[i:i + B]
            x = data.x[idx].contiguous()
            t = data.target[idx].contiguous()
            tot += float(net.train_step(x, t, lr_ep).item())
        hist.append(tot / (n // B))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4g}")
    return hist


def predict(net: UNet, x: torch.Tensor) -> torch.Tensor:
    """Profiles (delta / 1e-3) for inputs x, in batches of the network's batch size."""
    B = net.desc.batch
    outs = []
    for i in range(0, x.shape[0], B):
        xb = x[i:i + B]
        m = xb.shape[0]
        if m < B:
            xb = torch.cat([xb, xb[-1:].expand(B - m, *xb.shape[1:])])
        outs.append(net.forward(xb.contiguous()).clone()[:m])
    return torch.cat(outs)


def evaluate(net: UNet, seeds, nx: int = 256, ny: int = 128, steps: int = 10000, tau: float = 0.8, device="cuda",
             tol: float = 1e-3, max_evals: int = 400, time_limit: float = 120.0, r_min: int = 6, r_max: int = 12):
    """For each held-out seed: the prediction's relative error, and the L-BFGS
    inversion (the library's forward/adjoint) from the prediction and from
    delta = 0, to `tol` relative error: gradient evaluations and seconds."""
    from . import invert as I

    dev = torch.device(device)
    rows = []
    data = generate(len(seeds), int(seeds[0]), nx, ny, steps, chunk=len(seeds), tau=tau, device=device,
                    r_min=r_min, r_max=r_max)
    guess = predict(net, data.x).cpu().numpy().astype(np.float64)
    for i, s in enumerate(seeds):
        g = dict(kind=lbm.LBM_GEOM_DISKS, seed=int(s), r_min=r_min, r_max=r_max,
                 target_porosity=sample_recipe(int(s)))
        sv = lbm.Solver(9, nx, ny, precision=4, n_steps=steps, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=g,
                        device=dev)
        truth = data.target[i].cpu().numpy().astype(np.float64) * 1e-3
        f = sv.forward(torch.as_tensor(1.0 + truth, device=dev), torch.tensor([tau], dtype=torch.float64, device=dev),
                       1.0)
        _, ut = sv.macroscopic(f)
        row = {"seed": int(s), "prediction_rel_err": float(np.linalg.norm(guess[i] * 1e-3 - truth) / np.linalg.norm(truth))}
        for name, theta0 in (("zero", np.zeros(ny)), ("unet", guess[i])):
            inv = I.Inversion(sv, ut.contiguous(), 1.0, theta0=theta0, tau0=tau)
            t0 = time.perf_counter()
            res = inv.run_lbfgs(max_evals=max_evals, tol=tol, truth_delta=truth, time_limit=time_limit)
            row[name] = {"converged": bool(res.converged), "gradient_evaluations": inv.evaluations,
                         "seconds": round(time.perf_counter() - t0, 3), "rel_err": res.rel_err_inlet}
        rows.append(row)
    return rows


def evaluate_batched(net: UNet, seeds, nx: int = 256, ny: int = 128, steps: int = 10000, tau: float = 0.8,
                     device="cuda", tol: float = 1e-3, max_evals: int = 400, time_limit: float = 120.0,
                     r_min: int = 6, r_max: int = 12, from_guess: bool = True):
    """The held-out inversions of `evaluate`, all seeds in one packed batch
    (lock-step L-BFGS, invert.BatchInversion), started from the network's
    guesses (or from delta = 0): rounds (batched gradient evaluations),
    seconds for all of them, and the per-instance results."""
    from . import autotune
    from . import invert as I

    dev = torch.device(device)
    data = generate(len(seeds), int(seeds[0]), nx, ny, steps, chunk=len(seeds), tau=tau, device=device,
                    r_min=r_min, r_max=r_max)
    guess = predict(net, data.x).cpu().numpy().astype(np.float64)
    geoms = [dict(kind=lbm.LBM_GEOM_DISKS, seed=int(s), r_min=r_min, r_max=r_max, target_porosity=sample_recipe(int(s)))
             for s in seeds]
    b = lbm.Batch(9, [(nx, ny, 1)] * len(seeds), precision=4, n_steps=steps, inlet_kind=lbm.LBM_INLET_PROFILE,
                  geometries=geoms, device=dev)
    tuned = autotune.tune_batch(b)
    truth = [data.target[i].cpu().numpy().astype(np.float64) * 1e-3 for i in range(len(seeds))]
    rho_in = b.new_inlet()
    for i in range(len(seeds)):
        b.view_inlet(rho_in, i).copy_(torch.as_tensor(1.0 + truth[i], device=dev))
    taus = torch.full((len(seeds),), tau, dtype=torch.float64, device=dev)
    ut = b.velocity(b.forward(rho_in, taus, 1.0))
    theta0 = [guess[i] if from_guess else np.zeros(ny) for i in range(len(seeds))]
    inv = I.BatchInversion(b, ut, 1.0, tau, theta0=theta0)
    r = inv.run_lbfgs(truth_delta=truth, tol=tol, max_evals=max_evals, time_limit=time_limit)
    return {"instances": len(seeds), "layout": tuned["layout"], "start": "network guess" if from_guess else "delta = 0",
            "rounds": r["rounds"], "seconds": round(r["seconds"], 3), "converged": r["converged"],
            "evaluations": r["evaluations"], "rel_err": r["rel_err"],
            "seconds_per_instance": round(r["seconds"] / len(seeds), 3)}
