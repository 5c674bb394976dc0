"""The autotuner picks a kernel configuration by timing, caches it, and the
tuned plan still matches the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import autotune
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


def dev(x):
    return torch.as_tensor(np.asarray(x, np.float64), device="cuda")


@pytest.mark.parametrize("q", [9, 19])
def test_tune_then_parity(q, tmp_path):
    if q == 9:
        shape, g = (40, 96), dict(kind=lbm.LBM_GEOM_DISKS, seed=5, r_min=3, r_max=6, target_porosity=0.7)
        nx, ny, nz, T = 96, 40, 1, 50
    else:
        shape, g = (10, 12, 40), dict(kind=lbm.LBM_GEOM_SPHERES, seed=5, r_min=2, r_max=2, target_porosity=0.8,
                                     inlet_buffer=4)
        nx, ny, nz, T = 40, 12, 10, 20
    s = lbm.Solver(q, nx, ny, nz, precision=4, n_steps=T, inlet_kind=lbm.LBM_INLET_PROFILE, geometry=g)
    cache = str(tmp_path / "tune.json")
    r1 = autotune.tune(s, t_tune=16, repeats=1, cache=cache)
    assert not r1["cached"] and r1["timings_us"]
    r2 = autotune.tune(s, t_tune=16, repeats=1, cache=cache)
    assert r2["cached"] and r2["choice"] == r1["choice"]
    assert lbm.lbm_plan_get_kernels(s.plan)["step_family"] == r1["choice"]["step_family"]
    m = s.mask_field.cpu().numpy()
    n_in = ny * nz
    rin = 1.0 + W.inlet_profile(n_in, seed=6)
    ut = W.perturbation((s.plan.d, *shape), seed=7, scale=1e-3)
    f = s.forward(dev(rin), dev([0.8]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([0.8]), 1.0, lam)
    Lw, gw, gtw = O.gradient(q, m, rin.reshape((nz, ny) if q == 19 else (ny,)), 1.0, 0.8, T, ut, ckpt_stride=7)
    assert abs(L.item() - Lw) <= 1e-4 * Lw
    assert np.linalg.norm(g_in.cpu().numpy() - np.ravel(gw)) <= 1e-3 * np.linalg.norm(gw)
    assert abs(g_tau.item() - gtw) <= 1e-3 * abs(gtw)
