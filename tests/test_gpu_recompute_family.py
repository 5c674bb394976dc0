"""The reverse sweep's segment recompute on another kernel family than the
forward sweep (lbm_kernel_choice.recompute_family): every family computes
the same step, so the gradient matches the oracle at the FP32 tolerances and
the one-family run closely, with the recompute overlapped or serial."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("family", [lbm.LBM_FAMILY_VEC, lbm.LBM_FAMILY_SCALAR, lbm.LBM_FAMILY_TMA])
@pytest.mark.parametrize("overlap", [1, 0])
def test_recompute_family_gives_the_same_gradient(family, overlap):
    T, stride = 45, 7
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=17, r_min=3, r_max=6, target_porosity=0.7, inlet_buffer=4)
    s = lbm.Solver(9, 256, 64, precision=4, n_steps=T, ckpt_stride=stride, inlet_kind=lbm.LBM_INLET_PROFILE,
                   geometry=g, layout="dense")
    m = s.mask_field.cpu().numpy()
    rin = 1.0 + W.inlet_profile(64, seed=18)
    ut = W.perturbation((2, 64, 256), seed=19, scale=1e-4)
    out = []
    for rec in (lbm.LBM_FAMILY_AUTO, family):
        s.set_kernels(step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA, overlap=overlap,
                      recompute_family=rec)
        assert lbm.lbm_plan_get_kernels(s.plan)["recompute_family"] == rec
        f = s.forward(dev(rin), dev([0.8]), 1.0)
        L, lam = s.loss_grad(f, dev(ut))
        g_in, g_tau = s.adjoint(dev(rin), dev([0.8]), 1.0, lam)
        torch.cuda.synchronize()
        out.append((L.item(), g_in.cpu().numpy(), g_tau.item()))
    (L0, gi0, gt0), (L1, gi1, gt1) = out
    assert L1 == L0
    assert rel(gi1, gi0) < 1e-5 and abs(gt1 - gt0) <= 1e-5 * abs(gt0)
    Lw, gw, gtw = O.gradient(9, m, rin, 1.0, 0.8, T, ut, ckpt_stride=stride)
    assert rel(gi1, gw) < 1e-3 and abs(gt1 - gtw) <= 1e-3 * abs(gtw)


def test_recompute_family_is_checked():
    s = lbm.Solver(9, 64, 32, precision=4, n_steps=4, geometry=dict(kind=lbm.LBM_GEOM_CHANNEL))
    with pytest.raises(lbm.LBMError):
        lbm.lbm_plan_set_kernels(s.plan, recompute_family=9)
