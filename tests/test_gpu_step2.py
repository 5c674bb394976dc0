"""Two stream-collide steps per launch (the temporally blocked TMA kernel of
the dense D2Q9 FP32 layout) against the FP64 oracle and against one step per
launch: lbm_step from random states, and whole forward / gradient sweeps
whose checkpoint strides put the states the reverse sweep needs at odd and
even steps, on ragged tiles (nx not a multiple of 128, ny not a multiple of
the tile height) and on a lattice with more tiles than thread blocks."""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _solver(nx, ny, T, rows, two, stride=0, seed=7, profile=True):
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=seed, r_min=3, r_max=7, target_porosity=0.65, inlet_buffer=4)
    s = lbm.Solver(9, nx, ny, precision=4, n_steps=T, ckpt_stride=stride,
                   inlet_kind=lbm.LBM_INLET_PROFILE if profile else lbm.LBM_INLET_CONST, geometry=g, layout="dense")
    lbm.lbm_plan_set_kernels(s.plan, step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA,
                             tma_rows=rows, steps_per_launch=2 if two else 1)
    assert lbm.lbm_plan_get_kernels(s.plan)["steps_per_launch"] == (2 if two else 1)
    return s


SIZES = [(200, 37), (128, 64), (1024, 512)]


@pytest.mark.parametrize("rows", [8, 4])
@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("n", [2, 3, 6])
def test_step_pairs_from_random_state(nx, ny, rows, n):
    s = _solver(nx, ny, 1, rows, True)
    m = s.mask_field.cpu().numpy()
    q = 9
    _, w, _ = O.lattice(q)
    f0 = W.perturbation((q, ny, nx), seed=11, scale=2e-3)
    f0[:, m == 1] = 0.0
    rin = 1.0 + W.inlet_profile(ny, seed=12)
    tau = 0.8
    got = s.step(dev(rin), dev([tau]), 1.0, dev(f0, torch.float32), n).cpu().numpy()
    want = O.forward(q, m, rin, 1.0, tau, n, f0=f0 + w.reshape(q, 1, 1)) - w.reshape(q, 1, 1)
    fl = m == 0
    assert rel(got[:, fl], want[:, fl]) < 1e-5
    one = _solver(nx, ny, 1, rows, False)
    ref = one.step(dev(rin), dev([tau]), 1.0, dev(f0, torch.float32), n).cpu().numpy()
    assert np.abs(got[:, fl] - ref[:, fl]).max() <= 1e-6 * np.abs(ref[:, fl]).max()


@pytest.mark.parametrize("rows", [8, 4])
@pytest.mark.parametrize("nx,ny,T,stride", [(200, 37, 41, 6), (200, 37, 40, 7), (1024, 512, 24, 5),
                                            (512, 256, 60, 0)])
def test_sweeps_with_step_pairs_match_the_oracle(nx, ny, T, stride, rows):
    s = _solver(nx, ny, T, rows, True, stride=stride)
    m = s.mask_field.cpu().numpy()
    rin = 1.0 + W.inlet_profile(ny, seed=21)
    ut = W.perturbation((2, ny, nx), seed=22, scale=1e-4)
    f = s.forward(dev(rin), dev([0.8]), 1.0)
    L, lam = s.loss_grad(f, dev(ut))
    g_in, g_tau = s.adjoint(dev(rin), dev([0.8]), 1.0, lam)
    k = stride if stride else int(np.ceil(np.sqrt(T)))
    Lw, gw, gtw, fw = O.gradient(9, m, rin, 1.0, 0.8, T, ut, ckpt_stride=k, return_fT=True)
    _, u = s.macroscopic(f)
    _, uw = O.macroscopic(9, m, fw)
    assert rel(u.cpu().numpy(), uw) < 1e-4
    assert abs(L.item() - Lw) <= 1e-4 * abs(Lw)
    assert rel(g_in.cpu().numpy(), gw) < 1e-3
    assert abs(g_tau.item() - gtw) <= 1e-3 * abs(gtw)
    assert s.status() == lbm.LBM_OK


def test_step_pairs_constant_head_and_rest_fixed_point():
    """rho_in = rho_out from rest stays exactly zero through paired steps."""
    s = _solver(256, 64, 101, 8, True, profile=False)
    f = s.forward(dev([1.0]), dev([0.8]), 1.0)
    assert torch.count_nonzero(f).item() == 0
