"""Failure detection without a GPU fault: a bounded device-side wait that is
made to give up returns LBM_ERR_TIMEOUT through the status word, the kernel
returns, and the context stays usable; a non-finite input latches
LBM_ERR_NONFINITE."""
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


def dev(x):
    return torch.as_tensor(np.asarray(x, np.float64), device="cuda")


def test_grid_barrier_timeout_is_reported_and_context_survives(monkeypatch):
    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=3, r_min=3, r_max=6, target_porosity=0.7)
    monkeypatch.setenv("LBM_PERSIST", "1")
    monkeypatch.setenv("LBM_SPIN_LIMIT", "1")  # each grid-barrier wait gives up after one spin
    s = lbm.Solver(9, 128, 64, precision=4, n_steps=50, geometry=g)
    s.forward(dev([1.001]), dev([0.8]), 1.0)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_ERR_TIMEOUT
    assert s.status() == lbm.LBM_OK  # reading clears the word
    # the context is intact: a normal plan on the same geometry still matches the oracle
    monkeypatch.delenv("LBM_SPIN_LIMIT")
    s2 = lbm.Solver(9, 128, 64, precision=4, n_steps=50, link=s.link, mask=s.mask)
    f = s2.forward(dev([1.001]), dev([0.8]), 1.0)
    _, u = s2.macroscopic(f)
    m = s.mask_field.cpu().numpy()
    _, uw = O.macroscopic(9, m, O.forward(9, m, 1.001, 1.0, 0.8, 50))
    assert np.linalg.norm(u.cpu().numpy() - uw) / np.linalg.norm(uw) < 1e-4
    assert s2.status() == lbm.LBM_OK


def test_nonfinite_parameter_is_reported():
    g = dict(kind=lbm.LBM_GEOM_CHANNEL)
    s = lbm.Solver(9, 64, 32, precision=4, n_steps=20, geometry=g)
    ut = dev(W.perturbation((2, 32, 64), seed=1, scale=1e-3))
    f = s.forward(dev([float("nan")]), dev([0.8]), 1.0)
    L, lam = s.loss_grad(f, ut)
    torch.cuda.synchronize()
    assert s.status() == lbm.LBM_ERR_NONFINITE


def test_tma_wait_gives_up_once_per_sweep(monkeypatch):
    """The TMA producers are told to issue nothing (LBM_TEST_STALL_TMA), so
    the consumers' first wait is one that nothing completes.  It gives up
    after LBM_WAIT_US (50 ms here), latches LBM_ERR_TIMEOUT, and every later
    TMA launch of the 400-step sweep returns at entry: the sweep ends after
    about one wait limit instead of one per launch (20 s).  The context stays
    usable."""
    import time

    g = dict(kind=lbm.LBM_GEOM_DISKS, seed=3, r_min=3, r_max=6, target_porosity=0.7)
    monkeypatch.setenv("LBM_TEST_STALL_TMA", "1")
    monkeypatch.setenv("LBM_WAIT_US", "50000")
    s = lbm.Solver(9, 256, 128, precision=4, n_steps=400, geometry=g, layout="dense")
    lbm.lbm_plan_set_kernels(s.plan, step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.forward(dev([1.001]), dev([0.8]), 1.0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert s.status() == lbm.LBM_ERR_TIMEOUT
    assert dt < 4.0, f"the sweep took {dt:.2f} s: later launches did not return at entry"
    monkeypatch.delenv("LBM_TEST_STALL_TMA")
    monkeypatch.delenv("LBM_WAIT_US")
    s2 = lbm.Solver(9, 256, 128, precision=4, n_steps=40, link=s.link, mask=s.mask, layout="dense")
    lbm.lbm_plan_set_kernels(s2.plan, step_family=lbm.LBM_FAMILY_TMA, adjoint_family=lbm.LBM_FAMILY_TMA)
    f = s2.forward(dev([1.001]), dev([0.8]), 1.0)
    _, u = s2.macroscopic(f)
    m = s.mask_field.cpu().numpy()
    _, uw = O.macroscopic(9, m, O.forward(9, m, 1.001, 1.0, 0.8, 40))
    assert np.linalg.norm(u.cpu().numpy() - uw) / np.linalg.norm(uw) < 1e-4
    assert s2.status() == lbm.LBM_OK
