"""lbm_loss_grad_noalloc: the loss and seed for callers that cannot allocate
device memory (a plugin under a host application's allocator, a real-time
loop, a host that only hands over its existing buffers).  Its scratch is the
library's fixed device array instead of a caller workspace; its output must
match lbm_loss_grad's on the same inputs, call after call.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2310_00810_gb300 import lbm
from paper_2310_00810_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_00810_gb300 import build

    build.build()
    lbm.load()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("q,precision,norm,kind,with_roi", [
    (9, 4, lbm.LBM_NORM_SUM, lbm.LBM_LOSS_VEC, True),
    (9, 8, lbm.LBM_NORM_MEAN_FLUID, lbm.LBM_LOSS_NORM, True),
    (19, 4, lbm.LBM_NORM_MEAN_FLUID, lbm.LBM_LOSS_VEC, True),
    (9, 4, lbm.LBM_NORM_MEAN_FLUID, lbm.LBM_LOSS_VEC, False),  # no ROI: the mean over every fluid node
    (19, 8, lbm.LBM_NORM_SUM, lbm.LBM_LOSS_NORM, False),
])
def test_noalloc_matches_workspace_loss_twice(q, precision, norm, kind, with_roi):
    if q == 9:
        shape, g = (96, 260), dict(kind=lbm.LBM_GEOM_DISKS, seed=5, r_min=3, r_max=8, target_porosity=0.65)
    else:
        shape, g = (12, 20, 140), dict(kind=lbm.LBM_GEOM_SPHERES, seed=5, r_min=3, r_max=3, target_porosity=0.7)
    nx, ny, nz = shape[-1], shape[-2], (shape[0] if q == 19 else 1)
    s = lbm.Solver(q, nx, ny, nz, precision=precision, n_steps=1, loss_kind=kind, loss_norm=norm, geometry=g)
    d = 2 if q == 9 else 3
    roi = _dev(W.roi_band(shape, axis=len(shape) - 1, start=nx // 4), torch.uint8) if with_roi else None
    for call in range(2):
        f = _dev(W.perturbation((q,) + shape, seed=100 + call, scale=2e-3), s.plan.dtype)
        ut = _dev(W.perturbation((d,) + shape, seed=200 + call, scale=3e-3))
        want_loss, want_lam = s.loss_grad(f, ut, roi)
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        lam = torch.full_like(want_lam, float("nan"))
        s.run(lambda: lbm.lbm_loss_grad_noalloc(s.plan, f, ut, roi, loss, lam))
        torch.cuda.synchronize()
        assert abs(loss.item() - want_loss.item()) <= 1e-12 * abs(want_loss.item())
        assert torch.equal(lam, want_lam)


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the scratch address), further calls
    leave the device's free memory and torch's allocator untouched."""
    shape = (64, 200)
    s = lbm.Solver(9, 200, 64, precision=4, n_steps=1,
                   geometry=dict(kind=lbm.LBM_GEOM_DISKS, seed=3, r_min=3, r_max=6, target_porosity=0.7))
    f = _dev(W.perturbation((9,) + shape, seed=7, scale=2e-3), torch.float32)
    ut = _dev(W.perturbation((2,) + shape, seed=8, scale=3e-3))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(f)
    s.run(lambda: lbm.lbm_loss_grad_noalloc(s.plan, f, ut, None, loss, lam))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        s.run(lambda: lbm.lbm_loss_grad_noalloc(s.plan, f, ut, None, loss, lam))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.isfinite(loss.item()) and loss.item() > 0


def test_noalloc_rejects_lattices_beyond_its_scratch():
    ny = lbm.LBM_NOALLOC_MAX_BLOCKS // 2 + 1  # two blocks per row at 128 < nx <= 256
    plan = lbm.Plan(9, 256, ny, 1, precision=4, n_steps=1)
    link = torch.zeros(plan.N, dtype=torch.int32, device="cuda")
    lbm.lbm_bind_geometry(plan, link)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_loss_grad_noalloc(plan, torch.zeros(9 * plan.N, device="cuda"),
                                  torch.zeros(2 * plan.N, dtype=torch.float64, device="cuda"), None,
                                  torch.zeros(1, dtype=torch.float64, device="cuda"),
                                  torch.zeros(9 * plan.N, device="cuda"))
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    # the library itself refuses too (before any launch)
    vp = lambda t: __import__("ctypes").c_void_p(t.data_ptr())
    st = lbm.load().lbm_loss_grad_noalloc(plan.handle, vp(link), vp(link), None, vp(link), vp(link), None)
    assert st == lbm.LBM_ERR_INVALID_ARG
