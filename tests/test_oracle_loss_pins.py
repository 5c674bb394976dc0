"""Pins of the oracle's loss VALUE (section 3.1.2 / Eq. 7, Eq. 15, and the
compute_loss step of the section 2.2 listing), independent of the oracle's
own moment and loss code.

The loss of a final state f is a sum over the nodes of the region of
interest that are fluid of a per-node mismatch between the velocity of f and
the target velocity:

  vector form   |u - u_t|^2            (the default reading of Eq. 7)
  norm form     (|u| - |u_t|)^2        (the paper's compute_loss)

with weight 1 (Eq. 7, a plain sum) or 1 / N, N = the number of nodes in
ROI and fluid (Eq. 15, a mean).  Two independent routes fix it:

* closed forms: f is built from a chosen density and velocity per node
  (first-order equilibrium w_i rho (1 + 3 c_i . u), whose moments are exactly
  rho and rho u), and the target is built from u with a known offset (vector
  form: u_t = u + d, so the loss is sum |d|^2) or a known scale (norm form:
  u_t = s u, so the loss is sum (1 - s)^2 |u|^2); solids and non-ROI nodes
  carry large garbage so any leak shows;
* a numpy restatement on a state from a real forward run, with the moments
  formed here from the lattice velocities (not from the oracle's moments).

A dropped velocity component, a wrong sign, counting all fluid nodes
instead of ROI and fluid, a missing 1/N, or a wrong norm term each fails.
"""
import numpy as np
import pytest

from oracle import oracle as O

# Direction tables in the library's documented order.  D2Q9: rest, E, N, W,
# S, NE, NW, SW, SE (the paper's Fig. 1 / Eq. 18 order); D3Q19: rest, +x, -x,
# +y, -y, +z, -z, then the twelve edge directions.
C9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], np.float64)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
C19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], np.float64)
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _tables(q):
    return (C9, W9) if q == 9 else (C19, W19)


def test_direction_tables_match_the_oracle():
    """The tables above are the oracle's (order included), so f built here
    means to the oracle what it means to this test."""
    for q in (9, 19):
        c, w = _tables(q)
        oc, ow, _ = O.lattice(q)
        assert np.array_equal(oc[:, :c.shape[1]].astype(np.float64), c)
        assert np.array_equal(ow, w)


def _shape(q):
    return (7, 11) if q == 9 else (5, 6, 7)


def _case(q, seed):
    """A mask with solids, a ROI that covers part of the solids and part of
    the fluid, and f with prescribed rho, u at every fluid node."""
    rng = np.random.default_rng(seed)
    c, w = _tables(q)
    d = c.shape[1]
    shp = _shape(q)
    mask = (rng.random(shp) < 0.3).astype(np.uint8)
    roi = (rng.random(shp) < 0.6).astype(np.uint8)
    # make sure every category exists: ROI & fluid, ROI & solid, non-ROI fluid
    flat_m, flat_r = mask.reshape(-1), roi.reshape(-1)
    flat_m[:3], flat_r[:3] = 0, 1
    flat_m[3:5], flat_r[3:5] = 1, 1
    flat_m[5:7], flat_r[5:7] = 0, 0
    rho = 1.0 + 0.01 * rng.standard_normal(shp)
    u = 0.02 * rng.standard_normal((d,) + shp)
    cu = np.einsum("ia,a...->i...", c, u)
    f = w.reshape((-1,) + (1,) * len(shp)) * rho * (1.0 + 3.0 * cu)
    f[:, mask == 1] = 1e6 * rng.standard_normal((c.shape[0], int(mask.sum())))  # garbage: solids carry nothing
    sel = (mask == 0) & (roi == 1)
    return mask, roi, f, u, sel, rng


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("norm", [O.NORM_SUM, O.NORM_MEAN_FLUID])
def test_vector_loss_closed_form(q, norm):
    """u_t = u + d on ROI fluid nodes: L = w sum |d|^2, w = 1 or 1/N."""
    mask, roi, f, u, sel, rng = _case(q, 11 + q + norm)
    d = 1e-3 * rng.standard_normal(u.shape)
    ut = u + d
    ut[:, ~sel] = 1e3 * rng.standard_normal((u.shape[0], int((~sel).sum())))  # ignored nodes: garbage
    want = float((d[:, sel] ** 2).sum())
    if norm == O.NORM_MEAN_FLUID:
        want /= int(sel.sum())
    L, _ = O.loss(q, mask, f, ut, roi, O.LOSS_VEC, norm)
    assert abs(L - want) <= 1e-11 * want


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("norm", [O.NORM_SUM, O.NORM_MEAN_FLUID])
def test_norm_loss_closed_form(q, norm):
    """u_t = s u (s > 0 per node) on ROI fluid nodes: L = w sum (1 - s)^2 |u|^2."""
    mask, roi, f, u, sel, rng = _case(q, 23 + q + norm)
    s = 1.0 + 0.3 * rng.standard_normal(u.shape[1:])
    s = np.abs(s) + 0.05
    ut = u * s
    ut[:, ~sel] = 1e3 * rng.standard_normal((u.shape[0], int((~sel).sum())))
    want = float((((1.0 - s) ** 2) * (u ** 2).sum(axis=0))[sel].sum())
    if norm == O.NORM_MEAN_FLUID:
        want /= int(sel.sum())
    L, _ = O.loss(q, mask, f, ut, roi, O.LOSS_NORM, norm)
    assert abs(L - want) <= 1e-11 * want


@pytest.mark.parametrize("q", [9, 19])
def test_roi_none_means_every_fluid_node(q):
    """No ROI: the sum (and the count N of Eq. 15) runs over all fluid nodes."""
    mask, _, f, u, _, rng = _case(q, 37 + q)
    fl = mask == 0
    d = 1e-3 * rng.standard_normal(u.shape)
    ut = u + d
    s_all = float((d[:, fl] ** 2).sum())
    L_sum, _ = O.loss(q, mask, f, ut, None, O.LOSS_VEC, O.NORM_SUM)
    L_mean, _ = O.loss(q, mask, f, ut, None, O.LOSS_VEC, O.NORM_MEAN_FLUID)
    assert abs(L_sum - s_all) <= 1e-11 * s_all
    assert abs(L_mean - s_all / int(fl.sum())) <= 1e-11 * s_all / int(fl.sum())


@pytest.mark.parametrize("q", [9, 19])
@pytest.mark.parametrize("kind", [O.LOSS_VEC, O.LOSS_NORM])
@pytest.mark.parametrize("norm", [O.NORM_SUM, O.NORM_MEAN_FLUID])
def test_loss_restated_from_populations(q, kind, norm):
    """A state from a real forward run (walls, grains, Eq. 6 planes), the
    moments formed here from the lattice velocities, the loss summed here
    over ROI fluid nodes; the oracle must agree to rounding."""
    c, _ = _tables(q)
    if q == 9:
        m, _ = O.geometry(9, 24, 12, kind=O.GEOM_DISKS, seed=5, r_min=2, r_max=3, porosity=0.8, buffer=3)
        rin = 1.0 + 1e-3 * (1.0 + np.sin(np.linspace(0, 3, 12)))
    else:
        m, _ = O.geometry(19, 12, 8, 8, kind=O.GEOM_SPHERES, seed=7, r_min=2, r_max=2, porosity=0.85, buffer=2)
        rin = 1.002
    f = O.forward(q, m, rin, 1.0, 0.8, 40)
    rho = f.sum(axis=0)
    u = np.einsum("ia,i...->a...", c, f) / rho
    rng = np.random.default_rng(3)
    ut = u * (1.0 + 0.2 * rng.standard_normal(u.shape)) + 1e-4 * rng.standard_normal(u.shape)
    roi = (rng.random(m.shape) < 0.5).astype(np.uint8)
    sel = (m == 0) & (roi == 1)
    if kind == O.LOSS_VEC:
        per = ((u - ut) ** 2).sum(axis=0)
    else:
        per = (np.sqrt((u ** 2).sum(axis=0)) - np.sqrt((ut ** 2).sum(axis=0))) ** 2
    want = float(per[sel].sum())
    if norm == O.NORM_MEAN_FLUID:
        want /= int(sel.sum())
    L, _ = O.loss(q, m, f, ut, roi, kind, norm)
    assert abs(L - want) <= 1e-12 * want
