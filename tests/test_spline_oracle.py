"""Pins of the cubic-spline profile oracle against a library routine and
closed forms (CPU)."""
import numpy as np
import pytest

from oracle import spline_oracle as S

interp = pytest.importorskip("scipy.interpolate")


@pytest.mark.parametrize("K,n", [(3, 17), (5, 64), (8, 256), (16, 128), (4, 10)])
def test_basis_matches_scipy_natural_cubic_spline(K, n):
    r = np.random.Generator(np.random.PCG64(K * 1000 + n))
    c = r.normal(size=K)
    t = S.knots(K, n)
    want = interp.CubicSpline(t, c, bc_type="natural")(np.arange(n, dtype=np.float64))
    np.testing.assert_allclose(S.basis(K, n) @ c, want, rtol=0, atol=1e-12)


def test_closed_forms():
    # two knots: linear interpolation between the end rows
    n = 11
    np.testing.assert_allclose(S.basis(2, n) @ np.array([1.0, 3.0]), 1.0 + 2.0 * np.arange(n) / (n - 1), atol=1e-14)
    # a linear function of the knot positions is reproduced exactly (natural ends allow it)
    for K in (3, 6, 9):
        t = S.knots(K, 40)
        np.testing.assert_allclose(S.basis(K, 40) @ (0.5 - 0.25 * t), 0.5 - 0.25 * np.arange(40), atol=1e-12)
    # partition of unity, interpolation at the knots that fall on rows
    B = S.basis(5, 33)  # knots at rows 0, 8, 16, 24, 32
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(B[[0, 8, 16, 24, 32]], np.eye(5), atol=1e-13)
    # one knot: a constant
    assert np.array_equal(S.basis(1, 7), np.ones((7, 1)))


def test_tensor_profile_and_its_gradient():
    r = np.random.Generator(np.random.PCG64(3))
    ny, nz, Ky, Kz = 20, 12, 5, 3
    c = r.normal(size=(Kz, Ky))
    p = S.profile(c, ny, nz, 1.0)
    # separable: a rank-1 knot array gives a rank-1 profile through scipy in each direction
    cy, cz = r.normal(size=Ky), r.normal(size=Kz)
    sy = interp.CubicSpline(S.knots(Ky, ny), cy, bc_type="natural")(np.arange(ny, dtype=float))
    sz = interp.CubicSpline(S.knots(Kz, nz), cz, bc_type="natural")(np.arange(nz, dtype=float))
    np.testing.assert_allclose(S.profile(np.outer(cz, cy), ny, nz, 0.0), np.outer(sz, sy), atol=1e-12)
    # the gradient is the transpose: <g, B dc> = <B^T g, dc>, and finite differences agree
    g = r.normal(size=(nz, ny))
    dc = r.normal(size=(Kz, Ky))
    lhs = np.sum(g * (S.profile(c + dc, ny, nz, 1.0) - p))
    assert np.isclose(lhs, np.sum(S.grad(g, Ky, Kz, ny, nz) * dc), rtol=1e-12)
