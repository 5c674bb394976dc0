"""FP64 oracle of the cubic-spline inlet profile (test infrastructure only).

Section 3.1.2 imposes the target inlet pressure of the multi-parameter
inversion as a cubic spline through a few inlet densities.  Stated here from
the definition of the natural cubic spline:

  knots   t_k = k (n - 1) / (K - 1), k = 0..K-1 (K >= 2), over the rows 0..n-1
  spline  S(t) = M_k (t_{k+1} - t)^3 / (6 h) + M_{k+1} (t - t_k)^3 / (6 h)
                 + (c_k / h - M_k h / 6) (t_{k+1} - t) + (c_{k+1} / h - M_{k+1} h / 6) (t - t_k)
          on [t_k, t_{k+1}], h = t_{k+1} - t_k, with the second derivatives M from
          h M_{k-1} + 4 h M_k + h M_{k+1} = 6 (c_{k+1} - 2 c_k + c_{k-1}) / h   (k = 1..K-2)
          and M_0 = M_{K-1} = 0 (natural ends); K = 1 is the constant c_0
  profile rho_in(y, z) = rho_out + sum_{b, a} Bz[z, b] By[y, a] c[b, a]
          (a tensor product over rows y and layers z; nz = 1 uses Kz = 1)

The map from the knot values to the profile is linear, profile - rho_out =
B c, so the gradient with respect to c is B^T dL/drho_in.  Only tests/ may
import this module; the GPU path shares no code with it.
"""
from __future__ import annotations

import numpy as np


def knots(K: int, n: int) -> np.ndarray:
    return np.array([k * (n - 1) / (K - 1) for k in range(K)]) if K > 1 else np.zeros(1)


def second_derivatives(t: np.ndarray, c: np.ndarray) -> np.ndarray:
    """M_k of the natural spline through (t_k, c_k): the tridiagonal system of
    the definition, solved as a dense system (K is small)."""
    K = t.size
    M = np.zeros(K)
    if K < 3:
        return M
    A = np.zeros((K - 2, K - 2))
    r = np.zeros(K - 2)
    for k in range(1, K - 1):
        h0, h1 = t[k] - t[k - 1], t[k + 1] - t[k]
        i = k - 1
        A[i, i] = 2.0 * (h0 + h1)
        if i > 0:
            A[i, i - 1] = h0
        if i < K - 3:
            A[i, i + 1] = h1
        r[i] = 6.0 * ((c[k + 1] - c[k]) / h1 - (c[k] - c[k - 1]) / h0)
    M[1:-1] = np.linalg.solve(A, r)
    return M


def evaluate(t: np.ndarray, c: np.ndarray, y: np.ndarray) -> np.ndarray:
    """S(y) for the natural spline through (t_k, c_k)."""
    c = np.asarray(c, np.float64)
    if t.size == 1:
        return np.full(np.shape(y), c[0])
    M = second_derivatives(t, c)
    out = np.empty(np.shape(y))
    for j, yy in enumerate(np.ravel(y)):
        k = min(int(np.searchsorted(t, yy, side="right")) - 1, t.size - 2)
        k = max(k, 0)
        h = t[k + 1] - t[k]
        a, b = t[k + 1] - yy, yy - t[k]
        out.flat[j] = (M[k] * a ** 3 / (6 * h) + M[k + 1] * b ** 3 / (6 * h)
                       + (c[k] / h - M[k] * h / 6) * a + (c[k + 1] / h - M[k + 1] * h / 6) * b)
    return out


def basis(K: int, n: int) -> np.ndarray:
    """B[y, k]: column k is the spline through the k-th unit vector, at rows y = 0..n-1."""
    t = knots(K, n)
    y = np.arange(n, dtype=np.float64)
    return np.stack([evaluate(t, np.eye(K)[k], y) for k in range(K)], axis=1)


def profile(c: np.ndarray, ny: int, nz: int, rho_out: float) -> np.ndarray:
    """rho_in[z, y] from knot values c[Kz, Ky]."""
    c = np.atleast_2d(np.asarray(c, np.float64))
    By, Bz = basis(c.shape[1], ny), basis(c.shape[0], nz)
    return rho_out + Bz @ c @ By.T


def grad(g: np.ndarray, Ky: int, Kz: int, ny: int, nz: int) -> np.ndarray:
    """dL/dc[Kz, Ky] from dL/drho_in[z, y]."""
    g = np.asarray(g, np.float64).reshape(nz, ny)
    return basis(Kz, nz).T @ g @ basis(Ky, ny)
