"""One-dimensional polynomial machinery of the space-time basis (Sec. 5.1).

* L_i: Legendre polynomials on [0,1], orthonormal in L2(0,1).  Built from the
  textbook three-term recurrence of the classical Legendre polynomials P_i on
  [-1,1] (evaluated at s = 2 xi - 1) and normalised by sqrt(2 i + 1), since
  int_0^1 P_i(2 xi - 1)^2 d xi = 1 / (2 i + 1).
* l_m: the temporal trial functions, l_0 = 1 - xi, l_1 = xi and
  l_m(xi) = int_0^xi L_{m-1}(s) ds for m >= 2 (Eq. def:ilegendre).  Computed
  here by Gauss quadrature of that integral, not by a closed form.
* Gauss-Legendre rules on [0,1] (numpy's leggauss, mapped).
"""
from __future__ import annotations

import numpy as np


def gauss01(n: int):
    """n-point Gauss-Legendre rule on [0,1]: nodes, weights."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def legendre(nmax: int, x) -> np.ndarray:
    """L_0..L_nmax (orthonormal on [0,1]) at points x; shape (nmax+1,) + x.shape."""
    x = np.asarray(x, dtype=np.float64)
    s = 2.0 * x - 1.0
    P = np.zeros((nmax + 1,) + x.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = s
    for k in range(1, nmax):
        # (k+1) P_{k+1} = (2k+1) s P_k - k P_{k-1}
        P[k + 1] = ((2 * k + 1) * s * P[k] - k * P[k - 1]) / (k + 1)
    norm = np.sqrt(2.0 * np.arange(nmax + 1) + 1.0)
    return P * norm.reshape((-1,) + (1,) * x.ndim)


def legendre_deriv(nmax: int, x) -> np.ndarray:
    """d/dxi of L_0..L_nmax at x.

    Uses the classical identity P'_{k+1} = P'_{k-1} + (2k+1) P_k on [-1,1] and
    d/dxi = 2 d/ds.
    """
    x = np.asarray(x, dtype=np.float64)
    s = 2.0 * x - 1.0
    P = np.zeros((nmax + 2,) + x.shape)
    P[0] = 1.0
    P[1] = s
    for k in range(1, nmax + 1):
        P[k + 1] = ((2 * k + 1) * s * P[k] - k * P[k - 1]) / (k + 1)
    dP = np.zeros((nmax + 1,) + x.shape)
    for k in range(0, nmax):
        prev = dP[k - 1] if k >= 1 else 0.0
        dP[k + 1] = prev + (2 * k + 1) * P[k]
    norm = np.sqrt(2.0 * np.arange(nmax + 1) + 1.0)
    return 2.0 * dP * norm.reshape((-1,) + (1,) * x.ndim)


def trial_time(qmax: int, x) -> np.ndarray:
    """l_0..l_qmax at points x (Eq. def:ilegendre), by Gauss quadrature of the integral."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((qmax + 1,) + x.shape)
    out[0] = 1.0 - x
    if qmax >= 1:
        out[1] = x
    if qmax >= 2:
        # int_0^x L_{m-1}(s) ds = x * sum_g w_g L_{m-1}(x t_g), exact for degree <= 2 ng - 1
        tg, wg = gauss01(qmax + 1)
        xs = x[..., None] * tg
        Lv = legendre(qmax - 1, xs)  # (qmax, ..., ng)
        for m in range(2, qmax + 1):
            out[m] = x * np.sum(Lv[m - 1] * wg, axis=-1)
    return out


def trial_time_deriv(qmax: int, x) -> np.ndarray:
    """d/dxi of l_0..l_qmax: -1, 1 and L_{m-1} (fundamental theorem of calculus)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((qmax + 1,) + x.shape)
    out[0] = -1.0
    if qmax >= 1:
        out[1] = 1.0
    if qmax >= 2:
        Lv = legendre(qmax - 1, x)
        for m in range(2, qmax + 1):
            out[m] = Lv[m - 1]
    return out
