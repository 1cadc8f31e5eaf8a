"""Element maps F_K : [0,1]^3 -> K (Sec. 2.3).

Every hexahedron is mapped trilinearly from its 8 vertices; vertex v sits at
reference corner (a, b, c), v = a + 2 b + 4 c.  An axis-aligned brick or a
parallelepiped is the affine special case of the same formula.
"""
from __future__ import annotations

import numpy as np


def _corner_bits():
    v = np.arange(8)
    return np.stack([v & 1, (v >> 1) & 1, (v >> 2) & 1], axis=1).astype(np.float64)


_BITS = _corner_bits()


def shape(xh: np.ndarray) -> np.ndarray:
    """Trilinear shape functions N_v at reference points xh [..., 3] -> [..., 8]."""
    xh = np.asarray(xh, dtype=np.float64)
    f = np.where(_BITS[None, :, :] > 0.5, xh[..., None, :], 1.0 - xh[..., None, :])
    return np.prod(f, axis=-1)


def shape_grad(xh: np.ndarray) -> np.ndarray:
    """dN_v/dxh_a at reference points -> [..., 8, 3]."""
    xh = np.asarray(xh, dtype=np.float64)
    f = np.where(_BITS[None, :, :] > 0.5, xh[..., None, :], 1.0 - xh[..., None, :])
    df = np.where(_BITS[None, :, :] > 0.5, 1.0, -1.0) * np.ones_like(f)
    out = np.empty(f.shape)
    for a in range(3):
        others = [b for b in range(3) if b != a]
        out[..., a] = df[..., a] * f[..., others[0]] * f[..., others[1]]
    return out


def map_points(X8: np.ndarray, xh: np.ndarray) -> np.ndarray:
    """x = F(xh) for one element with vertices X8 [8, 3]."""
    return shape(xh) @ X8


def jacobian(X8: np.ndarray, xh: np.ndarray) -> np.ndarray:
    """DF[..., i, j] = d x_i / d xh_j."""
    dN = shape_grad(xh)  # [..., 8, 3]
    return np.einsum("vi,...vj->...ij", X8, dN)


def inverse_map(X8: np.ndarray, x: np.ndarray, guess: np.ndarray | None = None, tol=1e-15, maxit=50):
    """Reference coordinates xh with F(xh) = x, by Newton's method."""
    x = np.asarray(x, dtype=np.float64)
    xh = np.full(x.shape, 0.5) if guess is None else np.array(guess, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(X8))))
    for _ in range(maxit):
        r = map_points(X8, xh) - x
        if np.max(np.abs(r)) <= tol * scale:
            break
        DF = jacobian(X8, xh)
        xh = xh - np.linalg.solve(DF, r[..., None])[..., 0]
    return xh
