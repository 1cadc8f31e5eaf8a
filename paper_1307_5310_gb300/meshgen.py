"""Seeded synthetic inputs: hexahedral meshes, material data and coefficient vectors.

This module builds the *inputs* of the slab residual -- vertex coordinates,
element-to-vertex lists, face neighbours, per-element degrees, element-wise
constant eps/mu and random coefficient vectors.  It holds none of the method's
arithmetic (no basis functions, no quadrature, no residual terms), so both the
CUDA path and the CPU checker can be fed from it.

Conventions (the layout the C ABI documents):
  * vertex v of a hexahedron sits at reference corner (a, b, c) with
    v = a + 2 b + 4 c, i.e. x fastest;
  * faces are numbered 2 d + s with d the axis (0 = x, 1 = y, 2 = z) and
    s = 1 for the face at reference coordinate 1 (s = 0 for coordinate 0);
  * nbr[e, f] is the element across face f, or -1 on the domain boundary.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "box_mesh",
    "morton_order",
    "random_coeffs",
    "trial_size",
    "test_size",
    "dof_offsets",
]


def _part1by2(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(i: np.ndarray, j: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Permutation that sorts cells (i, j, k) along the Z-order curve."""
    code = _part1by2(i) | (_part1by2(j) << np.uint64(1)) | (_part1by2(k) << np.uint64(2))
    return np.argsort(code, kind="stable")


def box_mesh(
    nx: int,
    ny: int | None = None,
    nz: int | None = None,
    lo=(0.0, 0.0, 0.0),
    hi=(1.0, 1.0, 1.0),
    p: int = 1,
    q: int = 1,
    order: str = "lex",
    perturb: float = 0.0,
    eps=None,
    mu=None,
) -> dict:
    """Uniform nx*ny*nz hexahedral grid of the box [lo, hi].

    ``perturb`` > 0 moves every vertex by ``perturb * h * s(x) * (1, 1, 1)``
    with s = sin(2 pi x) sin(2 pi y) sin(2 pi z) evaluated on the unit box
    coordinates of the vertex and h the smallest cell size; the elements are
    then trilinear (curved).  Vertices on the boundary of the unit box do not
    move because s vanishes there.

    ``order`` = "lex" numbers cells with x fastest; "morton" numbers them along
    the Z-order curve (face neighbours then sit close in memory).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    gx = np.linspace(lo[0], hi[0], nx + 1)
    gy = np.linspace(lo[1], hi[1], ny + 1)
    gz = np.linspace(lo[2], hi[2], nz + 1)
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    vert = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()
    if perturb:
        h = float(np.min((hi - lo) / np.array([nx, ny, nz])))
        u = (vert - lo) / (hi - lo)
        s = np.sin(2 * np.pi * u[:, 0]) * np.sin(2 * np.pi * u[:, 1]) * np.sin(2 * np.pi * u[:, 2])
        vert = vert + (perturb * h * s)[:, None] * np.ones((1, 3))

    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    hexes = np.empty((ii.size, 8), dtype=np.int64)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        hexes[:, v] = vid(ii + a, jj + b, kk + c)

    if order == "lex":
        perm = np.arange(ii.size)
    elif order == "morton":
        perm = morton_order(ii, jj, kk)
    else:
        raise ValueError(f"unknown order {order!r}")
    hexes = hexes[perm]
    ii, jj, kk = ii[perm], jj[perm], kk[perm]
    cell_to_elem = np.empty(ii.size, dtype=np.int64)
    cell_to_elem[(kk * ny + jj) * nx + ii] = np.arange(ii.size)

    nbr = np.full((ii.size, 6), -1, dtype=np.int64)
    ijk = [ii, jj, kk]
    dims = [nx, ny, nz]
    for d in range(3):
        for s in (0, 1):
            step = 1 if s else -1
            nb = [a.copy() for a in ijk]
            nb[d] = nb[d] + step
            ok = (nb[d] >= 0) & (nb[d] < dims[d])
            cell = (nb[2] * ny + nb[1]) * nx + nb[0]
            nbr[ok, 2 * d + s] = cell_to_elem[cell[ok]]

    ne = ii.size
    mesh = {
        "vert": vert,
        "hex": hexes,
        "nbr": nbr,
        "p": np.full(ne, p, dtype=np.uint8),
        "q": np.full(ne, q, dtype=np.uint8),
        "eps": np.ones(ne) if eps is None else np.broadcast_to(np.asarray(eps, dtype=np.float64), (ne,)).copy(),
        "mu": np.ones(ne) if mu is None else np.broadcast_to(np.asarray(mu, dtype=np.float64), (ne,)).copy(),
        "geometry": "trilinear" if perturb else "brick",
        "cell": np.stack([ii, jj, kk], axis=1),
        "dims": (nx, ny, nz),
    }
    return mesh


def trial_size(p, q) -> np.ndarray:
    """Trial coefficients per element: 2 fields x 3 components x (q+1) modes x (p+1)^3."""
    p = np.asarray(p, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    return 6 * (q + 1) * (p + 1) ** 3


def test_size(p, q) -> np.ndarray:
    """Test coefficients (= residual entries = unknowns) per element: 6 q (p+1)^3."""
    p = np.asarray(p, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    return 6 * q * (p + 1) ** 3


def dof_offsets(mesh: dict, kind: str = "trial") -> np.ndarray:
    """Prefix offsets [n_elem + 1] of the per-element coefficient blocks."""
    sz = trial_size(mesh["p"], mesh["q"]) if kind == "trial" else test_size(mesh["p"], mesh["q"])
    off = np.zeros(sz.size + 1, dtype=np.int64)
    np.cumsum(sz, out=off[1:])
    return off


def random_coeffs(mesh: dict, seed: int, kind: str = "trial", lo=-1.0, hi=1.0) -> np.ndarray:
    """Coefficient vector with entries iid U[lo, hi) from PCG64(seed)."""
    n = int(dof_offsets(mesh, kind)[-1])
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, size=n)


def random_materials(mesh: dict, seed_eps: int, seed_mu: int, lo=1.0, hi=4.0) -> None:
    """Element-wise constant eps and mu, iid U[lo, hi) from PCG64 seeds."""
    ne = mesh["hex"].shape[0]
    mesh["eps"] = np.random.Generator(np.random.PCG64(seed_eps)).uniform(lo, hi, size=ne)
    mesh["mu"] = np.random.Generator(np.random.PCG64(seed_mu)).uniform(lo, hi, size=ne)
