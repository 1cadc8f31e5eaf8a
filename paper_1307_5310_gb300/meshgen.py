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
    affine=None,
) -> dict:
    """Uniform nx*ny*nz hexahedral grid of the box [lo, hi].

    ``perturb`` > 0 moves every vertex by ``perturb * h * s(x) * (1, 1, 1)``
    with s = sin(2 pi x) sin(2 pi y) sin(2 pi z) evaluated on the unit box
    coordinates of the vertex and h the smallest cell size; the elements are
    then trilinear (curved).  Vertices on the boundary of the unit box do not
    move because s vanishes there.

    ``order`` = "lex" numbers cells with x fastest; "morton" numbers them along
    the Z-order curve (face neighbours then sit close in memory).

    ``affine`` (a 3x3 matrix A with det A > 0) maps every vertex x to
    lo + A (x - lo) after the grid is built: all elements are then the same
    kind of parallelepiped (geometry "affine": constant Jacobian, not
    axis-aligned).
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
    if affine is not None:
        A = np.asarray(affine, dtype=np.float64).reshape(3, 3)
        if not np.linalg.det(A) > 0:
            raise ValueError("affine map must have a positive determinant")
        if perturb:
            raise ValueError("affine and perturb exclude each other")
        vert = lo + (vert - lo) @ A.T
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
        "geometry": "trilinear" if perturb else ("affine" if affine is not None else "brick"),
        "cell": np.stack([ii, jj, kk], axis=1),
        "dims": (nx, ny, nz),
    }
    return mesh


def trial_size(p, q, nk=1) -> np.ndarray:
    """Trial coefficients per element: 2 fields x 3 components x (N_K q + 1) temporal
    coefficients (the slab start and q modes per sub-interval) x (p+1)^3."""
    p = np.asarray(p, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    return 6 * (np.asarray(nk, dtype=np.int64) * q + 1) * (p + 1) ** 3


def test_size(p, q, nk=1) -> np.ndarray:
    """Test coefficients (= residual entries = unknowns) per element: 6 N_K q (p+1)^3."""
    p = np.asarray(p, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    return 6 * np.asarray(nk, dtype=np.int64) * q * (p + 1) ** 3


def dof_offsets(mesh: dict, kind: str = "trial") -> np.ndarray:
    """Prefix offsets [n_elem + 1] of the per-element coefficient blocks."""
    nk = mesh.get("nk", 1)
    sz = trial_size(mesh["p"], mesh["q"], nk) if kind == "trial" else test_size(mesh["p"], mesh["q"], nk)
    off = np.zeros(sz.size + 1, dtype=np.int64)
    np.cumsum(sz, out=off[1:])
    return off


def random_coeffs(mesh: dict, seed: int, kind: str = "trial", lo=-1.0, hi=1.0) -> np.ndarray:
    """Coefficient vector with entries iid U[lo, hi) from PCG64(seed)."""
    n = int(dof_offsets(mesh, kind)[-1])
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, size=n)


def random_nk(mesh: dict, seed: int, choices=(1, 2, 4)) -> None:
    """Per-element number of temporal sub-intervals N_K, uniform over ``choices`` (PCG64)."""
    ne = mesh["hex"].shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh["nk"] = np.asarray(choices, dtype=np.uint8)[rng.integers(0, len(choices), size=ne)]


def random_materials(mesh: dict, seed_eps: int, seed_mu: int, lo=1.0, hi=4.0) -> None:
    """Element-wise constant eps and mu, iid U[lo, hi) from PCG64 seeds."""
    ne = mesh["hex"].shape[0]
    mesh["eps"] = np.random.Generator(np.random.PCG64(seed_eps)).uniform(lo, hi, size=ne)
    mesh["mu"] = np.random.Generator(np.random.PCG64(seed_mu)).uniform(lo, hi, size=ne)


def corner_octree_mesh(n0: int, radii, p=1, q=1, order: str = "morton") -> dict:
    """Unit cube, base grid n0^3, refined towards the corner (0,0,0), 2:1 balanced.

    A cell of level L (edge 1/(n0 2^L)) is split while L < len(radii) and the
    distance of its corner nearest the origin is below radii[L]; afterwards
    cells are split until face neighbours differ by at most one level.
    Conforming faces get nbr >= 0; a face shared by one coarse and four fine
    cells gets nbr = -2 on both sides and one row per fine cell in ``hang``:
    (coarse element, coarse face, fine element, fine face, u, v), where u and
    v (0 or 1) locate the fine face's quarter along the lower and the higher
    of the two tangential axes.  Elements are numbered along the Z-order curve
    of their corners at the finest level (``order="morton"``).
    """
    L_max_req = len(radii)
    leaves = {(0, i, j, k) for i in range(n0) for j in range(n0) for k in range(n0)}

    def refine(cell):
        L, i, j, k = cell
        leaves.discard(cell)
        for c in range(8):
            leaves.add((L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)))

    for L in range(L_max_req):
        h = 1.0 / (n0 * 2 ** L)
        for cell in [c for c in leaves if c[0] == L]:
            _, i, j, k = cell
            if np.sqrt((i * h) ** 2 + (j * h) ** 2 + (k * h) ** 2) < radii[L]:
                refine(cell)

    def covering(L, c):
        """The leaf that contains level-L cell position c (at level <= L), or None."""
        for Lp in range(L, -1, -1):
            s = L - Lp
            key = (Lp, c[0] >> s, c[1] >> s, c[2] >> s)
            if key in leaves:
                return key
        return None

    changed = True
    while changed:
        changed = False
        for cell in sorted(leaves, key=lambda c: -c[0]):
            if cell not in leaves:
                continue
            L, i, j, k = cell
            nL = n0 * 2 ** L
            for d in range(3):
                for s in (-1, 1):
                    c = [i, j, k]
                    c[d] += s
                    if c[d] < 0 or c[d] >= nL:
                        continue
                    cov = covering(L, c)
                    if cov is not None and cov[0] < L - 1:
                        refine(cov)
                        changed = True

    Lmax = max(c[0] for c in leaves)
    scale = 2 ** Lmax
    cells = sorted(leaves)
    ii = np.array([c[1] << (Lmax - c[0]) for c in cells])
    jj = np.array([c[2] << (Lmax - c[0]) for c in cells])
    kk = np.array([c[3] << (Lmax - c[0]) for c in cells])
    perm = morton_order(ii, jj, kk) if order == "morton" else np.arange(len(cells))
    cells = [cells[t] for t in perm]
    index = {c: e for e, c in enumerate(cells)}
    ne = len(cells)
    nfine = n0 * scale
    vid = {}
    vert = []
    hexes = np.empty((ne, 8), dtype=np.int64)
    for e, (L, i, j, k) in enumerate(cells):
        f = 2 ** (Lmax - L)
        for v in range(8):
            key = ((i + (v & 1)) * f, (j + ((v >> 1) & 1)) * f, (k + ((v >> 2) & 1)) * f)
            if key not in vid:
                vid[key] = len(vert)
                vert.append(key)
            hexes[e, v] = vid[key]
    vert = np.array(vert, dtype=np.float64) / nfine
    nbr = np.full((ne, 6), -1, dtype=np.int64)
    hang = []
    for e, (L, i, j, k) in enumerate(cells):
        nL = n0 * 2 ** L
        for d in range(3):
            for s in (0, 1):
                c = [i, j, k]
                c[d] += 1 if s else -1
                if c[d] < 0 or c[d] >= nL:
                    continue
                key = (L,) + tuple(c)
                if key in index:
                    nbr[e, 2 * d + s] = index[key]
                    continue
                par = (L - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1)
                if L > 0 and par in index:
                    # this (fine) face is a quarter of the coarse neighbour's face
                    nbr[e, 2 * d + s] = -2
                    t1, t2 = [a for a in range(3) if a != d]
                    hang.append((index[par], 2 * d + (1 - s), e, 2 * d + s, c[t1] & 1, c[t2] & 1))
                else:
                    nbr[e, 2 * d + s] = -2  # coarse side: four finer neighbours
    hang = np.array(hang, dtype=np.int64).reshape(-1, 6)
    return {
        "vert": vert, "hex": hexes, "nbr": nbr, "hang": hang,
        "p": np.full(ne, p, dtype=np.uint8), "q": np.full(ne, q, dtype=np.uint8),
        "eps": np.ones(ne), "mu": np.ones(ne), "geometry": "brick",
        "level": np.array([c[0] for c in cells], dtype=np.int64),
    }


def random_hp(mesh: dict, seed: int, p_range=(1, 7), q_range=(1, 4), eps_values=(1.0, 2.25, 4.0)) -> None:
    """Per-element p ~ U{p_range}, q ~ U{q_range}, eps ~ U{eps_values}, mu = 1 (PCG64 seed)."""
    ne = mesh["hex"].shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh["p"] = rng.integers(p_range[0], p_range[1] + 1, ne).astype(np.uint8)
    mesh["q"] = rng.integers(q_range[0], q_range[1] + 1, ne).astype(np.uint8)
    mesh["eps"] = np.asarray(eps_values, dtype=np.float64)[rng.integers(0, len(eps_values), ne)]
    mesh["mu"] = np.ones(ne)
