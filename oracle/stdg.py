"""Space-time DG slab residual by full tensor Gauss quadrature in physical space.

Test infrastructure (see the package docstring).  Everything here follows the
paper's definitions literally:

* trial functions (Sec. 5.1): U = DF^{-T} [ l_m(xi) L_j(x^) L_k(y^) L_l(z^) e_c ],
  test functions: V = DF^{-T} [ L_i(xi) L_j L_k L_l e_c ], i < q
  (covariant transformation, Sec. 2.3), xi = (t - t0) / dt;
* the bilinear form (Eq. bilinearform:C)
      C_h(U, V) = (eps d_t E, v) + (mu d_t H, w) - (H, curl v) + (curl E, w)
                  + <{H}, [v]_T>_{F0 u Fb} - <[E]_T, {w}>_{F0 u Fb},
  with {v} = (v1 + v2)/2, [v]_T = n1 x v1 + n2 x v2 on interior faces and
  {v} = v, [v]_T = n x v on boundary faces (Sec. 2.4);
* the stabilisation S_h of Eq. bilinearform:S on interior faces whose two
  elements have different temporal degrees, with the projector onto the
  common temporal test space computed as an L2 projection by quadrature;
* optionally the dissipative (upwind-type) term of Sec. 4.2,
      D_h(U, V) = <alpha_E [E]_T, [Pi~ v]_T>_{F0} + <alpha_E [E - g]_T, [v]_T>_{Fb}
                  + <alpha_H [H]_T, [Pi~ w]_T>_{F0},
  alpha_E = c / {sqrt(mu/eps)}, alpha_H = c / {sqrt(eps/mu)}, c >= 0
  (``c_diss``; on a boundary face the average is the element's own value);
* the load L(V) = (J, v) - <n x g, w>_{Fb} and the residual
  R_h(V) = B_h(U, V) - L(V) (Eq. residual).

Inner products are space-time integrals over I_n x K; they are evaluated with
p+2 Gauss points per spatial direction and q+2 in time (for a face shared by
elements of different degree: the larger of the two).  Physical fields are
obtained from reference fields through DF^{-T} (values) and (1/J) DF (curl,
the Piola identity, checked against finite differences in the tests).

Local refinement in time (Sec. 2.2, Sec. 4.1): element K may split the slab
into N_K equal sub-intervals I_k^K (``mesh["nk"]``, default 1).  The trial
space is continuous piecewise P_q in time, the test space discontinuous
piecewise P_{q-1}; on a face whose two elements have different temporal test
spaces, S_h projects onto their intersection (piecewise P_{min(q)-1} on the
coarser partition), computed by quadrature on the finer partition.

Coefficient layout of one element (trial): [field E,H][component x,y,z]
[temporal index M][spatial index s], s = (l (p+1) + k)(p+1) + j with j the x^
degree, M = 0 the slab-start coefficient u_0 and M = 1 + k q + (m - 1) the
mode m >= 1 of sub-interval k (mode 0 of sub-interval k > 0 is mode 1 of
sub-interval k - 1: continuity).  With N_K = 1 this is [mode m = 0..q].
Test/residual layout: [field][component][k q + i][s], i = 0..q-1.

Face neighbours are found from the element-to-vertex lists (shared vertex
quadruples); the neighbour's reference coordinates of every face quadrature
point are obtained by inverting its map with Newton's method.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, geometry

_LEVI = np.zeros((3, 3, 3))
_LEVI[0, 1, 2] = _LEVI[1, 2, 0] = _LEVI[2, 0, 1] = 1.0
_LEVI[0, 2, 1] = _LEVI[2, 1, 0] = _LEVI[1, 0, 2] = -1.0

# reference corners on face (d, s): vertices with bit d equal to s
_FACE_VERTS = [[v for v in range(8) if ((v >> d) & 1) == s] for d in range(3) for s in (0, 1)]


def _cross(a, b):
    a, b = np.broadcast_arrays(a, b)
    return np.cross(a, b, axis=-1)


# ----------------------------------------------------------------------------
# spatial basis tables
# ----------------------------------------------------------------------------

def spatial_basis(p: int, xh: np.ndarray):
    """phi[P, s] and grad phi[P, s, 3] of L_j(x^)L_k(y^)L_l(z^) at points xh [P, 3]."""
    n = p + 1
    Lx = basis.legendre(p, xh[:, 0])  # [n, P]
    Ly = basis.legendre(p, xh[:, 1])
    Lz = basis.legendre(p, xh[:, 2])
    dLx = basis.legendre_deriv(p, xh[:, 0])
    dLy = basis.legendre_deriv(p, xh[:, 1])
    dLz = basis.legendre_deriv(p, xh[:, 2])
    P = xh.shape[0]
    phi = np.empty((P, n, n, n))  # [P, l, k, j]
    g = np.empty((P, n, n, n, 3))
    for l in range(n):
        for k in range(n):
            for j in range(n):
                phi[:, l, k, j] = Lx[j] * Ly[k] * Lz[l]
                g[:, l, k, j, 0] = dLx[j] * Ly[k] * Lz[l]
                g[:, l, k, j, 1] = Lx[j] * dLy[k] * Lz[l]
                g[:, l, k, j, 2] = Lx[j] * Ly[k] * dLz[l]
    return phi.reshape(P, n ** 3), g.reshape(P, n ** 3, 3)


def _grid3(nq: int):
    x, w = basis.gauss01(nq)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def _face_grid(d: int, s: int, nq: int):
    """Gauss points on reference face x^_d = s: points [A, 3], weights [A]."""
    x, w = basis.gauss01(nq)
    a1, a2 = [a for a in range(3) if a != d]
    U, V = np.meshgrid(x, x, indexing="ij")
    pts = np.zeros((nq * nq, 3))
    pts[:, d] = float(s)
    pts[:, a1] = U.ravel()
    pts[:, a2] = V.ravel()
    return pts, np.outer(w, w).ravel()


# ----------------------------------------------------------------------------
# mesh topology (from vertex ids only)
# ----------------------------------------------------------------------------

def face_neighbours(hexes: np.ndarray) -> np.ndarray:
    """[n_elem, 6, 2] array (neighbour element, neighbour face) or -1, by shared vertex quadruples."""
    ne = hexes.shape[0]
    table = {}
    out = np.full((ne, 6, 2), -1, dtype=np.int64)
    for e in range(ne):
        for f in range(6):
            key = tuple(sorted(int(hexes[e, v]) for v in _FACE_VERTS[f]))
            if key in table:
                e2, f2 = table.pop(key)
                out[e, f] = (e2, f2)
                out[e2, f2] = (e, f)
            else:
                table[key] = (e, f)
    return out


# ----------------------------------------------------------------------------
# field evaluation
# ----------------------------------------------------------------------------

@dataclass
class _Pts:
    """Geometry and basis at a set of reference points of one element."""
    xh: np.ndarray      # [P, 3]
    x: np.ndarray       # [P, 3] physical
    DF: np.ndarray      # [P, 3, 3]
    DFinv: np.ndarray   # [P, 3, 3]
    J: np.ndarray       # [P]
    phi: np.ndarray     # [P, N3]
    gphi: np.ndarray    # [P, N3, 3]


def _points(X8, p, xh) -> _Pts:
    DF = geometry.jacobian(X8, xh)
    J = np.linalg.det(DF)
    if np.any(J <= 0):
        raise ValueError("element map with non-positive Jacobian")
    phi, gphi = spatial_basis(p, xh)
    return _Pts(xh, geometry.map_points(X8, xh), DF, np.linalg.inv(DF), J, phi, gphi)


def _sub_of(nk: int, tau: np.ndarray):
    """Sub-interval index and local coordinate of slab times tau in [0, 1]."""
    k = np.minimum(np.floor(tau * nk).astype(np.int64), nk - 1)
    return k, tau * nk - k


def trial_time_nk(q: int, nk: int, tau: np.ndarray, deriv: bool = False) -> np.ndarray:
    """[N_K q + 1, T] factors of the trial coefficients (layout above) at slab times tau;
    with ``deriv`` the derivative d/dxi, xi = (t - t0)/dt the slab coordinate."""
    k, s = _sub_of(nk, tau)
    lt = basis.trial_time_deriv(q, s) * nk if deriv else basis.trial_time(q, s)  # [q+1, T]
    out = np.zeros((nk * q + 1, tau.size))
    cols = np.arange(tau.size)
    out[np.where(k == 0, 0, 1 + (k - 1) * q), cols] += lt[0]
    for m in range(1, q + 1):
        out[1 + k * q + m - 1, cols] += lt[m]
    return out


def test_time_nk(q: int, nk: int, tau: np.ndarray) -> np.ndarray:
    """[N_K q, T]: L_i on sub-interval k (row k q + i), zero outside it."""
    k, s = _sub_of(nk, tau)
    L = basis.legendre(q - 1, s)
    out = np.zeros((nk * q, tau.size))
    cols = np.arange(tau.size)
    for i in range(q):
        out[k * q + i, cols] = L[i]
    return out


def time_rule(q: int, nk: int):
    """Gauss rule with q+2 points on each of nk equal sub-intervals of [0, 1]."""
    x, w = basis.gauss01(q + 2)
    tau = ((np.arange(nk)[:, None] + x[None, :]) / nk).ravel()
    return tau, np.tile(w / nk, nk)


def _fields(u, pts: _Pts, q: int, tau: np.ndarray, dt: float, derivs: bool = True, nk: int = 1):
    """Physical E (or H) values, time derivative and curl at (tau x points).

    u: [B, 3, N_K q + 1, N3] trial coefficients of one field (None means zero).
    Returns val, dtval, curl, each [B, T, P, 3] (dtval, curl are None unless
    ``derivs``).
    """
    if u is None:
        return 0.0, 0.0, 0.0
    B = u.shape[0]
    P = pts.phi.shape[0]
    M = u.shape[2]
    lt = trial_time_nk(q, nk, tau)        # [M, T]
    S = (u.reshape(-1, u.shape[-1]) @ pts.phi.T).reshape(B, 3, M, P)
    ref = np.einsum("mt,bcmp->btpc", lt, S, optimize=True)      # reference field
    val = np.einsum("pci,btpc->btpi", pts.DFinv, ref, optimize=True)  # DF^{-T} ref
    if not derivs:
        return val, None, None
    dlt = trial_time_nk(q, nk, tau, deriv=True)  # [M, T]
    dref = np.einsum("mt,bcmp->btpc", dlt, S, optimize=True)
    gp = pts.gphi.transpose(1, 0, 2).reshape(pts.gphi.shape[1], -1)   # [N3, P*3]
    G = (u.reshape(-1, u.shape[-1]) @ gp).reshape(B, 3, M, P, 3)
    gref = np.einsum("mt,bcmpa->btpca", lt, G, optimize=True)   # d ref_c / d x^_a
    # reference curl: (curl)_i = eps_{i a c} d_a ref_c
    cref = np.einsum("iac,btpca->btpi", _LEVI, gref, optimize=True)
    dtval = np.einsum("pci,btpc->btpi", pts.DFinv, dref, optimize=True) / dt
    # Piola identity: curl (DF^{-T} ref) = (1/J) DF curl_ref
    curl = np.einsum("pij,btpj->btpi", pts.DF, cref, optimize=True) / pts.J[None, None, :, None]
    return val, dtval, curl


def _test_project(a: np.ndarray, pts: _Pts, Lt: np.ndarray, wgt: np.ndarray) -> np.ndarray:
    """sum over points of wgt * a . v for every test function v = DF^{-T} L_i phi_s e_d.

    a: [B, T, P, 3] physical vector field; Lt: [q, T] temporal test factors;
    wgt: [T, P] quadrature weights (including dt and the measure).
    Returns [B, 3, q, N3].
    """
    # a . DF^{-T} e_d = (DF^{-1} a)_d
    b = np.einsum("pdi,btpi->btpd", pts.DFinv, a) * wgt[None, :, :, None]
    return np.einsum("it,ps,btpd->bdis", Lt, pts.phi, b, optimize=True)


def _test_project_curl(a: np.ndarray, pts: _Pts, Lt: np.ndarray, wgt: np.ndarray) -> np.ndarray:
    """sum over points of wgt * a . curl v, curl v = (1/J) DF (grad^ phi_s x e_d) L_i."""
    # a . (1/J) DF (g x e_d) = (1/J) (DF^T a) . (g x e_d) = (1/J) ((DF^T a) x g)_d
    b = np.einsum("pij,btpi->btpj", pts.DF, a) / pts.J[None, None, :, None]
    b = b * wgt[None, :, :, None]
    # ((b) x g)_d = eps_{d a c} b_a g_c
    return np.einsum("it,dac,btpa,psc->bdis", Lt, _LEVI, b, pts.gphi, optimize=True)


# ----------------------------------------------------------------------------
# the oracle
# ----------------------------------------------------------------------------

class Oracle:
    """Residual, assembly, slab solve and energy for one mesh.

    mesh: dict with vert [nv,3], hex [ne,8], p [ne], q [ne], eps [ne], mu [ne].
    """

    def __init__(self, mesh: dict, c_diss: float = 0.0):
        self.c_diss = float(c_diss)
        self.vert = np.asarray(mesh["vert"], dtype=np.float64)
        self.hex = np.asarray(mesh["hex"], dtype=np.int64)
        self.ne = self.hex.shape[0]
        self.p = np.asarray(mesh["p"], dtype=np.int64).reshape(self.ne)
        self.q = np.asarray(mesh["q"], dtype=np.int64).reshape(self.ne)
        self.eps = np.asarray(mesh["eps"], dtype=np.float64).reshape(self.ne)
        self.mu = np.asarray(mesh["mu"], dtype=np.float64).reshape(self.ne)
        self.nk = np.asarray(mesh.get("nk", np.ones(self.ne)), dtype=np.int64).reshape(self.ne)
        if np.any(self.nk < 1):
            raise ValueError("N_K must be >= 1")
        self.nbr = face_neighbours(self.hex)
        self.pieces = self._face_pieces()
        n3 = (self.p + 1) ** 3
        self.trial_sz = 6 * (self.nk * self.q + 1) * n3
        self.test_sz = 6 * self.nk * self.q * n3
        self.trial_off = np.concatenate([[0], np.cumsum(self.trial_sz)])
        self.test_off = np.concatenate([[0], np.cumsum(self.test_sz)])
        self._vol_cache = {}

    # -- helpers -------------------------------------------------------------
    def X8(self, e: int) -> np.ndarray:
        return self.vert[self.hex[e]]

    def trial_block(self, U, e: int) -> np.ndarray:
        """[..., 2, 3, q+1, N3] view of element e's trial coefficients.

        U is a trial vector [..., N_trial] or a dict {element: block [B, 2, 3, q+1, N3]}
        holding only some elements' blocks (the others are zero).
        """
        p, M = int(self.p[e]), int(self.nk[e] * self.q[e]) + 1
        if isinstance(U, dict):
            if e in U:
                return U[e]
            B = next(iter(U.values())).shape[0]
            return np.zeros((B, 2, 3, M, (p + 1) ** 3))
        blk = U[..., self.trial_off[e]:self.trial_off[e + 1]]
        return blk.reshape(blk.shape[:-1] + (2, 3, M, (p + 1) ** 3))

    def _pts(self, e: int, p: int, xh: np.ndarray, tag) -> _Pts:
        """Geometry/basis tables at reference points xh of element e.

        Tables that only depend on the element's shape (not its position) are
        cached, keyed by the vertex coordinates relative to vertex 0.
        """
        X8 = self.X8(e)
        key = (p, tag, tuple(np.round(X8 - X8[0], 13).ravel()))
        hit = self._vol_cache.get(key)
        if hit is None:
            if len(self._vol_cache) > 20000:
                self._vol_cache.clear()
            hit = _points(X8, p, xh)
            self._vol_cache[key] = hit
        return _Pts(hit.xh, geometry.map_points(X8, xh), hit.DF, hit.DFinv, hit.J, hit.phi, hit.gphi)

    # -- face topology -----------------------------------------------------------
    def _locate(self, x, exclude):
        """Element (other than ``exclude``) whose closed reference cube contains point x, or -1."""
        if not hasattr(self, "_bbox"):
            X = self.vert[self.hex]  # [ne, 8, 3]
            lo, hi = X.min(axis=1), X.max(axis=1)
            self._bbox = (lo, hi)
            # bucket grid with cells as large as the largest element
            self._h = float(np.max(hi - lo))
            self._o = lo.min(axis=0)
            buckets = {}
            i0 = np.floor((lo - self._o) / self._h).astype(np.int64)
            i1 = np.floor((hi - self._o) / self._h).astype(np.int64)
            for e in range(self.ne):
                for i in range(i0[e, 0], i1[e, 0] + 1):
                    for j in range(i0[e, 1], i1[e, 1] + 1):
                        for k in range(i0[e, 2], i1[e, 2] + 1):
                            buckets.setdefault((i, j, k), []).append(e)
            self._buckets = {k: np.array(v) for k, v in buckets.items()}
            self._tol = 1e-9 * max(1.0, float(np.max(np.abs(self.vert))))
        lo, hi = self._bbox
        tol = self._tol
        key = tuple(np.floor((x - self._o) / self._h).astype(np.int64))
        pool = self._buckets.get(key, np.zeros(0, dtype=np.int64))
        cand = pool[np.all((x >= lo[pool] - tol) & (x <= hi[pool] + tol), axis=1)]
        for e2 in cand:
            if e2 == exclude:
                continue
            xh = geometry.inverse_map(self.X8(e2), x[None, :])[0]
            if np.all(xh > -1e-9) and np.all(xh < 1 + 1e-9):
                return int(e2)
        return -1

    def _face_pieces(self):
        """Per element face: a list of (neighbour or -1, (u0, u1, v0, v1)) pieces.

        The rectangle is a part of the element's reference face in its two
        tangential coordinates (lower axis first).  Faces matched by shared
        vertices are one piece; other faces are probed just outside their
        centre: no element there means boundary, a larger element means this
        face is a quarter of that element's face (one piece), smaller elements
        mean four quarter pieces, each with the element found outside its
        centre.
        """
        pieces = [[None] * 6 for _ in range(self.ne)]
        dN = geometry.shape_grad(np.full((1, 3), 0.5))[0]  # [8, 3]
        vol = np.abs(np.linalg.det(np.einsum("evi,vj->eij", self.vert[self.hex], dN)))
        for e in range(self.ne):
            for f in range(6):
                if self.nbr[e, f, 0] >= 0:
                    pieces[e][f] = [(int(self.nbr[e, f, 0]), (0.0, 1.0, 0.0, 1.0))]
                    continue
                d, s = divmod(f, 2)

                def probe(u, v):
                    xh = np.full((1, 3), 0.5)
                    a1, a2 = [a for a in range(3) if a != d]
                    xh[0, d] = s
                    xh[0, a1], xh[0, a2] = u, v
                    x = geometry.map_points(self.X8(e), xh)[0]
                    DF = geometry.jacobian(self.X8(e), xh)[0]
                    out = DF[:, d] * (1.0 if s == 1 else -1.0)
                    return self._locate(x + 1e-4 * out, e)

                e2 = probe(0.5, 0.5)
                if e2 < 0:
                    pieces[e][f] = []
                elif vol[e2] > 1.5 * vol[e] or vol[e2] > 0.75 * vol[e] and probe(0.25, 0.25) == e2:
                    pieces[e][f] = [(e2, (0.0, 1.0, 0.0, 1.0))]
                else:
                    pieces[e][f] = [(probe(0.25 + 0.5 * u, 0.25 + 0.5 * v), (0.5 * u, 0.5 * u + 0.5, 0.5 * v, 0.5 * v + 0.5))
                                    for v in (0, 1) for u in (0, 1)]
        return pieces

    # -- volume terms ----------------------------------------------------------
    def _volume(self, e, uE, uH, dt, t0, src):
        """Volume part of R for element e: [B, 2, 3, q, N3]."""
        p, q, nk = int(self.p[e]), int(self.q[e]), int(self.nk[e])
        X8 = self.X8(e)
        xh, wx = _grid3(p + 2)
        pts = self._pts(e, p, xh, ("vol", p + 2))
        tau, wt = time_rule(q, nk)
        Lt = test_time_nk(q, nk, tau)  # [N_K q, T]
        wgt = dt * np.outer(wt, wx * pts.J)  # [T, P] : dt dxi * J dx^
        E, dE, cE = _fields(uE, pts, q, tau, dt, nk=nk)
        H, dH, cH = _fields(uH, pts, q, tau, dt, nk=nk)
        RE = _test_project(self.eps[e] * dE, pts, Lt, wgt) - _test_project_curl(H, pts, Lt, wgt)
        RH = _test_project(self.mu[e] * dH + cE, pts, Lt, wgt)
        if src is not None:
            # l_E(v) = (J, v): subtract
            t = t0 + dt * tau
            Jv = src(pts.x[None, :, :], t[:, None])  # [T, P, 3]
            RE = RE - _test_project(np.broadcast_to(Jv, (1,) + Jv.shape), pts, Lt, wgt)
        return np.stack([RE, RH], axis=1)

    # -- face terms ------------------------------------------------------------
    @staticmethod
    def _common_test_factors(q, nk, q2, nk2, tau, wt, Lt):
        """Pi~ L at the time points tau: the L2 projection (Eq. bilinearform:S) of the own
        temporal test factors Lt [N_K q, T] onto the largest common test space of the two
        elements, piecewise P_{min(q,q2)-1} on the coarser of the two (nested) partitions.
        None when that space is the own test space (Pi~ = identity on it)."""
        qt = min(q, q2)
        if qt == q and nk2 >= nk:
            return None
        Lc = test_time_nk(qt, min(nk, nk2), tau)
        gram = np.einsum("kt,t,lt->kl", Lc, wt, Lc)
        return np.linalg.solve(gram, np.einsum("kt,t,it->ki", Lc, wt, Lt)).T @ Lc

    def _face(self, e, f, e2, rect, uE, uH, vE, vH, dt, t0, g):
        """Contribution of one piece of face f of e (neighbour e2 or -1) to the rows of e.

        uE/uH: own coefficients [B, 3, q+1, N3]; vE/vH: the neighbour's (or None).
        rect = (u0, u1, v0, v1): the piece in e's tangential reference coordinates.
        """
        p, q, nk = int(self.p[e]), int(self.q[e]), int(self.nk[e])
        d, s = divmod(f, 2)
        X8 = self.X8(e)
        interior = e2 >= 0
        p2 = int(self.p[e2]) if interior else p
        q2 = int(self.q[e2]) if interior else q
        nk2 = int(self.nk[e2]) if interior else nk
        nq = max(p, p2) + 2
        xh, wa = _face_grid(d, s, nq)
        a1_, a2_ = [a for a in range(3) if a != d]
        u0, u1, v0, v1 = rect
        xh[:, a1_] = u0 + (u1 - u0) * xh[:, a1_]
        xh[:, a2_] = v0 + (v1 - v0) * xh[:, a2_]
        wa = wa * (u1 - u0) * (v1 - v0)
        pts = self._pts(e, p, xh, ("face", f, nq, rect))
        # surface measure and outward normal from the two tangent vectors
        a1, a2 = [a for a in range(3) if a != d]
        t1, t2 = pts.DF[:, :, a1], pts.DF[:, :, a2]
        c = _cross(t1, t2)
        dS = np.linalg.norm(c, axis=1)
        n = c / dS[:, None]
        outward = pts.DF[:, :, d] * (1.0 if s == 1 else -1.0)
        n = n * np.sign(np.sum(n * outward, axis=1))[:, None]
        # time rule on the finer of the two partitions (they are nested or equal)
        tau, wt = time_rule(max(q, q2), max(nk, nk2))
        Lt = test_time_nk(q, nk, tau)  # [N_K q, T]
        wgt = dt * np.outer(wt, wa * dS)  # [T, A]
        E1, _, _ = _fields(uE, pts, q, tau, dt, derivs=False, nk=nk)
        H1, _, _ = _fields(uH, pts, q, tau, dt, derivs=False, nk=nk)
        nn = n[None, None, :, :]
        if interior:
            X8b = self.X8(e2)
            key = ("inv", f, nq, p2, rect, tuple(np.round(X8b - X8[0], 13).ravel()))
            xh2 = self._vol_cache.get(key + (tuple(np.round(X8 - X8[0], 13).ravel()),))
            if xh2 is None:
                xh2 = geometry.inverse_map(X8b, pts.x)
                self._vol_cache[key + (tuple(np.round(X8 - X8[0], 13).ravel()),)] = xh2
            pts2 = self._pts(e2, p2, xh2, ("nbrface", tuple(np.round(xh2, 12).ravel())))
            E2, _, _ = _fields(vE, pts2, q2, tau, dt, derivs=False, nk=nk2)
            H2, _, _ = _fields(vH, pts2, q2, tau, dt, derivs=False, nk=nk2)
            Havg = 0.5 * (H1 + H2)
            Eavg = 0.5 * (E1 + E2)
            jE = _cross(nn, E1) - _cross(nn, E2)  # [E]_T = n1 x E1 + n2 x E2, n2 = -n1
            jH = _cross(nn, H1) - _cross(nn, H2)
            # E-eq:  <{H}, n x v>  = v . ({H} x n)
            RE = _test_project(_cross(Havg, nn), pts, Lt, wgt)
            # H-eq: -<[E]_T, {w}> , {w} = w / 2
            RH = _test_project(-0.5 * jE, pts, Lt, wgt)
            PL = self._common_test_factors(q, nk, q2, nk2, tau, wt, Lt)
            if self.c_diss > 0:
                # D_h: <alpha [F]_T, [Pi~ v]_T>; for the rows of e, [v]_T = n x v, and
                # a . (n x v) = v . (a x n)
                aE = self.c_diss / (0.5 * (np.sqrt(self.mu[e] / self.eps[e]) + np.sqrt(self.mu[e2] / self.eps[e2])))
                aH = self.c_diss / (0.5 * (np.sqrt(self.eps[e] / self.mu[e]) + np.sqrt(self.eps[e2] / self.mu[e2])))
                Lp = Lt if PL is None else PL
                RE = RE + aE * _test_project(_cross(jE, nn), pts, Lp, wgt)
                RH = RH + aH * _test_project(_cross(jH, nn), pts, Lp, wgt)
            if PL is not None:
                # S_h: test factors (Pi~ L_i - L_i)
                Ld = PL - Lt
                # E rows: 1/2 ( <{H}, n x (Pi~v - v)> + <[H]_T, (Pi~v - v)/2> )
                RE = RE + 0.5 * _test_project(_cross(Havg, nn) + 0.5 * jH, pts, Ld, wgt)
                # H rows: -1/2 ( <{E}, n x (Pi~w - w)> + <[E]_T, (Pi~w - w)/2> )
                RH = RH - 0.5 * _test_project(_cross(Eavg, nn) + 0.5 * jE, pts, Ld, wgt)
        else:
            # boundary: {H} = H, [v]_T = n x v ; [E]_T = n x E, {w} = w
            RE = _test_project(_cross(H1, nn), pts, Lt, wgt)
            RH = _test_project(-_cross(nn, E1), pts, Lt, wgt)
            gv = None
            if g is not None:
                # -l_H(w) = + <n x g, w>
                t = t0 + dt * tau
                gv = g(pts.x[None, :, :], t[:, None])  # [T, A, 3]
                RH = RH + _test_project(_cross(nn, gv[None]), pts, Lt, wgt)
            if self.c_diss > 0:
                # D_h on F_b: <alpha_E n x (E - g), n x v>, alpha_E = c / sqrt(mu/eps) of e
                aE = self.c_diss / np.sqrt(self.mu[e] / self.eps[e])
                jb = _cross(nn, E1 if gv is None else E1 - gv[None])
                RE = RE + aE * _test_project(_cross(jb, nn), pts, Lt, wgt)
        return np.stack([RE, RH], axis=1)

    # -- public API ------------------------------------------------------------
    def element_residual(self, e, U, t0, dt, src=None, g=None, parts="all"):
        """R for the test functions of element e, layout [B, 2, 3, q, N3].

        U: [B, N_trial] or [N_trial]; ``parts`` = "all" | "own" | ("nbr", e2)
        selects the contribution of element e's own coefficients (volume and
        own face traces, no load) or of neighbour element e2's coefficients.
        """
        if not isinstance(U, dict):
            U = np.atleast_2d(U)
        u = self.trial_block(U, e)
        B = u.shape[0]
        p, q = int(self.p[e]), int(self.q[e])
        R = np.zeros((B, 2, 3, int(self.nk[e]) * q, (p + 1) ** 3))
        if parts in ("all", "own"):
            R += self._volume(e, u[:, 0], u[:, 1], dt, t0, src if parts == "all" else None)
        for f in range(6):
            plist = self.pieces[e][f]
            if not plist:  # boundary face
                if parts in ("all", "own"):
                    R += self._face(e, f, -1, (0.0, 1.0, 0.0, 1.0), u[:, 0], u[:, 1], None, None, dt, t0,
                                    g if parts == "all" else None)
                continue
            for e2, rect in plist:
                if parts == "all":
                    own, nb = u, self.trial_block(U, e2)
                elif parts == "own":
                    own, nb = u, None
                else:
                    if parts[1] != e2:
                        continue
                    own, nb = None, self.trial_block(U, e2)
                R += self._face(e, f, e2, rect, None if own is None else own[:, 0], None if own is None else own[:, 1],
                                None if nb is None else nb[:, 0], None if nb is None else nb[:, 1], dt, t0, None)
        return R

    def neighbours_of(self, e):
        """Elements that share a face (or a piece of one) with e."""
        return sorted({e2 for f in range(6) for e2, _ in self.pieces[e][f]})

    def residual(self, U, t0, dt, src=None, g=None, elems=None) -> np.ndarray:
        """R_h(U) = B_h(U, .) - L(.) in the test layout (concatenated over ``elems``)."""
        elems = range(self.ne) if elems is None else elems
        out = [self.element_residual(e, U, t0, dt, src, g)[0].ravel() for e in elems]
        return np.concatenate(out) if out else np.zeros(0)

    def assemble(self, t0, dt, src=None, g=None):
        """Sparse A (test x trial) and b with R_h(U) = A U - b."""
        rows, cols, vals = [], [], []
        ntr = int(self.trial_off[-1])
        b = -self.residual(np.zeros(ntr), t0, dt, src, g)
        for e in range(self.ne):
            r0 = self.test_off[e]
            blocks = [("own", e)] + [(("nbr", e2), e2) for e2 in self.neighbours_of(e)]
            for part, e2 in blocks:
                m = int(self.trial_sz[e2])
                # unit vectors of element e2's trial block (only that block is formed)
                Ub = {e2: np.eye(m).reshape(m, 2, 3, int(self.nk[e2] * self.q[e2]) + 1, (int(self.p[e2]) + 1) ** 3)}
                Rb = self.element_residual(e, Ub, t0, dt, None, None, parts=part).reshape(m, -1)
                Rb = Rb.T  # [test, m]
                ii, jj = np.nonzero(Rb)
                rows.append(r0 + ii)
                cols.append(self.trial_off[e2] + jj)
                vals.append(Rb[ii, jj])
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(int(self.test_off[-1]), ntr))
        A.sum_duplicates()
        return A, b

    def time_derivative(self, U, dt, elems=None) -> np.ndarray:
        """The preconditioner form of Eq. preconditioner (Sec. 5.4), the time-derivative
        terms of C_h alone, P(U, V) = (eps d_t E, v) + (mu d_t H, w), for every test basis
        function V, in the test layout (concatenated over ``elems``)."""
        elems = range(self.ne) if elems is None else elems
        U = np.atleast_2d(U)
        out = []
        for e in elems:
            u = self.trial_block(U, e)
            p, q, nk = int(self.p[e]), int(self.q[e]), int(self.nk[e])
            xh, wx = _grid3(p + 2)
            pts = self._pts(e, p, xh, ("vol", p + 2))
            tau, wt = time_rule(q, nk)
            Lt = test_time_nk(q, nk, tau)
            wgt = dt * np.outer(wt, wx * pts.J)
            _, dE, _ = _fields(u[:, 0], pts, q, tau, dt, nk=nk)
            _, dH, _ = _fields(u[:, 1], pts, q, tau, dt, nk=nk)
            RE = _test_project(self.eps[e] * dE, pts, Lt, wgt)
            RH = _test_project(self.mu[e] * dH, pts, Lt, wgt)
            out.append(np.stack([RE, RH], axis=1)[0].ravel())
        return np.concatenate(out) if out else np.zeros(0)

    def unknown_mask(self) -> np.ndarray:
        """Boolean mask over the trial vector: True for modes m >= 1 (the slab unknowns)."""
        mask = np.zeros(int(self.trial_off[-1]), dtype=bool)
        for e in range(self.ne):
            n3 = (self.p[e] + 1) ** 3
            blk = np.zeros((2, 3, self.nk[e] * self.q[e] + 1, n3), dtype=bool)
            blk[:, :, 1:, :] = True
            mask[self.trial_off[e]:self.trial_off[e + 1]] = blk.ravel()
        return mask

    def slab_solve(self, u0, t0, dt, src=None, g=None, A_b=None):
        """Solve R_h(U) = 0 for modes m >= 1 given the slab-start coefficients.

        u0: spatial coefficients at t0, layout per element [2, 3, N3] concatenated.
        Returns the full trial vector U.
        """
        A, b = self.assemble(t0, dt, src, g) if A_b is None else A_b
        U = self.embed_start(u0)
        mask = self.unknown_mask()
        rhs = b - A[:, ~mask] @ U[~mask]
        if getattr(self, "_lu_key", None) is not A:
            # sparse LU of the unknown block, reused while the operator is the same object
            self._lu = spla.splu(A[:, mask].tocsc())
            self._lu_key = A
        U[mask] = self._lu.solve(rhs)
        return U

    def embed_start(self, u0) -> np.ndarray:
        """Trial vector with the slab-start coefficient u0 and all other modes 0."""
        U = np.zeros(int(self.trial_off[-1]))
        o0 = 0
        for e in range(self.ne):
            n3 = int((self.p[e] + 1) ** 3)
            blk = np.zeros((2, 3, int(self.nk[e] * self.q[e]) + 1, n3))
            blk[:, :, 0, :] = u0[o0:o0 + 6 * n3].reshape(2, 3, n3)
            o0 += 6 * n3
            U[self.trial_off[e]:self.trial_off[e + 1]] = blk.ravel()
        return U

    def end_state(self, U) -> np.ndarray:
        """Spatial coefficients of the trial function at xi = 1."""
        return self._state_at(U, 1.0)

    def start_state(self, U) -> np.ndarray:
        return self._state_at(U, 0.0)

    def _state_at(self, U, xi) -> np.ndarray:
        out = []
        for e in range(self.ne):
            u = self.trial_block(U, e)
            lt = trial_time_nk(int(self.q[e]), int(self.nk[e]), np.array([xi]))[:, 0]
            out.append(np.einsum("m,fcms->fcs", lt, u).ravel())
        return np.concatenate(out)

    def energy(self, u) -> float:
        """E(t) = 1/2 int eps E.E + mu H.H for spatial coefficients u [per element 2,3,N3]."""
        tot = 0.0
        o = 0
        for e in range(self.ne):
            p = int(self.p[e])
            n3 = (p + 1) ** 3
            blk = u[o:o + 6 * n3].reshape(2, 3, n3)
            o += 6 * n3
            xh, w = _grid3(p + 2)
            pts = _points(self.X8(e), p, xh)
            ref = np.einsum("fcs,ps->fpc", blk, pts.phi)
            phys = np.einsum("pci,fpc->fpi", pts.DFinv, ref)
            dens = self.eps[e] * np.sum(phys[0] ** 2, axis=1) + self.mu[e] * np.sum(phys[1] ** 2, axis=1)
            tot += 0.5 * np.sum(w * pts.J * dens)
        return tot

    def project(self, Efn, Hfn) -> np.ndarray:
        """L2 projection of E0(x), H0(x) onto the covariant spatial spaces (per element [2,3,N3])."""
        out = []
        for e in range(self.ne):
            p = int(self.p[e])
            n3 = (p + 1) ** 3
            xh, w = _grid3(p + 2)
            pts = _points(self.X8(e), p, xh)
            # basis functions DF^{-T} phi_s e_c at points: [P, 3(phys), 3(c), N3]
            Bf = np.einsum("pci,ps->pics", pts.DFinv, pts.phi).reshape(len(w), 3, 3 * n3)
            M = np.einsum("p,pia,pib->ab", w * pts.J, Bf, Bf)
            blk = []
            for fn in (Efn, Hfn):
                v = fn(pts.x) if fn is not None else np.zeros((len(w), 3))
                rhs = np.einsum("p,pia,pi->a", w * pts.J, Bf, v)
                blk.append(np.linalg.solve(M, rhs))
            out.append(np.concatenate(blk))
        return np.concatenate(out)

    def test_projection_in_time(self, U) -> np.ndarray:
        """pi U: the L2 projection of U onto the element's temporal test space, as
        coefficients of the test functions L_i on each sub-interval (test layout)."""
        out = []
        for e in range(self.ne):
            q, nk = int(self.q[e]), int(self.nk[e])
            u = self.trial_block(U, e)
            tau, wt = time_rule(q, nk)
            lt = trial_time_nk(q, nk, tau)
            Lt = test_time_nk(q, nk, tau)
            # int_{I_k} L_i^k L_i^k dxi = 1/N_K
            B = nk * np.einsum("it,t,mt->im", Lt, wt, lt)
            out.append(np.einsum("im,fcms->fcis", B, u).ravel())
        return np.concatenate(out)
