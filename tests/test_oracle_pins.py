"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: closed forms of the
1-D tables, a library Legendre routine, finite differences, a hand-derived
two-element result, the discrete energy identity (Theorems 3.1 / 4.1), an
exact polynomial solution, the Gauss-collocation / Pade equivalence of
continuous Galerkin in time, rigid-motion invariance and the analytic PEC
cavity mode of Sec. 6.1.1.  The last tests plant mistakes in the oracle and
check that the pins catch them.
"""
import math

import numpy as np
import pytest

from oracle import basis, geometry, stdg
from paper_1307_5310_gb300 import meshgen

W_CAV = math.sqrt(2.0) * math.pi


def cavity_E(x, t=0.0):
    z = np.zeros(x.shape[0])
    return np.stack([z, z, np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.cos(W_CAV * t)], 1)


def cavity_H(x, t=0.0):
    s = math.sin(W_CAV * t) / math.sqrt(2.0)
    return np.stack([-np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * s,
                     np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * s,
                     np.zeros(x.shape[0])], 1)


# --------------------------------------------------------------------------
# P1: 1-D tables against closed forms
# --------------------------------------------------------------------------

def _quad_tables(q, n):
    tau, wt = basis.gauss01(q + 4)
    L = basis.legendre(q, tau)
    l = basis.trial_time(q, tau)
    dl = basis.trial_time_deriv(q, tau)
    A = np.einsum("it,t,mt->im", L[:q], wt, dl)
    B = np.einsum("it,t,mt->im", L[:q], wt, l)
    x, w = basis.gauss01(n + 2)
    Ls = basis.legendre(n - 1, x)
    dLs = basis.legendre_deriv(n - 1, x)
    D = np.einsum("ax,x,bx->ab", Ls, w, dLs)
    M = np.einsum("ax,x,bx->ab", Ls, w, Ls)
    return A, B, D, M


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_time_tables_closed_form(q):
    A, B, _, _ = _quad_tables(q, 3)
    # A_im = int L_i l_m' : -delta_i0 for m = 0, delta_{i,m-1} for m >= 1
    Ac = np.zeros((q, q + 1))
    Ac[0, 0] = -1.0
    for m in range(1, q + 1):
        Ac[m - 1, m] = 1.0
    assert np.abs(A - Ac).max() < 1e-14
    # B_im = int L_i l_m (banded; derived from l_m = (P_m - P_{m-2}) / (2 sqrt(2m-1)))
    Bc = np.zeros((q, q + 1))
    Bc[0, 0] = 0.5
    Bc[0, 1] = 0.5
    if q >= 2:
        Bc[1, 0] = -1.0 / (2 * math.sqrt(3.0))
        Bc[1, 1] = 1.0 / (2 * math.sqrt(3.0))
    for m in range(2, q + 1):
        if m <= q - 1:
            Bc[m, m] = 1.0 / (2 * math.sqrt(2 * m - 1) * math.sqrt(2 * m + 1))
        Bc[m - 2, m] = -1.0 / (2 * math.sqrt(2 * m - 1) * math.sqrt(2 * m - 3))
    assert np.abs(B - Bc).max() < 1e-14
    assert np.count_nonzero(np.abs(B) > 1e-14) == (2 if q == 1 else 2 * q + 1)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_space_tables_closed_form(n):
    _, _, D, M = _quad_tables(1, n)
    assert np.abs(M - np.eye(n)).max() < 1e-13
    Dc = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            if a < b and (b - a) % 2 == 1:
                Dc[a, b] = 2 * math.sqrt(2 * a + 1) * math.sqrt(2 * b + 1)
    assert np.abs(D - Dc).max() < 1e-12
    assert np.count_nonzero(np.abs(D) > 1e-12) == n * n // 4
    # face values L_j(1) = sqrt(2j+1), L_j(0) = (-1)^j sqrt(2j+1)
    v1 = basis.legendre(n - 1, np.array([1.0]))[:, 0]
    v0 = basis.legendre(n - 1, np.array([0.0]))[:, 0]
    j = np.arange(n)
    assert np.abs(v1 - np.sqrt(2 * j + 1)).max() < 1e-13
    assert np.abs(v0 - (-1.0) ** j * np.sqrt(2 * j + 1)).max() < 1e-13


def test_legendre_matches_library():
    x = np.linspace(0, 1, 17)
    L = basis.legendre(7, x)
    for k in range(8):
        ref = np.polynomial.legendre.Legendre.basis(k)(2 * x - 1) * math.sqrt(2 * k + 1)
        assert np.abs(L[k] - ref).max() < 1e-12
        dref = np.polynomial.legendre.Legendre.basis(k).deriv()(2 * x - 1) * 2 * math.sqrt(2 * k + 1)
        assert np.abs(basis.legendre_deriv(7, x)[k] - dref).max() < 1e-10


def test_trial_time_end_values():
    l0 = basis.trial_time(5, np.array([0.0]))[:, 0]
    l1 = basis.trial_time(5, np.array([1.0]))[:, 0]
    assert np.allclose(l0, [1, 0, 0, 0, 0, 0], atol=1e-15)
    assert np.allclose(l1, [0, 1, 0, 0, 0, 0], atol=1e-15)


# --------------------------------------------------------------------------
# geometry: Piola curl against finite differences
# --------------------------------------------------------------------------

def test_piola_curl_finite_difference():
    rng = np.random.Generator(np.random.PCG64(7))
    X8 = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) * 0.5
    X8 = X8 + 0.05 * rng.uniform(-1, 1, X8.shape)
    p = 2
    coef = rng.uniform(-1, 1, (1, 3, 2, 27))
    coef[:, :, 1] = 0.0

    def field(x):
        xh = geometry.inverse_map(X8, x)
        pts = stdg._points(X8, p, xh)
        val, _, _ = stdg._fields(coef, pts, 1, np.array([0.0]), 1.0, derivs=False)
        return val[0, 0]

    xh0 = np.array([[0.3, 0.6, 0.45]])
    pts = stdg._points(X8, p, xh0)
    _, _, curl = stdg._fields(coef, pts, 1, np.array([0.0]), 1.0)
    x0 = pts.x[0]
    h = 1e-5
    grad = np.zeros((3, 3))  # grad[i, a] = d F_i / d x_a
    for a in range(3):
        dx = np.zeros(3)
        dx[a] = h
        grad[:, a] = (field((x0 + dx)[None])[0] - field((x0 - dx)[None])[0]) / (2 * h)
    fd = np.array([grad[2, 1] - grad[1, 2], grad[0, 2] - grad[2, 0], grad[1, 0] - grad[0, 1]])
    assert np.abs(fd - curl[0, 0, 0]).max() < 1e-6


# --------------------------------------------------------------------------
# P8: brute force, two unit cubes with p = 0, q = 1 (hand-derived)
# --------------------------------------------------------------------------

def test_two_cube_p0_closed_form():
    m = meshgen.box_mesh(2, 1, 1, hi=(2.0, 1.0, 1.0), p=0, q=1)
    m["eps"] = np.array([2.0, 3.0])
    m["mu"] = np.array([1.5, 0.5])
    o = stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(3))
    U = rng.uniform(-1, 1, o.trial_off[-1])
    dt = 0.37
    R = o.residual(U, 0.0, dt).reshape(2, 2, 3)
    u = U.reshape(2, 2, 3, 2)  # [el][field][c][m]
    ex = np.array([1.0, 0, 0])
    for k, other, nrm in ((0, 1, ex), (1, 0, -ex)):
        # unit cube: covariant = physical for p = 0; constant fields
        Ebar = 0.5 * (u[:, 0, :, 0] + u[:, 0, :, 1])
        Hbar = 0.5 * (u[:, 1, :, 0] + u[:, 1, :, 1])
        RE = m["eps"][k] * (u[k, 0, :, 1] - u[k, 0, :, 0])
        RH = m["mu"][k] * (u[k, 1, :, 1] - u[k, 1, :, 0])
        # boundary faces of a cube minus the shared one sum their normals to -nrm
        for d in range(3):
            ed = np.eye(3)[d]
            RE[d] += dt * 0.5 * np.dot(Hbar[other] - Hbar[k], np.cross(nrm, ed))
            RH[d] += dt * 0.5 * np.cross(nrm, Ebar[k] + Ebar[other])[d]
        assert np.abs(R[k, 0] - RE).max() < 1e-14
        assert np.abs(R[k, 1] - RH).max() < 1e-14


def test_two_cube_p0_dissipation_closed_form():
    """D_h (Sec. 4.2) on two unit cubes, p = 0, q = 1, by hand: the E rows of
    component d collect alpha dt (mean E jump)_d over every face tangential to
    d (boundary faces: alpha_E = c sqrt(eps/mu) of the element, jump = E), the
    H rows only the interior face."""
    m = meshgen.box_mesh(2, 1, 1, hi=(2.0, 1.0, 1.0), p=0, q=1)
    m["eps"] = np.array([2.0, 3.0])
    m["mu"] = np.array([1.5, 0.5])
    c = 0.7
    o, o0 = stdg.Oracle(m, c_diss=c), stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(4))
    U = rng.uniform(-1, 1, o.trial_off[-1])
    dt = 0.29
    D = (o.residual(U, 0.0, dt) - o0.residual(U, 0.0, dt)).reshape(2, 2, 3)
    u = U.reshape(2, 2, 3, 2)
    Ebar = 0.5 * (u[:, 0, :, 0] + u[:, 0, :, 1])
    Hbar = 0.5 * (u[:, 1, :, 0] + u[:, 1, :, 1])
    eps, mu = m["eps"], m["mu"]
    aE = c / (0.5 * (np.sqrt(mu[0] / eps[0]) + np.sqrt(mu[1] / eps[1])))
    aH = c / (0.5 * (np.sqrt(eps[0] / mu[0]) + np.sqrt(eps[1] / mu[1])))
    quad = 0.0
    for k in (0, 1):
        ab = c * np.sqrt(eps[k] / mu[k])
        nb = np.array([4, 3, 3])  # boundary faces tangential to x, y, z
        DE = ab * dt * nb * Ebar[k]
        DH = np.zeros(3)
        for d in (1, 2):  # tangential to the shared x-face
            DE[d] += aE * dt * (Ebar[k, d] - Ebar[1 - k, d])
            DH[d] += aH * dt * (Hbar[k, d] - Hbar[1 - k, d])
        assert np.abs(D[k, 0] - DE).max() < 1e-14
        assert np.abs(D[k, 1] - DH).max() < 1e-14
        quad += ab * dt * float(nb @ Ebar[k] ** 2)
    jE, jH = Ebar[0, 1:] - Ebar[1, 1:], Hbar[0, 1:] - Hbar[1, 1:]
    quad += aE * dt * float(jE @ jE) + aH * dt * float(jH @ jH)
    # dissipation identity: R(U) . Pi U = E(t1) - E(t0) + D(U, Pi U), the last a sum of squares
    lhs = o.residual(U, 0.0, dt) @ o.test_projection_in_time(U)
    dE = o.energy(o.end_state(U)) - o.energy(o.start_state(U))
    assert abs(lhs - dE - quad) < 1e-13


@pytest.mark.parametrize("case", ["brick", "uneven_q", "uneven_p"])
def test_dissipation_nonnegative(case):
    """With c > 0 the energy identity gains -D(U, Pi U) <= 0, linear in c."""
    m = meshgen.box_mesh(2, p=2, q=2)
    if case == "uneven_q":
        m["q"] = np.array([1, 2, 3, 1, 2, 3, 4, 1], dtype=np.uint8)
    elif case == "uneven_p":
        m["p"] = np.array([1, 2, 3, 1, 2, 3, 1, 2], dtype=np.uint8)
    meshgen.random_materials(m, 5, 6)
    U = meshgen.random_coeffs(m, 11)
    dt = 0.13
    out = []
    for c in (0.0, 0.5, 1.0):
        o = stdg.Oracle(m, c_diss=c)
        piU = o.test_projection_in_time(U)
        dE = o.energy(o.end_state(U)) - o.energy(o.start_state(U))
        out.append(o.residual(U, 0.0, dt) @ piU - dE)
    assert abs(out[0]) <= 1e-12 * max(1.0, abs(out[2]))
    assert out[1] > 0 and abs(out[2] - 2 * out[1]) <= 1e-11 * out[2]


# --------------------------------------------------------------------------
# P4: discrete energy identity for arbitrary U (Theorems 3.1 / 4.1)
# --------------------------------------------------------------------------

def _energy_identity(m, dt=0.13, seed=11):
    o = stdg.Oracle(m)
    U = meshgen.random_coeffs(m, seed)
    R = o.residual(U, 0.0, dt)
    piU = o.test_projection_in_time(U)
    dE = o.energy(o.end_state(U)) - o.energy(o.start_state(U))
    return R @ piU, dE


SHEAR = [[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.2, 1.1]]


@pytest.mark.parametrize("case", ["brick", "aniso", "affine", "curved", "uneven_q", "uneven_p"])
def test_energy_identity(case):
    if case == "brick":
        m = meshgen.box_mesh(2, p=2, q=2)
    elif case == "affine":
        m = meshgen.box_mesh(2, 2, 1, p=2, q=2, affine=SHEAR)
    elif case == "aniso":
        m = meshgen.box_mesh(3, 2, 1, hi=(1.0, 0.5, 0.25), p=1, q=3)
    elif case == "curved":
        m = meshgen.box_mesh(3, p=2, q=2, perturb=0.3)
    elif case == "uneven_q":
        m = meshgen.box_mesh(2, p=2, q=1)
        m["q"] = np.array([1, 2, 3, 1, 2, 3, 4, 1], dtype=np.uint8)
    else:
        m = meshgen.box_mesh(2, p=2, q=2)
        m["p"] = np.array([1, 2, 3, 1, 2, 3, 1, 2], dtype=np.uint8)
    meshgen.random_materials(m, 5, 6)
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) <= 1e-12 * max(1.0, abs(dE))


@pytest.mark.parametrize("uneven", [False, True])
def test_energy_identity_hanging(uneven):
    """2:1 hanging faces (corner-refined octree): the identity needs every face piece."""
    m = meshgen.corner_octree_mesh(2, [0.8], p=2, q=2)
    assert m["hang"].shape[0] == 12
    if uneven:
        meshgen.random_hp(m, 3, p_range=(1, 3), q_range=(1, 3))
    else:
        meshgen.random_materials(m, 5, 6)
    o = stdg.Oracle(m)
    # the oracle finds the hanging faces itself: 3 coarse faces in 4 pieces each, 12 fine faces
    assert sum(len(o.pieces[e][f]) == 4 for e in range(o.ne) for f in range(6)) == 3
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) <= 1e-12 * max(1.0, abs(dE))


def test_patch_hanging():
    """E = (y, x, 0), H = (0, 0, 1) is reproduced exactly across 2:1 faces."""
    m = meshgen.corner_octree_mesh(2, [0.8], p=1, q=1)
    meshgen.random_hp(m, 9, p_range=(1, 2), q_range=(1, 3), eps_values=(1.0,))
    o = stdg.Oracle(m)
    Ef = lambda x: np.stack([x[:, 1], x[:, 0], 0 * x[:, 0]], 1)
    Hf = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], 1 + 0 * x[:, 0]], 1)
    u0 = o.project(Ef, Hf)
    U = o.embed_start(u0)
    for e in range(o.ne):
        blk = o.trial_block(U, e)
        blk[:, :, 1, :] = blk[:, :, 0, :]

    def g(x, t):
        z = np.zeros(np.broadcast(x[..., 0], t).shape)
        return np.stack([x[..., 1] + z, x[..., 0] + z, z], -1)

    assert np.abs(o.residual(U, 0.0, 0.2, g=g)).max() < 1e-12


# --------------------------------------------------------------------------
# P6: polynomial patch test E = (0,0,x), H = (0,t,0), g = E
# --------------------------------------------------------------------------

def _patch(m, t0=0.3, dt=0.2, c_diss=0.0):
    o = stdg.Oracle(m, c_diss=c_diss)

    def Ef(x):
        z = np.zeros(x.shape[0])
        return np.stack([z, z, x[:, 0]], 1)

    def Hf(t):
        return lambda x: np.stack([0 * x[:, 0], t + 0 * x[:, 0], 0 * x[:, 0]], 1)

    u0 = o.project(Ef, Hf(t0))
    u1 = o.project(Ef, Hf(t0 + dt))
    U = o.embed_start(u0)
    o0 = 0
    for e in range(o.ne):
        n3 = (int(o.p[e]) + 1) ** 3
        blk = o.trial_block(U, e)
        blk[:, :, 1, :] = u1[o0:o0 + 6 * n3].reshape(2, 3, n3)
        o0 += 6 * n3

    def g(x, t):
        z = np.zeros(np.broadcast(x[..., 0], t).shape)
        return np.stack([z, z, x[..., 0] + z], -1)

    return o, U, u0, g, t0, dt


@pytest.mark.parametrize("case", ["brick", "curved", "uneven"])
def test_patch_exact(case):
    if case == "brick":
        m = meshgen.box_mesh(2, 2, 1, p=1, q=1)
    elif case == "curved":
        m = meshgen.box_mesh(2, p=2, q=1, perturb=0.4)
    else:
        # S_h replaces the neighbour's temporal test factors by their projection
        # onto P_{min(q1,q2)-1}; it is consistent for this solution (H linear in
        # t) only where min(q1, q2) >= 2.  q = 1 faces are covered by the
        # time-constant patch below.
        m = meshgen.box_mesh(2, p=2, q=1)
        m["p"] = np.array([1, 2, 1, 2, 2, 1, 2, 1], dtype=np.uint8)
        m["q"] = np.array([2, 3, 4, 2, 3, 2, 2, 3], dtype=np.uint8)
    o, U, u0, g, t0, dt = _patch(m)
    R = o.residual(U, t0, dt, g=g)
    assert np.abs(R).max() < 1e-12
    Us = o.slab_solve(u0, t0, dt, g=g)
    assert np.abs(Us - U).max() < 1e-11


@pytest.mark.parametrize("case", ["brick", "uneven"])
def test_patch_exact_dissipative(case):
    """D_h vanishes on a solution with continuous tangential traces and E = g on F_b."""
    m = meshgen.box_mesh(2, 2, 1, p=1, q=1) if case == "brick" else meshgen.box_mesh(2, p=2, q=2)
    if case == "uneven":
        m["p"] = np.array([1, 2, 1, 2, 2, 1, 2, 1], dtype=np.uint8)
        m["q"] = np.array([2, 3, 4, 2, 3, 2, 2, 3], dtype=np.uint8)
    o, U, u0, g, t0, dt = _patch(m, c_diss=0.8)
    assert np.abs(o.residual(U, t0, dt, g=g)).max() < 1e-12
    # without the boundary data the E - g term of D_h is what remains on F_b
    assert np.abs(o.residual(U, t0, dt)).max() > 1e-3


def test_patch_time_constant_uneven_q():
    """E = (y, x, 0), H = (0, 0, 1) solves Maxwell (eps = mu = 1, J = 0, g = E) and is constant in time."""
    m = meshgen.box_mesh(2, p=1, q=1)
    m["p"] = np.array([1, 2, 1, 2, 2, 1, 2, 1], dtype=np.uint8)
    m["q"] = np.array([1, 2, 3, 1, 2, 1, 4, 2], dtype=np.uint8)
    o = stdg.Oracle(m)
    Ef = lambda x: np.stack([x[:, 1], x[:, 0], 0 * x[:, 0]], 1)
    Hf = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], 1 + 0 * x[:, 0]], 1)
    u0 = o.project(Ef, Hf)
    U = o.embed_start(u0)
    for e in range(o.ne):
        blk = o.trial_block(U, e)
        blk[:, :, 1, :] = blk[:, :, 0, :]

    def g(x, t):
        z = np.zeros(np.broadcast(x[..., 0], t).shape)
        return np.stack([x[..., 1] + z, x[..., 0] + z, z], -1)

    assert np.abs(o.residual(U, 0.0, 0.3, g=g)).max() < 1e-12
    assert np.abs(o.slab_solve(u0, 0.0, 0.3, g=g) - U).max() < 1e-11


# --------------------------------------------------------------------------
# P3: cG(q) in time = q-stage Gauss collocation = diagonal Pade R_{q,q}
# --------------------------------------------------------------------------

def _pade_num(q, z):
    return sum(math.factorial(2 * q - k) * math.factorial(q) /
               (math.factorial(2 * q) * math.factorial(k) * math.factorial(q - k)) * z ** k
               for k in range(q + 1))


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_scalar_ode_pade(q):
    tau, wt = basis.gauss01(q + 3)
    L = basis.legendre(q - 1, tau)
    l = basis.trial_time(q, tau)
    dl = basis.trial_time_deriv(q, tau)
    for z in (-0.7, 0.3, -2.5):
        # u' = (z/dt) u tested with L_i: sum_m (int L_i l_m' - z int L_i l_m) u_m = 0
        Mt = np.einsum("it,t,mt->im", L, wt, dl) - z * np.einsum("it,t,mt->im", L, wt, l)
        u1 = np.linalg.solve(Mt[:, 1:], -Mt[:, 0])  # u_0 = 1
        end = basis.trial_time(q, np.array([1.0]))[1:, 0] @ u1
        ref = _pade_num(q, z) / _pade_num(q, -z)
        assert abs(end - ref) < 1e-13


def test_maxwell_gauss_collocation():
    """Slab solutions for q = 2, 3 equal R_{q,q}(dt L) u0, L = -M^{-1} K from the q = 1 operator."""
    dt = 0.21
    base = meshgen.box_mesh(2, 1, 1, hi=(1.0, 0.5, 0.5), p=1, q=1)
    meshgen.random_materials(base, 1, 2)
    o1 = stdg.Oracle(base)
    A1, _ = o1.assemble(0.0, dt)
    A1 = A1.toarray()
    mask = o1.unknown_mask()
    # q = 1 rows: M (u1 - u0) + dt K (u0 + u1) / 2
    Au0, Au1 = A1[:, ~mask], A1[:, mask]
    M = 0.5 * (Au1 - Au0)
    K = (Au1 + Au0) / dt
    # M must be the plain L2 mass matrix of the covariant space
    n3 = 8
    for e in range(o1.ne):
        blk = slice(e * 6 * n3, (e + 1) * 6 * n3)
        Mb = M[blk, blk]
        assert np.abs(Mb - Mb.T).max() < 1e-13
        assert np.linalg.eigvalsh(Mb).min() > 0
    Lop = -np.linalg.solve(M, K)
    rng = np.random.Generator(np.random.PCG64(4))
    u0 = rng.uniform(-1, 1, M.shape[0])
    for q in (2, 3):
        m = dict(base)
        m["q"] = np.full(base["hex"].shape[0], q, dtype=np.uint8)
        o = stdg.Oracle(m)
        U = o.slab_solve(u0, 0.0, dt)
        end = o.end_state(U)
        Z = dt * Lop
        num = sum(math.factorial(2 * q - k) * math.factorial(q) /
                  (math.factorial(2 * q) * math.factorial(k) * math.factorial(q - k)) *
                  np.linalg.matrix_power(Z, k) for k in range(q + 1))
        den = sum(math.factorial(2 * q - k) * math.factorial(q) /
                  (math.factorial(2 * q) * math.factorial(k) * math.factorial(q - k)) *
                  np.linalg.matrix_power(-Z, k) for k in range(q + 1))
        ref = np.linalg.solve(den, num @ u0)
        assert np.abs(end - ref).max() < 1e-11 * np.abs(ref).max()


# --------------------------------------------------------------------------
# P7: invariance under rigid motions
# --------------------------------------------------------------------------

def test_rigid_motion_invariance():
    m = meshgen.box_mesh(2, p=2, q=2, perturb=0.3)
    meshgen.random_materials(m, 8, 9)
    U = meshgen.random_coeffs(m, 3)
    R0 = stdg.Oracle(m).residual(U, 0.0, 0.1)
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    Q = Q @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    m2 = dict(m)
    m2["vert"] = m["vert"] @ Q.T + np.array([3.0, -1.0, 0.5])
    R1 = stdg.Oracle(m2).residual(U, 0.0, 0.1)
    assert np.abs(R1 - R0).max() < 1e-12 * np.abs(R0).max()


# --------------------------------------------------------------------------
# P5: analytic PEC cavity mode (Sec. 6.1.1 with m = n = 1 on the unit cube)
# --------------------------------------------------------------------------

def _cavity_run(N, p, q, nslab, dt):
    m = meshgen.box_mesh(N, p=p, q=q)
    o = stdg.Oracle(m)
    u = o.project(cavity_E, None)
    A_b = o.assemble(0.0, dt)
    E0 = o.energy(u)
    energies = [E0]
    for n in range(nslab):
        U = o.slab_solve(u, n * dt, dt, A_b=A_b)
        u = o.end_state(U)
        energies.append(o.energy(u))
    T = nslab * dt
    ue = o.project(lambda x: cavity_E(x, T), lambda x: cavity_H(x, T))
    err = math.sqrt(2 * o.energy(u - ue))  # eps = mu = 1: L2 norm of (E, H)
    return err, np.array(energies)


@pytest.mark.slow
def test_cavity_mode_plain_config():
    # 4^3 bricks, p = 2, q = 1, 20 slabs of 0.05
    err, en = _cavity_run(4, 2, 1, 20, 0.05)
    assert abs(en[0] - 0.125) < 1e-5
    assert np.abs(en - en[0]).max() <= 1e-12 * en[0]
    assert err < 1.5e-2


def test_cavity_mode_p_convergence():
    errs = [_cavity_run(2, p, p, 2, 0.05)[0] for p in (1, 2, 3)]
    # exponential in p: the reduction factor per degree does not shrink (an
    # algebraic rate p^-k would give factors (2/1)^k > (3/2)^k)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 > 4 and r2 >= r1


# --------------------------------------------------------------------------
# planted mistakes: the pins must catch them
# --------------------------------------------------------------------------

def test_planted_mistakes_fail_pins(monkeypatch):
    m = meshgen.box_mesh(2, p=1, q=2)
    meshgen.random_materials(m, 5, 6)
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) < 1e-12

    # 1) sign of the volume curl of the test function flipped
    orig = stdg._test_project_curl
    monkeypatch.setattr(stdg, "_test_project_curl", lambda *a: -orig(*a))
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) > 1e-6
    monkeypatch.setattr(stdg, "_test_project_curl", orig)

    # 2) trial time functions l_0 and l_1 swapped (wrong slab orientation)
    orig_t = basis.trial_time

    def swapped(q, x):
        out = orig_t(q, x)
        return out[[1, 0] + list(range(2, q + 1))]
    monkeypatch.setattr(basis, "trial_time", swapped)
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) > 1e-6
    monkeypatch.setattr(basis, "trial_time", orig_t)

    # 3) interior face average taken without the factor 1/2 is caught by the patch test
    o, U, u0, g, t0, dt = _patch(meshgen.box_mesh(2, 1, 1, p=1, q=1))
    R = o.residual(U, t0, dt, g=g)
    assert np.abs(R).max() < 1e-12
    orig_face = stdg.Oracle._face

    def bad_face(self, e, f, e2, rect, uE, uH, vE, vH, dt, t0, g):
        r = orig_face(self, e, f, e2, rect, uE, uH, vE, vH, dt, t0, g)
        if e2 >= 0:
            r = r.copy()
            r[:, 0] *= 2.0
        return r
    monkeypatch.setattr(stdg.Oracle, "_face", bad_face)
    R = o.residual(U, t0, dt, g=g)
    assert np.abs(R).max() > 1e-3


# --------------------------------------------------------------------------
# Local refinement in time (N_K sub-intervals per element, Sec. 2.2 / 4.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nk,q", [(2, 1), (2, 2), (4, 2), (3, 3)])
def test_uniform_time_refinement_is_substepping(nk, q):
    """Every element with N_K equal sub-intervals: the common test space is the own one
    (S_h = 0) and the sub-interval equations decouple in time order, so one slab equals
    N_K slabs of dt / N_K."""
    m = meshgen.box_mesh(2, 2, 1, hi=(1.0, 0.6, 0.5), p=1, q=q)
    meshgen.random_materials(m, 3, 4)
    o1 = stdg.Oracle(m)
    mk = dict(m)
    mk["nk"] = np.full(m["hex"].shape[0], nk)
    ok = stdg.Oracle(mk)
    u0 = np.random.Generator(np.random.PCG64(5)).uniform(-1, 1, o1.ne * 6 * 8)
    dt, t0 = 0.3, 0.1
    u = u0
    for k in range(nk):
        u = o1.end_state(o1.slab_solve(u, t0 + k * dt / nk, dt / nk))
    uk = ok.end_state(ok.slab_solve(u0, t0, dt))
    assert np.abs(uk - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("uneven_q", [False, True])
def test_energy_identity_time_refinement(uneven_q):
    """Theorem 4.1 with local refinement in time: R(U) . pi U = E(t_n+1) - E(t_n) for any U."""
    m = meshgen.box_mesh(2, p=2, q=2)
    meshgen.random_nk(m, 7)
    if uneven_q:
        m["q"] = np.array([1, 2, 3, 1, 2, 3, 2, 1], dtype=np.uint8)
    assert len(set(m["nk"].tolist())) > 1
    meshgen.random_materials(m, 5, 6)
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) <= 1e-12 * max(1.0, abs(dE))


def test_planted_time_refinement_mistakes_fail_pins(monkeypatch):
    """With mixed N_K, dropping S_h or projecting onto the finer partition breaks the
    energy identity (Theorem 4.1)."""
    m = meshgen.box_mesh(2, p=1, q=2)
    m["nk"] = np.array([1, 2, 4, 2, 1, 4, 2, 1], dtype=np.uint8)
    meshgen.random_materials(m, 5, 6)
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) <= 1e-12 * max(1.0, abs(dE))
    orig = stdg.Oracle._common_test_factors
    monkeypatch.setattr(stdg.Oracle, "_common_test_factors", staticmethod(lambda *a: None))
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) > 1e-6

    def finer(q, nk, q2, nk2, tau, wt, Lt):
        return orig(q, nk, q2, nk2, tau, wt, Lt) if nk2 == nk else orig(q, nk, q2, max(nk, nk2), tau, wt, Lt)
    monkeypatch.setattr(stdg.Oracle, "_common_test_factors", staticmethod(finer))
    lhs, dE = _energy_identity(m)
    assert abs(lhs - dE) > 1e-6


def test_patch_time_refinement():
    """E = (0,0,x), H = (0,t,0), g = E with N_K in {1, 2, 4} and q >= 2: exact
    (the linear-in-t H lies in every common test space)."""
    m = meshgen.box_mesh(2, p=1, q=2)
    m["nk"] = np.array([1, 2, 4, 2, 1, 4, 2, 1], dtype=np.uint8)
    m["q"] = np.array([2, 2, 3, 2, 3, 2, 2, 3], dtype=np.uint8)
    o = stdg.Oracle(m)
    t0, dt = 0.3, 0.2
    Ef = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 0]], 1)
    Hf = lambda t: (lambda x: np.stack([0 * x[:, 0], t + 0 * x[:, 0], 0 * x[:, 0]], 1))
    u0 = o.project(Ef, Hf(t0))
    U = o.embed_start(u0)
    for e in range(o.ne):
        nk, q = int(o.nk[e]), int(o.q[e])
        blk = o.trial_block(U, e)
        for k in range(nk):
            uk = o.project(Ef, Hf(t0 + (k + 1) * dt / nk))
            n3 = 8
            off = int(sum(6 * n3 for _ in range(e)))
            blk[:, :, 1 + k * q, :] = uk[off:off + 6 * n3].reshape(2, 3, n3)

    def g(x, t):
        z = np.zeros(np.broadcast(x[..., 0], t).shape)
        return np.stack([z, z, x[..., 0] + z], -1)

    assert np.abs(o.residual(U, t0, dt, g=g)).max() < 1e-12
    Us = o.slab_solve(u0, t0, dt, g=g)
    assert np.abs(Us - U).max() < 1e-11


# --------------------------------------------------------------------------
# Sec. 6.1.2: manufactured solution with a current, local refinement in time
# --------------------------------------------------------------------------

def _mms_fields(x, t):
    """E = e^t x(x-1)z(1-z) e_y, H = e^t x(x-1)(1-2z) e_x - e^t (2x-1)z(1-z) e_z on the unit
    cube (eps = mu = 1): H solves mu dH/dt + curl E = 0, the current is J = dE/dt - curl H,
    and n x E = 0 on the whole boundary (PEC)."""
    X, Z = x[..., 0], x[..., 2]
    zero = np.zeros(np.broadcast(X, t).shape)
    et = np.exp(t)
    E = np.stack([zero, et * X * (X - 1) * Z * (1 - Z) + zero, zero], -1)
    H = np.stack([et * X * (X - 1) * (1 - 2 * Z) + zero, zero, -et * (2 * X - 1) * Z * (1 - Z) + zero], -1)
    J = np.stack([zero, et * (X * (X - 1) * Z * (1 - Z) + 2 * X * (X - 1) - 2 * Z * (1 - Z)) + zero, zero], -1)
    return E, H, J


@pytest.mark.parametrize("q", [1, 2])
def test_mms_nodal_superconvergence_time_refinement(q):
    """The fields are quadratic in x and z, so Q_2 in space represents them exactly and only
    the time discretisation errs: at the slab ends cG(q) converges with order 2q (the nodal
    superconvergence the paper reports in Sec. 6.1.2), here with N_K in {1, 2} mixed."""
    m = meshgen.box_mesh(2, p=2, q=q)
    m["nk"] = np.array([1, 2, 1, 2, 2, 1, 2, 1], dtype=np.uint8)
    o = stdg.Oracle(m)
    E0 = lambda x: _mms_fields(x, 0.0)[0]
    H0 = lambda x: _mms_fields(x, 0.0)[1]
    J = lambda x, t: _mms_fields(x, t)[2]
    T = 0.4
    ue = o.project(lambda x: _mms_fields(x, T)[0], lambda x: _mms_fields(x, T)[1])
    errs = []
    for ns in (2, 4):
        dt = T / ns
        A, _ = o.assemble(0.0, dt)
        zero = np.zeros(int(o.trial_off[-1]))
        u = o.project(E0, H0)
        for n in range(ns):
            b = -o.residual(zero, n * dt, dt, src=J)
            u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=(A, b)))
        errs.append(np.sqrt(2 * o.energy(u - ue)))
    order = np.log2(errs[0] / errs[1])
    assert abs(order - 2 * q) < 0.3, (errs, order)


@pytest.mark.parametrize("p,q", [(0, 1), (2, 2), (1, 3)])
def test_time_derivative_form_closed_form(p, q):
    """Eq. preconditioner on bricks: the spatial Legendre basis is orthonormal and DF is the
    constant diag(hx, hy, hz), so (eps d_t E, v) couples only equal spatial modes of one
    component, with weight eps G_c, G = (hy hz/hx, hx hz/hy, hx hy/hz) (Sec. 2.3).  In time,
    int_0^1 L_i l_m' is -delta_i0 for m = 0 and delta_{i,m-1} for m >= 1 (the derivative of
    the trial basis is the orthonormal Legendre basis of one degree less, Sec. 5.1).  So
    P(U)[f,c,i,s] = mat_f G_c (U[f,c,i+1,s] - delta_i0 U[f,c,0,s]) exactly."""
    m = meshgen.box_mesh(3, 2, 1, hi=(0.9, 0.5, 0.2), p=p, q=q)
    meshgen.random_materials(m, 71, 72)
    orc = stdg.Oracle(m)
    U = meshgen.random_coeffs(m, 73)
    dt = 0.037
    got = orc.time_derivative(U, dt)
    n3 = (p + 1) ** 3
    h = np.array([0.9 / 3, 0.5 / 2, 0.2 / 1])
    G = np.array([h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2]])
    want = []
    for e in range(orc.ne):
        u = U[e * 6 * (q + 1) * n3:(e + 1) * 6 * (q + 1) * n3].reshape(2, 3, q + 1, n3)
        mat = np.array([m["eps"][e], m["mu"][e]])
        r = u[:, :, 1:, :].copy()
        r[:, :, 0, :] -= u[:, :, 0, :]
        want.append((mat[:, None, None, None] * G[None, :, None, None] * r).ravel())
    want = np.concatenate(want)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def _time_derivative_pin_error(m, U, dt):
    """Largest deviation of Oracle.time_derivative from mat_f G_c (U_{i+1} - delta_i0 U_0)."""
    orc = stdg.Oracle(m)
    got = orc.time_derivative(U, dt)
    p, q = int(m["p"][0]), int(m["q"][0])
    n3 = (p + 1) ** 3
    lo, hi = np.min(m["vert"], axis=0), np.max(m["vert"], axis=0)
    ncell = np.array([len(np.unique(m["vert"][:, d])) - 1 for d in range(3)])
    h = (hi - lo) / ncell
    G = np.array([h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2]])
    want = []
    for e in range(orc.ne):
        u = U[e * 6 * (q + 1) * n3:(e + 1) * 6 * (q + 1) * n3].reshape(2, 3, q + 1, n3)
        mat = np.array([m["eps"][e], m["mu"][e]])
        r = u[:, :, 1:, :].copy()
        r[:, :, 0, :] -= u[:, :, 0, :]
        want.append((mat[:, None, None, None] * G[None, :, None, None] * r).ravel())
    want = np.concatenate(want)
    return np.max(np.abs(got - want)) / np.max(np.abs(want))


def test_planted_mistakes_fail_time_derivative_pin(monkeypatch):
    """The closed-form pin of Eq. preconditioner catches a dropped Jacobian, eps and mu
    swapped, and the derivative of the wrong trial functions."""
    m = meshgen.box_mesh(3, 2, 1, hi=(0.9, 0.5, 0.2), p=1, q=2)
    meshgen.random_materials(m, 81, 82)
    U = meshgen.random_coeffs(m, 83)
    dt = 0.05
    assert _time_derivative_pin_error(m, U, dt) < 1e-13

    # 1) eps and mu swapped in the form
    orig_init = stdg.Oracle.__init__

    def swapped(self, mesh, c_diss=0.0):
        orig_init(self, mesh, c_diss)
        self.eps, self.mu = self.mu, self.eps
    monkeypatch.setattr(stdg.Oracle, "__init__", swapped)
    assert _time_derivative_pin_error(m, U, dt) > 1e-3
    monkeypatch.setattr(stdg.Oracle, "__init__", orig_init)

    # 2) the measure J dropped from the projection weights
    orig_tp = stdg._test_project

    def no_measure(a, pts, Lt, wgt):
        return orig_tp(a, pts, Lt, wgt / pts.J[None, :])
    monkeypatch.setattr(stdg, "_test_project", no_measure)
    assert _time_derivative_pin_error(m, U, dt) > 1e-3
    monkeypatch.setattr(stdg, "_test_project", orig_tp)

    # 3) the time derivative taken of the test basis instead of the trial basis
    orig_trial = stdg.trial_time_nk

    def wrong_deriv(q, nk, tau, deriv=False):
        out = orig_trial(q, nk, tau, deriv)
        return out[::-1] if deriv else out
    monkeypatch.setattr(stdg, "trial_time_nk", wrong_deriv)
    assert _time_derivative_pin_error(m, U, dt) > 1e-3

