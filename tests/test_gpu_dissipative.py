"""Dissipative upwind variant D_h (Sec. 4.2) on the CUDA path vs the oracle.

Residual parity (FP64 1e-12, FP32 2e-6 relative, see test_gpu_parity.py for
the derivation of the bars), boundary data in the E - g term, slab solves,
and the dissipation identity: with J = 0 and PEC walls the energy never grows
and matches the oracle slab by slab.
"""
import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu

C = 0.8


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


CASES = [(2, 2, 2, 2, 2), (3, 2, 1, 1, 3), (2, 1, 2, 4, 3), (1, 2, 1, 7, 1), (2, 2, 1, 5, 4)]


@pytest.mark.parametrize("nx,ny,nz,p,q", CASES)
def test_residual_fp64(stm, nx, ny, nz, p, q):
    m = meshgen.box_mesh(nx, ny, nz, hi=(1.0, 0.7, 1.3), p=p, q=q, order="morton")
    meshgen.random_materials(m, 1, 2)
    U = meshgen.random_coeffs(m, 3)
    Ro = stdg.Oracle(m, c_diss=C).residual(U, 0.2, 0.05)
    s = stm.Slab(m, c_diss=C)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.2, 0.05)
    assert rel(R, Ro) < 1e-12
    # the term is really there: the non-dissipative residual differs
    assert rel(stdg.Oracle(m).residual(U, 0.2, 0.05), Ro) > 1e-3


@pytest.mark.parametrize("p,q", [(3, 2), (4, 3), (7, 1), (5, 4), (0, 2)])
def test_residual_fp32(stm, p, q):
    """Single-pass FP32 kernel with D_h for every size whose shared memory fits (all of these)."""
    m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.7, 1.3), p=p, q=q, order="morton")
    meshgen.random_materials(m, 1, 2)
    U = meshgen.random_coeffs(m, 3).astype(np.float32)
    Ro = stdg.Oracle(m, c_diss=C).residual(U.astype(np.float64), 0.2, 0.05)
    s = stm.Slab(m, c_diss=C)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U, R, 0.2, 0.05, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


def test_residual_uneven_p(stm):
    """Per-element spatial degrees (one q): the neighbour's face modes are truncated or padded."""
    m = meshgen.box_mesh(2, p=2, q=2)
    m["p"] = np.array([1, 2, 3, 1, 2, 3, 1, 2], dtype=np.uint8)
    meshgen.random_materials(m, 5, 6)
    U = meshgen.random_coeffs(m, 7)
    Ro = stdg.Oracle(m, c_diss=C).residual(U, 0.0, 0.1)
    s = stm.Slab(m, c_diss=C)
    for prec, dt_, bar in ((stm.STM_FP64, np.float64, 1e-12), (stm.STM_FP32, np.float32, 2e-6)):
        R = np.empty(s.n_test, dt_)
        s.residual_apply(U.astype(dt_), R, 0.0, 0.1, prec=prec)
        assert rel(R, Ro) < bar


def test_boundary_data(stm):
    """E = (0,0,x), H = (0,t,0), g = E stays exact with D_h (E - g = 0 on F_b, no jumps);
    the E - g term of random U matches the oracle."""
    m = meshgen.box_mesh(2, 2, 1, p=2, q=1)
    o = stdg.Oracle(m, c_diss=C)
    t0, dt = 0.3, 0.2
    Ef = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 0]], 1)
    u0 = o.project(Ef, lambda x: np.stack([0 * x[:, 0], t0 + 0 * x[:, 0], 0 * x[:, 0]], 1))
    u1 = o.project(Ef, lambda x: np.stack([0 * x[:, 0], t0 + dt + 0 * x[:, 0], 0 * x[:, 0]], 1))
    s = stm.Slab(m, tol=1e-14, max_it=2000, c_diss=C)
    s.set_boundary(lambda x, t: np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 0]], 1))
    s.set_state(u0, t=t0)
    rc, _ = s.slab_solve(dt)
    assert rc == stm.STM_OK
    assert np.abs(s.get_state()[0] - u1).max() < 1e-11
    meshgen.random_materials(m, 8, 9)
    o = stdg.Oracle(m, c_diss=C)
    s = stm.Slab(m, c_diss=C)
    # broadcasts for the oracle's x [1, A, 3], t [T, 1] and the library's x [n, 3], t [n]
    g = lambda x, t: np.stack(np.broadcast_arrays(np.sin(x[..., 1]) * (1 + t), x[..., 2] * x[..., 0] + 0 * t,
                                                  np.cos(x[..., 0] + t)), -1)
    s.set_boundary(g)
    U = meshgen.random_coeffs(m, 16)
    Ro = o.residual(U, t0, dt, g=g)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, t0, dt)
    assert rel(R, Ro) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solves_dissipate(stm, precision):
    """4^3 PEC cavity, random eps/mu, p = 2, q = 2, 10 slabs: GPU slab solves match the
    oracle's direct solves and the energy decreases every slab (Sec. 4.2 identity)."""
    m = meshgen.box_mesh(4, p=2, q=2)
    meshgen.random_materials(m, 11, 12)
    o = stdg.Oracle(m, c_diss=C)
    rng = np.random.Generator(np.random.PCG64(13))
    u = rng.uniform(-1, 1, o.ne * 6 * 27)
    dt = 0.05
    A_b = o.assemble(0.0, dt)
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=3000, c_diss=C)
    s.set_state(u)
    e_prev = s.energy()
    for n in range(10):
        u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=A_b))
        rc, rep = s.slab_solve(dt)
        assert rc == stm.STM_OK, rep
        assert rep["energy"] < e_prev
        e_prev = rep["energy"]
        assert abs(rep["energy"] - o.energy(u)) <= (1e-12 if precision == "fp64" else 1e-9) * o.energy(u)
    assert rel(s.get_state()[0], u) < (1e-12 if precision == "fp64" else 1e-9)


def test_unsupported_meshes(stm):
    for m in (meshgen.box_mesh(3, p=1, q=1, perturb=0.05),
              meshgen.corner_octree_mesh(2, [0.8], p=1, q=1)):
        with pytest.raises(stm.StmError):
            stm.Slab(m, c_diss=C)
    m = meshgen.box_mesh(2, p=1, q=1)
    m["q"] = np.array([1, 2, 1, 2, 1, 2, 1, 2], dtype=np.uint8)
    with pytest.raises(stm.StmError):
        stm.Slab(m, c_diss=C)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_with_dissipation(stm, prec):
    """The GMRES operator A P^{-1} with D_h in A (P of Eq. preconditioner has no D_h term)."""
    m = meshgen.box_mesh(3, 2, 2, p=4, q=3, order="morton")
    meshgen.random_materials(m, 5, 6)
    dt = 0.05
    orc = stdg.Oracle(m, c_diss=C)
    X = meshgen.random_coeffs(m, 7, kind="test")
    U = np.zeros(int(orc.trial_off[-1]))
    U[orc.unknown_mask()] = X
    V, AX = orc.time_derivative(U, dt), orc.residual(U, 0.0, dt)
    s = stm.Slab(m, c_diss=C)
    if prec == "fp64":
        W = np.empty(s.n_test)
        s.operator_apply(V, W, dt, pre=True)
        assert rel(W, AX) < 1e-12
    else:
        W = np.empty(s.n_test, np.float32)
        s.operator_apply(V.astype(np.float32), W, dt, pre=True, prec=stm.STM_FP32)
        assert rel(W, AX) < 2e-6
