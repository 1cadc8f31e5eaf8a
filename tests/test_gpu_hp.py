"""Uneven spatial and temporal degrees per element (the hp batch form): CUDA
path vs the oracle.  Faces between elements of different degree use the
truncated / zero-padded orthonormal face modes and the projection onto the
common temporal test space of Eq. bilinearform:S (FP64 at 1e-12, FP32 at
2e-6, mixed-precision solves at 1e-9 relative L2)."""
import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


def hp_mesh(dims, seed, pmax=4, qmax=4, pmin=1):
    m = meshgen.box_mesh(*dims, hi=(1.0, 0.8, 0.6), p=1, q=1, order="morton")
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = m["hex"].shape[0]
    m["p"] = rng.integers(pmin, pmax + 1, ne).astype(np.uint8)
    m["q"] = rng.integers(1, qmax + 1, ne).astype(np.uint8)
    meshgen.random_materials(m, seed + 1, seed + 2)
    return m


@pytest.mark.parametrize("dims,seed,pmax,qmax", [((3, 3, 2), 1, 4, 4), ((4, 2, 2), 2, 7, 3), ((2, 2, 2), 3, 2, 6)])
def test_residual_hp_fp64(stm, dims, seed, pmax, qmax):
    m = hp_mesh(dims, seed, pmax, qmax)
    U = meshgen.random_coeffs(m, seed + 3)
    Ro = stdg.Oracle(m).residual(U, 0.0, 0.04)
    s = stm.Slab(m)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.0, 0.04)
    assert rel(R, Ro) < 1e-12


def test_residual_hp_fp32(stm):
    m = hp_mesh((3, 3, 2), 11)
    U32 = meshgen.random_coeffs(m, 12).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.04)
    s = stm.Slab(m)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U32, R, 0.0, 0.04, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


def test_projection_energy_hp(stm):
    m = hp_mesh((3, 2, 2), 21)
    o = stdg.Oracle(m)
    E0 = lambda x: np.stack([np.sin(2 * x[:, 1]), x[:, 0] * x[:, 2], np.cos(3 * x[:, 0])], 1)
    H0 = lambda x: np.stack([x[:, 2] ** 2, np.exp(x[:, 0]), 0 * x[:, 0] + 0.5], 1)
    uo = o.project(E0, H0)
    s = stm.Slab(m)
    s.set_initial(E0, H0)
    assert rel(s.get_state()[0], uo) < 1e-12
    assert abs(s.energy() - o.energy(uo)) < 1e-12 * o.energy(uo)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solve_hp(stm, precision):
    m = hp_mesh((3, 2, 2), 31, pmax=3, qmax=3)
    o = stdg.Oracle(m)
    n_state = int(np.sum(6 * (m["p"].astype(np.int64) + 1) ** 3))
    u0 = np.random.Generator(np.random.PCG64(32)).uniform(-1, 1, n_state)
    dt = 0.03
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=4000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], uo) < (1e-12 if precision == "fp64" else 1e-9)
