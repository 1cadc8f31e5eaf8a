"""General affine elements (parallelepipeds, STM_GEOM_AFFINE): the constant 3x3
metric mass of Sec. 5.2 ("mass residual") inside the residual kernels, the
3x3 block preconditioner, projection and energy -- CUDA path vs the CPU
oracle through the C ABI (FP64 at 1e-12, FP32 at 2e-6, mixed solve at 1e-9)."""
import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu

SHEAR = [[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.2, 1.1]]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


def mesh(dims, p, q, seed=1):
    m = meshgen.box_mesh(*dims, hi=(1.0, 0.8, 0.6), p=p, q=q, order="morton", affine=SHEAR)
    meshgen.random_materials(m, seed, seed + 1)
    return m


@pytest.mark.parametrize("p,q,dims", [(2, 2, (3, 2, 2)), (3, 1, (2, 2, 2)), (1, 3, (3, 3, 2)), (4, 3, (2, 2, 1))])
def test_residual_affine_fp64(stm, p, q, dims):
    m = mesh(dims, p, q)
    U = meshgen.random_coeffs(m, 3)
    Ro = stdg.Oracle(m).residual(U, 0.0, 0.07)
    s = stm.Slab(m)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.0, 0.07)
    assert rel(R, Ro) < 1e-12


def test_residual_affine_fp32(stm):
    m = mesh((3, 2, 2), 3, 2, seed=4)
    U32 = meshgen.random_coeffs(m, 6).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.05)
    s = stm.Slab(m)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U32, R, 0.0, 0.05, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


def test_energy_and_projection_affine(stm):
    m = mesh((3, 2, 2), 3, 1, seed=7)
    o = stdg.Oracle(m)
    E0 = lambda x: np.stack([np.sin(3 * x[:, 0]) * x[:, 1], np.cos(2 * x[:, 2]) + x[:, 0], x[:, 0] * x[:, 2]], 1)
    H0 = lambda x: np.stack([x[:, 2] ** 2, np.sin(x[:, 0] + x[:, 1]), np.exp(-x[:, 1])], 1)
    uo = o.project(E0, H0)
    s = stm.Slab(m)
    s.set_initial(E0, H0)
    assert rel(s.get_state()[0], uo) < 1e-12
    u = np.random.Generator(np.random.PCG64(9)).uniform(-1, 1, s.n_state)
    s.set_state(u)
    assert abs(s.energy() - o.energy(u)) < 1e-12 * o.energy(u)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solve_affine(stm, precision):
    m = mesh((2, 2, 2), 2, 2, seed=10)
    o = stdg.Oracle(m)
    u0 = np.random.Generator(np.random.PCG64(12)).uniform(-1, 1, o.ne * 6 * 27)
    dt = 0.05
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=4000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], uo) < (1e-12 if precision == "fp64" else 1e-9)


def test_gauss_source_affine(stm):
    m = mesh((3, 3, 2), 3, 2, seed=13)
    U = meshgen.random_coeffs(m, 15)
    src = [dict(centre=(0.5, 0.45, 0.35), dir=(0.0, 0.6, 0.8), sigma_x=0.15, t0=0.1, sigma_t=0.05, amp=2.0)]

    def J(x, t):
        r2 = np.sum((x - np.asarray(src[0]["centre"])) ** 2, axis=-1)
        a = 2.0 * np.exp(-r2 / (2 * 0.15 ** 2)) * np.exp(-(t - 0.1) ** 2 / (2 * 0.05 ** 2))
        return a[..., None] * np.asarray(src[0]["dir"])

    Ro = stdg.Oracle(m).residual(U, 0.05, 0.06, src=J)
    s = stm.Slab(m)
    s.set_source_gauss(src)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.05, 0.06)
    assert rel(R, Ro) < 1e-12


def test_affine_refuses(stm):
    m = mesh((2, 2, 2), 2, 2)
    m["vert"] = m["vert"] + 0.01 * np.sin(7 * m["vert"])  # no longer parallelepipeds
    with pytest.raises(stm.StmError) as ex:
        stm.Slab(m)
    assert ex.value.code == stm.STM_EUNSUPPORTED
    m = mesh((2, 2, 2), 2, 2)
    m["p"] = np.array([1, 2, 1, 2, 1, 2, 1, 2], dtype=np.uint8)
    with pytest.raises(stm.StmError) as ex:
        stm.Slab(m)
    assert ex.value.code == stm.STM_EUNSUPPORTED
