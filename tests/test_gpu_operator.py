"""The operator of the slab's GMRES iteration (stm_operator_apply) against the oracle.

For unknowns X (test layout: temporal modes 1..q) let U be X with slab-start mode 0 = 0
and no load.  Then A X is the oracle's residual of U (Eq. residual), and P X is the
oracle's preconditioner form of U (Eq. preconditioner, the time-derivative terms).  So
stm_operator_apply(P X, pre=1) = A P^{-1} P X must give A X, and stm_operator_apply(X,
pre=0) too.  On bricks (uniform and hp) and general affine elements P^{-1} is exact
(scalar, resp. constant 3x3, blocks per element, field and component).

Bars: FP64 1e-12 relative L2.  FP32 2e-6: V is rounded to float, which moves X by one
float rounding (6e-8 relative) through P^{-1}, and the FP32 arithmetic adds the same
few-dozen-term rounding as the FP32 residual tests.  The uniform-brick FP32 cases cover
the single-pass Krylov kernel (p = 4, 5 with q = 3; other degrees the generic single-pass
kernel), tiles of several elements and a Morton-ordered mesh whose face neighbours are not
at fixed index offsets.
"""
import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu

SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.9, -0.2], [0.15, 0.0, 1.1]])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


def _case(m, seed, dt):
    orc = stdg.Oracle(m)
    X = meshgen.random_coeffs(m, seed, kind="test")
    U = np.zeros(int(orc.trial_off[-1]))
    U[orc.unknown_mask()] = X
    return X, orc.time_derivative(U, dt), orc.residual(U, 0.0, dt)


BRICKS = [(3, 2, 2, 4, 3, "lex"), (2, 2, 2, 4, 3, "morton"), (2, 1, 2, 5, 3, "lex"), (2, 2, 2, 2, 2, "morton"),
          (1, 2, 1, 6, 3, "lex"), (2, 2, 1, 7, 2, "lex"), (3, 1, 1, 0, 1, "lex"), (2, 1, 1, 3, 6, "lex")]


@pytest.mark.parametrize("nx,ny,nz,p,q,order", BRICKS)
def test_operator_bricks(stm, nx, ny, nz, p, q, order):
    m = meshgen.box_mesh(nx, ny, nz, hi=(1.0, 0.7, 1.3), p=p, q=q, order=order)
    meshgen.random_materials(m, 31, 32)
    dt = 0.05
    X, V, AX = _case(m, 33, dt)
    s = stm.Slab(m)
    W = np.empty(s.n_test)
    s.operator_apply(V, W, dt, pre=True)
    assert rel(W, AX) < 1e-12
    s.operator_apply(X, W, dt, pre=False)
    assert rel(W, AX) < 1e-12
    W32 = np.empty(s.n_test, np.float32)
    s.operator_apply(V.astype(np.float32), W32, dt, pre=True, prec=stm.STM_FP32)
    assert rel(W32, AX) < 2e-6
    s.operator_apply(X.astype(np.float32), W32, dt, pre=False, prec=stm.STM_FP32)
    assert rel(W32, AX) < 2e-6


def test_operator_device_buffers(stm):
    """Device buffers (the path the solver takes), FP32, the Krylov kernel's degree."""
    import torch

    m = meshgen.box_mesh(4, 3, 2, p=4, q=3)
    meshgen.random_materials(m, 34, 35)
    dt = 0.04
    X, V, AX = _case(m, 36, dt)
    s = stm.Slab(m)
    Vd = torch.from_numpy(V.astype(np.float32)).cuda()
    Wd = torch.empty(s.n_test, dtype=torch.float32, device="cuda")
    s.operator_apply(Vd, Wd, dt, pre=True, prec=stm.STM_FP32)
    torch.cuda.synchronize()
    assert rel(Wd.cpu().numpy(), AX) < 2e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_hp(stm, prec):
    """Uneven (p, q) with 2:1 faces: every class kernel with P^{-1} on load."""
    m = meshgen.corner_octree_mesh(2, [0.8, 0.4])
    meshgen.random_hp(m, 37, p_range=(1, 5), q_range=(1, 4))
    dt = 0.03
    X, V, AX = _case(m, 38, dt)
    s = stm.Slab(m)
    if prec == "fp64":
        W = np.empty(s.n_test)
        s.operator_apply(V, W, dt, pre=True)
        assert rel(W, AX) < 1e-12
    else:
        W = np.empty(s.n_test, np.float32)
        s.operator_apply(V.astype(np.float32), W, dt, pre=True, prec=stm.STM_FP32)
        assert rel(W, AX) < 2e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_affine(stm, prec):
    """General affine elements: the 3x3 block inverse, then the metric-mass operator."""
    m = meshgen.box_mesh(2, 2, 1, p=3, q=2, affine=SHEAR)
    meshgen.random_materials(m, 39, 40)
    dt = 0.05
    X, V, AX = _case(m, 41, dt)
    s = stm.Slab(m)
    if prec == "fp64":
        W = np.empty(s.n_test)
        s.operator_apply(V, W, dt, pre=True)
        assert rel(W, AX) < 1e-12
    else:
        W = np.empty(s.n_test, np.float32)
        s.operator_apply(V.astype(np.float32), W, dt, pre=True, prec=stm.STM_FP32)
        assert rel(W, AX) < 2e-6


def test_operator_rejects_bad_arguments(stm):
    m = meshgen.box_mesh(1, p=1, q=1)
    s = stm.Slab(m)
    V = np.zeros(s.n_test)
    W = np.empty(s.n_test)
    lib = stm.lib()
    import ctypes as C

    pv, pw = V.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p)
    assert lib.stm_operator_apply(s.ctx, 0.0, pv, pw, 1, stm.STM_FP64, stm.STM_MEM_HOST) == stm.STM_EINVAL
    assert lib.stm_operator_apply(s.ctx, 0.1, pv, pw, 2, stm.STM_FP64, stm.STM_MEM_HOST) == stm.STM_EINVAL
    assert lib.stm_operator_apply(s.ctx, 0.1, pv, pw, 1, 7, stm.STM_MEM_HOST) == stm.STM_EINVAL
    assert lib.stm_operator_apply(s.ctx, 0.1, None, pw, 1, stm.STM_FP64, stm.STM_MEM_HOST) == stm.STM_EINVAL
