"""Local refinement in time (N_K sub-intervals per element, Sec. 2.2 / 4.1) on the
CUDA path vs the oracle.

Neighbours with different partitions couple through the projection onto the
largest common temporal test space (Eq. bilinearform:S), applied in the
kernels as temporal transfer matrices between nested sub-intervals.  Bars as
in test_gpu_parity.py: FP64 1e-12, FP32 2e-6 relative.
"""
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


def _mesh(case):
    if case == "nk_mixed":
        m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.7, 1.3), p=2, q=2, order="morton")
        meshgen.random_nk(m, 21, (1, 2, 4))
    elif case == "nk_q_mixed":
        m = meshgen.box_mesh(2, 2, 2, p=2, q=2)
        m["nk"] = np.array([1, 2, 4, 8, 2, 1, 4, 2], dtype=np.uint8)
        m["q"] = np.array([2, 3, 1, 2, 4, 2, 3, 1], dtype=np.uint8)
    elif case == "nk_p_mixed":
        m = meshgen.box_mesh(2, 2, 2, p=2, q=2)
        m["nk"] = np.array([2, 1, 4, 2, 1, 8, 2, 4], dtype=np.uint8)
        m["p"] = np.array([1, 3, 2, 2, 3, 1, 2, 4], dtype=np.uint8)
    else:  # uniform N_K = 2
        m = meshgen.box_mesh(3, 2, 2, p=3, q=2)
        m["nk"] = np.full(12, 2, dtype=np.uint8)
    meshgen.random_materials(m, 22, 23)
    return m


@pytest.mark.parametrize("case", ["nk_mixed", "nk_q_mixed", "nk_p_mixed", "nk_uniform"])
def test_residual(stm, case):
    m = _mesh(case)
    U = meshgen.random_coeffs(m, 24)
    Ro = stdg.Oracle(m).residual(U, 0.1, 0.07)
    s = stm.Slab(m)
    assert s.n_test == Ro.size
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.1, 0.07)
    assert rel(R, Ro) < 1e-12
    R32 = np.empty(s.n_test, np.float32)
    s.residual_apply(U.astype(np.float32), R32, 0.1, 0.07, prec=stm.STM_FP32)
    assert rel(R32, stdg.Oracle(m).residual(U.astype(np.float32).astype(np.float64), 0.1, 0.07)) < 2e-6


def test_uniform_refinement_is_substepping(stm):
    """N_K = 4 everywhere: one slab equals four slabs of dt / 4 on the same library."""
    m = meshgen.box_mesh(3, 2, 2, p=2, q=2)
    meshgen.random_materials(m, 1, 2)
    m4 = dict(m)
    m4["nk"] = np.full(12, 4, dtype=np.uint8)
    u0 = np.random.Generator(np.random.PCG64(3)).uniform(-1, 1, 12 * 6 * 27)
    dt = 0.08
    s1, s4 = stm.Slab(m, tol=1e-14, max_it=3000), stm.Slab(m4, tol=1e-14, max_it=3000)
    s1.set_state(u0)
    s4.set_state(u0)
    for _ in range(4):
        assert s1.slab_solve(dt / 4)[0] == stm.STM_OK
    assert s4.slab_solve(dt)[0] == stm.STM_OK
    assert rel(s4.get_state()[0], s1.get_state()[0]) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solves_vs_oracle(stm, precision):
    """Mixed N_K and q, random eps/mu, 8 slabs: the oracle's direct solves, and the
    discrete energy stays constant (Theorem 4.1, J = 0, PEC)."""
    m = _mesh("nk_q_mixed")
    o = stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(25))
    u = rng.uniform(-1, 1, o.ne * 6 * 27)
    dt = 0.06
    A_b = o.assemble(0.0, dt)
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=4000)
    s.set_state(u)
    e0 = s.energy()
    for n in range(8):
        u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=A_b))
        rc, rep = s.slab_solve(dt)
        assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], u) < (1e-12 if precision == "fp64" else 1e-9)
    assert abs(s.energy() - e0) <= (1e-12 if precision == "fp64" else 1e-8) * e0


def test_unsupported(stm):
    m = meshgen.corner_octree_mesh(2, [0.8], p=1, q=1)
    m["nk"] = np.full(m["hex"].shape[0], 2, dtype=np.uint8)
    with pytest.raises(stm.StmError):
        stm.Slab(m)
    m = meshgen.box_mesh(2, p=1, q=1)
    m["nk"] = np.full(8, 2, dtype=np.uint8)
    with pytest.raises(stm.StmError):
        stm.Slab(m, c_diss=0.5)
    m["nk"] = np.full(8, 3, dtype=np.uint8)
    with pytest.raises(stm.StmError):
        stm.Slab(m)


def _mms(x, t):
    """Manufactured solution of Sec. 6.1.2 (unit cube, eps = mu = 1, PEC): E, H and J."""
    X, Z = x[..., 0], x[..., 2]
    zero = np.zeros(np.broadcast(X, t).shape)
    et = np.exp(t)
    E = np.stack([zero, et * X * (X - 1) * Z * (1 - Z) + zero, zero], -1)
    H = np.stack([et * X * (X - 1) * (1 - 2 * Z) + zero, zero, -et * (2 * X - 1) * Z * (1 - Z) + zero], -1)
    J = np.stack([zero, et * (X * (X - 1) * Z * (1 - Z) + 2 * X * (X - 1) - 2 * Z * (1 - Z)) + zero, zero], -1)
    return E, H, J


def test_host_current_time_refined(stm):
    """stm_set_source on a mesh with mixed N_K and q: the load uses each element's
    sub-intervals; residual vs the oracle's (J, v)."""
    m = _mesh("nk_q_mixed")
    J = lambda x, t: _mms(x, t)[2] + np.stack(np.broadcast_arrays(0 * x[..., 0], np.sin(x[..., 0] + 3 * t), 0 * t), -1)
    U = meshgen.random_coeffs(m, 27)
    s = stm.Slab(m)
    s.set_source(J)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.1, 0.07)
    assert rel(R, stdg.Oracle(m).residual(U, 0.1, 0.07, src=J)) < 1e-12


@pytest.mark.parametrize("q", [1, 2])
def test_mms_nodal_order_time_refined(stm, q):
    """Sec. 6.1.2 on the CUDA path: Q_2 in space is exact for the fields, N_K in {1, 2}
    mixed; the slab-end error converges with order 2q."""
    m = meshgen.box_mesh(2, p=2, q=q)
    m["nk"] = np.array([1, 2, 1, 2, 2, 1, 2, 1], dtype=np.uint8)
    o = stdg.Oracle(m)
    T = 0.4
    ue = o.project(lambda x: _mms(x, T)[0], lambda x: _mms(x, T)[1])
    errs = []
    for ns in (2, 4):
        s = stm.Slab(m, tol=1e-13, max_it=3000)
        s.set_source(lambda x, t: _mms(x, t)[2])
        s.set_initial(lambda x: _mms(x, 0.0)[0], lambda x: _mms(x, 0.0)[1])
        for _ in range(ns):
            rc, rep = s.slab_solve(T / ns)
            assert rc == stm.STM_OK, rep
        u, t = s.get_state()
        assert abs(t - T) < 1e-12
        errs.append(np.sqrt(2 * o.energy(u - ue)))
    order = np.log2(errs[0] / errs[1])
    assert abs(order - 2 * q) < 0.3, (errs, order)


@pytest.mark.parametrize("case", ["nk_q_mixed", "nk_p_mixed"])
def test_sources_and_boundary_data_uneven(stm, case):
    """Gaussian pulses and boundary data g on meshes with uneven degrees and N_K: the pulses
    projected on the device per (p, q, N_K) class and sub-interval, g sampled and projected
    on the host per element; residual vs the oracle's."""
    m = _mesh(case)
    srcs = [dict(centre=(0.5, 0.45, 0.55), dir=(0.0, 0.0, 1.0), sigma_x=0.15, t0=0.1, sigma_t=0.05, amp=1.0),
            dict(centre=(0.3, 0.6, 0.4), dir=(0.6, 0.0, 0.8), sigma_x=0.1, t0=0.12, sigma_t=0.08, amp=2.5)]

    def J(x, t):
        out = 0.0
        for sd in srcs:
            r2 = np.sum((x - np.asarray(sd["centre"])) ** 2, axis=-1)
            a = sd["amp"] * np.exp(-r2 / (2 * sd["sigma_x"] ** 2)) * np.exp(-(t - sd["t0"]) ** 2 / (2 * sd["sigma_t"] ** 2))
            out = out + a[..., None] * np.asarray(sd["dir"])
        return out

    g = lambda x, t: np.stack(np.broadcast_arrays(np.sin(x[..., 1]) * (1 + t), x[..., 2] * x[..., 0] + 0 * t,
                                                  np.cos(x[..., 0] + t)), -1)
    U = meshgen.random_coeffs(m, 29)
    s = stm.Slab(m)
    s.set_source_gauss(srcs)
    s.set_boundary(g)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.05, 0.06)
    assert rel(R, stdg.Oracle(m).residual(U, 0.05, 0.06, src=J, g=g)) < 1e-12
