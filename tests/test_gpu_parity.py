"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: FP64 results are held to 1e-12 relative L2 (the target for the
double-precision path).  FP32 residuals: inputs are rounded to float first
(the oracle sees the same rounded values), and the bar is 2e-6 relative L2 --
each residual entry sums at most a few dozen products of O(1) terms, so
float rounding (u = 6e-8) with this amplification stays below 1e-6.
"""
import math

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


CASES = [
    (2, 2, 2, 1, 1), (3, 2, 2, 2, 2), (2, 2, 3, 3, 3), (2, 2, 2, 4, 4), (3, 1, 1, 0, 1),
    (2, 2, 2, 5, 2), (1, 1, 2, 7, 1), (2, 1, 2, 6, 3), (5, 3, 2, 2, 1), (2, 2, 2, 4, 3),
    (2, 1, 1, 2, 5), (1, 1, 2, 3, 6),
]


@pytest.mark.parametrize("nx,ny,nz,p,q", CASES)
def test_residual_fp64(stm, nx, ny, nz, p, q):
    m = meshgen.box_mesh(nx, ny, nz, hi=(1.0, 0.7, 1.3), p=p, q=q, order="morton")
    meshgen.random_materials(m, 1, 2)
    U = meshgen.random_coeffs(m, 3)
    Ro = stdg.Oracle(m).residual(U, 0.2, 0.05)
    s = stm.Slab(m)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.2, 0.05)
    assert rel(R, Ro) < 1e-12


@pytest.mark.parametrize("nx,ny,nz,p,q", [(2, 2, 2, 2, 2), (3, 2, 2, 4, 3), (1, 2, 1, 7, 4)])
def test_residual_fp32(stm, nx, ny, nz, p, q):
    m = meshgen.box_mesh(nx, ny, nz, hi=(1.0, 0.7, 1.3), p=p, q=q)
    meshgen.random_materials(m, 4, 5)
    U32 = meshgen.random_coeffs(m, 6).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.03)
    s = stm.Slab(m)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U32, R, 0.0, 0.03, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


def test_residual_device_memory(stm):
    import torch

    m = meshgen.box_mesh(3, 3, 2, p=3, q=2, order="morton")
    meshgen.random_materials(m, 7, 8)
    U = meshgen.random_coeffs(m, 9)
    s = stm.Slab(m)
    Rh = np.empty(s.n_test)
    s.residual_apply(U, Rh, 0.0, 0.1)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
    s.residual_apply(Ud, Rd, 0.0, 0.1)
    torch.cuda.synchronize()
    assert np.array_equal(Rd.cpu().numpy(), Rh)  # same kernels, same order: bitwise


@pytest.mark.parametrize("offset", [0, 1])
def test_state_transfer_page_locked(stm, offset):
    """stm_set_state / stm_get_state with page-locked host buffers (the kernel transfer; offset 1
    misaligns the buffers by 8 bytes, the scalar variant), pageable numpy arrays (the copy
    engines) and device memory all move the state bit for bit."""
    import torch

    m = meshgen.box_mesh(3, 2, 2, p=3, q=2, order="morton")
    s = stm.Slab(m)
    n = s.n_state
    u = np.random.Generator(np.random.PCG64(41)).uniform(-1, 1, n)
    hin, hout = stm.HostBuffer(n + 1), stm.HostBuffer(n + 1)
    a_in, a_out = hin.array[offset:offset + n], hout.array[offset:offset + n]
    a_in[:] = u
    a_out[:] = 0.0
    s.set_state(a_in, t=0.25)
    back, t = s.get_state(a_out)
    assert t == 0.25 and np.array_equal(a_out, u)
    plain, _ = s.get_state(np.empty(n))
    assert np.array_equal(plain, u)
    ud = torch.empty(n, dtype=torch.float64, device="cuda")
    s.get_state(ud)
    torch.cuda.synchronize()
    assert np.array_equal(ud.cpu().numpy(), u)
    s.set_state(np.ascontiguousarray(u[::-1]))
    s.get_state(a_out)
    assert np.array_equal(a_out, u[::-1])
    hin.close()
    hout.close()


def test_energy_and_projection(stm):
    m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.5, 0.8), p=3, q=1)
    meshgen.random_materials(m, 1, 9)
    o = stdg.Oracle(m)
    E0 = lambda x: np.stack([np.sin(x[:, 1]), x[:, 0] * x[:, 2], np.cos(3 * x[:, 0])], 1)
    H0 = lambda x: np.stack([x[:, 2] ** 2, np.exp(x[:, 0]), 0 * x[:, 0] + 0.5], 1)
    uo = o.project(E0, H0)
    s = stm.Slab(m)
    s.set_initial(E0, H0)
    ug, _ = s.get_state()
    assert rel(ug, uo) < 1e-12
    assert abs(s.energy() - o.energy(uo)) < 1e-12 * o.energy(uo)


def _cavity(x, t=0.0):
    z = np.zeros(x.shape[0])
    return np.stack([z, z, np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.cos(math.sqrt(2) * math.pi * t)], 1)


def test_slab_solve_plain_config(stm):
    """4^3 PEC cavity, p = 2, q = 1, 20 slabs of 0.05: GPU GMRES vs the oracle's direct solves."""
    m = meshgen.box_mesh(4, p=2, q=1)
    o = stdg.Oracle(m)
    dt = 0.05
    u = o.project(_cavity, None)
    A_b = o.assemble(0.0, dt)
    s = stm.Slab(m, tol=1e-14, restart=10, max_it=2000)
    s.set_initial(_cavity, None)
    for n in range(20):
        u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=A_b))
        rc, rep = s.slab_solve(dt)
        assert rc == stm.STM_OK, rep
    ug, t = s.get_state()
    assert abs(t - 1.0) < 1e-12
    assert rel(ug, u) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solve_one_graph_launch(stm, precision):
    """The plain configuration (4^3 PEC cavity, p = 2, q = 1) with the whole slab solve captured
    as one CUDA graph of 16 restart cycles (cycles after the stop test are skipped on the
    device; one host read per slab): the same result as cycle-by-cycle launches and the
    oracle's direct solves."""
    m = meshgen.box_mesh(4, p=2, q=1)
    o = stdg.Oracle(m)
    dt = 0.05
    u = o.project(_cavity, None)
    A_b = o.assemble(0.0, dt)
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    tol = 1e-14 if precision == "fp64" else 1e-11
    s1 = stm.Slab(m, precision=prec, tol=tol, restart=10, max_it=2000, cycles_per_launch=16)
    s2 = stm.Slab(m, precision=prec, tol=tol, restart=10, max_it=2000)
    s1.set_initial(_cavity, None)
    s2.set_initial(_cavity, None)
    for n in range(5):
        u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=A_b))
        rc1, rep1 = s1.slab_solve(dt)
        rc2, rep2 = s2.slab_solve(dt)
        assert rc1 == stm.STM_OK and rc2 == stm.STM_OK, (rep1, rep2)
        assert rep1["restarts"] < 16 and rep1["iterations"] == rep2["iterations"]
    u1, u2 = s1.get_state()[0], s2.get_state()[0]
    assert np.array_equal(u1, u2)
    assert rel(u1, u) < (1e-12 if precision == "fp64" else 1e-9)


@pytest.mark.parametrize("q", [2, 3])
def test_slab_solve_higher_q(stm, q):
    m = meshgen.box_mesh(2, 3, 2, hi=(0.5, 0.75, 0.5), p=2, q=q)
    meshgen.random_materials(m, 2, 3)
    o = stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(5))
    u0 = rng.uniform(-1, 1, o.ne * 6 * 27)
    dt = 0.04
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    s = stm.Slab(m, tol=1e-14, max_it=2000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    ug, _ = s.get_state()
    assert rel(ug, uo) < 1e-12


def test_energy_conserved_100_slabs(stm):
    """PEC cavity, random piecewise eps/mu, J = 0: energy constant to 1e-12 relative over 100 slabs."""
    m = meshgen.box_mesh(4, p=3, q=2)
    meshgen.random_materials(m, 11, 12)
    s = stm.Slab(m, tol=1e-15, max_it=5000)
    rng = np.random.Generator(np.random.PCG64(13))
    s.set_state(rng.uniform(-1, 1, s.n_state))
    e0 = s.energy()
    drift = 0.0
    for _ in range(100):
        s.slab_solve(0.02)
        drift = max(drift, abs(s.energy() - e0) / e0)
    assert drift < 1e-12


@pytest.mark.parametrize("reorth", [True, False])
def test_slab_solve_mixed_precision(stm, reorth):
    """FP32 inner GMRES + FP64 refinement: slab solution within 1e-9 of the oracle's direct solve."""
    m = meshgen.box_mesh(3, 3, 2, hi=(0.75, 0.75, 0.5), p=3, q=2, order="morton")
    meshgen.random_materials(m, 6, 7)
    o = stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(8))
    u0 = rng.uniform(-1, 1, o.ne * 6 * 64)
    dt = 0.25 / 7
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    s = stm.Slab(m, precision=stm.STM_MIXED, tol=1e-11, max_it=3000, reorth=reorth)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    ug, _ = s.get_state()
    assert rel(ug, uo) < 1e-9
    s64 = stm.Slab(m, tol=1e-11, max_it=3000, reorth=reorth)
    s64.set_state(u0)
    rc, rep64 = s64.slab_solve(dt)
    assert rc == stm.STM_OK
    assert rel(s64.get_state()[0], uo) < 1e-9


def test_headline_full_size_sampled(stm):
    """The bench workload in the launch configuration the bench times: 64^3 bricks in Morton
    order, p = 4, q = 3, eps/mu ~ U[1,4] (PCG64 1307/1308), coefficients ~ U[-1,1] (1309).
    FP64 residual, FP32 residual (single-pass kernel), and the GMRES operator A P^{-1} in FP64
    and FP32 (the mixed solve's Krylov kernel), each checked against the oracle on sampled
    elements (corners, faces and random interior ones) with their face neighbours.  For the
    operator, V = P X with P from its closed form on bricks (mat_f G_c, pinned against the
    oracle's time-derivative form), so the expected value is the oracle's residual of X."""
    import torch

    n, p, q = 64, 4, 3
    m = meshgen.box_mesh(n, p=p, q=q, order="morton")
    meshgen.random_materials(m, 1307, 1308)
    ne, n3 = m["hex"].shape[0], (p + 1) ** 3
    tper, per = 6 * (q + 1) * n3, 6 * q * n3
    dt = (1.0 / n) / (2 * p + 1)
    rng = np.random.Generator(np.random.PCG64(1311))
    sample = sorted(set([0, ne - 1, int(np.argmax(m["vert"][m["hex"][:, 7]].sum(1)))] +
                        [int(x) for x in rng.integers(0, ne, 9)]))
    keep = set(sample)
    for e in sample:
        keep |= {int(x) for x in m["nbr"][e] if x >= 0}
    keep = np.array(sorted(keep))
    sub = {k: m[k][keep] for k in ("hex", "p", "q", "eps", "mu")}
    sub.update(vert=m["vert"], geometry=m["geometry"])
    loc = {int(e): i for i, e in enumerate(keep)}
    o = stdg.Oracle(sub)
    s = stm.Slab(m)

    def check(Rdev, Ublocks, bar):
        Rs = Rdev.view(ne, per)[torch.tensor(sample, device=Rdev.device)].double().cpu().numpy()
        for k, e in enumerate(sample):
            Ro = o.element_residual(loc[e], Ublocks, 0.0, dt)[0].ravel()
            assert rel(Rs[k], Ro) < bar, (e, rel(Rs[k], Ro))

    U = meshgen.random_coeffs(m, 1309)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
    s.residual_apply(Ud, Rd, 0.0, dt)
    check(Rd, np.concatenate([U[e * tper:(e + 1) * tper] for e in keep]), 1e-12)
    U32 = Ud.float()
    R32 = torch.empty(s.n_test, dtype=torch.float32, device="cuda")
    s.residual_apply(U32, R32, 0.0, dt, prec=stm.STM_FP32)
    U32h = U32.view(ne, tper)[torch.from_numpy(keep).cuda()].double().cpu().numpy().ravel()
    check(R32, U32h, 2e-6)
    del Ud, U32, Rd, R32, U

    # the operator: X unknowns (test layout), V = P X = mat_f G_c X, G_c = h on cubes of edge h
    X = torch.from_numpy(meshgen.random_coeffs(m, 1310, kind="test")).cuda()
    mats = torch.from_numpy(np.stack([m["eps"], m["mu"]], 1) / n).cuda()
    V = (X.view(ne, 2, 3 * q * n3) * mats[:, :, None]).reshape(-1)
    Xk = X.view(ne, per)[torch.from_numpy(keep).cuda()].cpu().numpy()
    Ux = np.zeros((len(keep), 2, 3, q + 1, n3))
    Ux[:, :, :, 1:, :] = Xk.reshape(len(keep), 2, 3, q, n3)
    W = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
    s.operator_apply(V, W, dt, pre=True)
    check(W, Ux.ravel(), 1e-12)
    W32 = torch.empty(s.n_test, dtype=torch.float32, device="cuda")
    s.operator_apply(V.float(), W32, dt, pre=True, prec=stm.STM_FP32)
    check(W32, Ux.ravel(), 2e-6)
    # hand the ~35 GB of full-size buffers back to the device for the tests that follow
    s.close()
    del X, V, W, W32
    torch.cuda.empty_cache()
