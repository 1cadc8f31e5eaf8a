"""Curved (trilinear) elements, Gaussian current sources and boundary data:
CUDA path vs the CPU oracle through the C ABI (FP64 at 1e-12, FP32 at 2e-6
relative L2, as in test_gpu_parity)."""
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


def gauss_sources():
    return [dict(centre=(0.5, 0.45, 0.55), dir=(0.0, 0.0, 1.0), sigma_x=0.15, t0=0.1, sigma_t=0.05, amp=1.0),
            dict(centre=(0.3, 0.6, 0.4), dir=(0.6, 0.0, 0.8), sigma_x=0.1, t0=0.12, sigma_t=0.08, amp=2.5)]


def oracle_J(sources):
    def J(x, t):
        out = 0.0
        for sd in sources:
            r2 = np.sum((x - np.asarray(sd["centre"])) ** 2, axis=-1)
            a = sd["amp"] * np.exp(-r2 / (2 * sd["sigma_x"] ** 2)) * np.exp(-(t - sd["t0"]) ** 2 / (2 * sd["sigma_t"] ** 2))
            out = out + a[..., None] * np.asarray(sd["dir"])
        return out
    return J


@pytest.mark.parametrize("p,q,dims", [(2, 2, (3, 2, 2)), (3, 1, (2, 2, 2)), (1, 3, (3, 3, 2)), (5, 4, (2, 1, 1))])
def test_residual_curved_fp64(stm, p, q, dims):
    m = meshgen.box_mesh(*dims, p=p, q=q, perturb=0.4, order="morton")
    meshgen.random_materials(m, 1, 2)
    U = meshgen.random_coeffs(m, 3)
    Ro = stdg.Oracle(m).residual(U, 0.0, 0.07)
    s = stm.Slab(m)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.0, 0.07)
    assert rel(R, Ro) < 1e-12


def test_residual_curved_fp32(stm):
    m = meshgen.box_mesh(3, 2, 2, p=3, q=2, perturb=0.4)
    meshgen.random_materials(m, 4, 5)
    U32 = meshgen.random_coeffs(m, 6).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.05)
    s = stm.Slab(m)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U32, R, 0.0, 0.05, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


@pytest.mark.parametrize("p,q,dims", [(3, 2, (3, 2, 2)), (4, 1, (2, 2, 1)), (5, 4, (2, 1, 1)), (6, 3, (2, 1, 1)),
                                      (7, 6, (2, 1, 1))])
def test_residual_curved_fp32_tensor_cores(stm, p, q, dims):
    """FP32 curved mass on the tensor cores (tcgen05, 3xTF32) against the oracle and against
    the CUDA-core FP32 kernel, both at FP32 accuracy."""
    m = meshgen.box_mesh(*dims, p=p, q=q, perturb=0.4, order="morton")
    meshgen.random_materials(m, 4, 5)
    U32 = meshgen.random_coeffs(m, 6).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.05)
    out = {}
    for tc in (True, False):
        s = stm.Slab(m, tensor_cores=tc)
        R = np.empty(s.n_test, np.float32)
        s.residual_apply(U32, R, 0.0, 0.05, prec=stm.STM_FP32)
        out[tc] = R
        s.close()
    assert rel(out[True], Ro) < 2e-6
    assert rel(out[True], out[False]) < 2e-6


def test_slab_solve_curved_mixed_tensor_cores(stm):
    """Mixed-precision slab solve on trilinear hexes with p = 3 (FP32 inner mass on the tensor
    cores) against the oracle's direct solve at 1e-9."""
    m = meshgen.box_mesh(2, 2, 2, hi=(0.5, 0.5, 0.5), p=3, q=2, perturb=0.3)
    meshgen.random_materials(m, 16, 17)
    o = stdg.Oracle(m)
    u0 = np.random.Generator(np.random.PCG64(18)).uniform(-1, 1, o.ne * 6 * 64)
    dt = 0.25 / 7
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    s = stm.Slab(m, precision=stm.STM_MIXED, tol=1e-11, max_it=4000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], uo) < 1e-9


def test_energy_curved(stm):
    m = meshgen.box_mesh(3, 2, 2, p=3, q=1, perturb=0.4)
    meshgen.random_materials(m, 7, 8)
    o = stdg.Oracle(m)
    u = np.random.Generator(np.random.PCG64(9)).uniform(-1, 1, o.ne * 6 * 64)
    s = stm.Slab(m)
    s.set_state(u)
    assert abs(s.energy() - o.energy(u)) < 1e-12 * o.energy(u)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solve_curved(stm, precision):
    m = meshgen.box_mesh(2, 2, 2, hi=(0.5, 0.5, 0.5), p=2, q=2, perturb=0.3)
    meshgen.random_materials(m, 10, 11)
    o = stdg.Oracle(m)
    u0 = np.random.Generator(np.random.PCG64(12)).uniform(-1, 1, o.ne * 6 * 27)
    dt = 0.25 / 5
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=4000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], uo) < (1e-12 if precision == "fp64" else 1e-9)


@pytest.mark.parametrize("curved", [False, True])
def test_gauss_source(stm, curved):
    m = meshgen.box_mesh(3, 3, 2, p=3, q=2, perturb=0.3 if curved else 0.0)
    meshgen.random_materials(m, 13, 14)
    U = meshgen.random_coeffs(m, 15)
    src = gauss_sources()
    Ro = stdg.Oracle(m).residual(U, 0.05, 0.06, src=oracle_J(src))
    s = stm.Slab(m)
    s.set_source_gauss(src)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.05, 0.06)
    assert rel(R, Ro) < 1e-12
    # the source contribution alone (R with J minus R without) against the oracle's
    s.set_source_gauss([])
    R0 = np.empty(s.n_test)
    s.residual_apply(U, R0, 0.05, 0.06)
    Ro0 = stdg.Oracle(m).residual(U, 0.05, 0.06)
    assert np.linalg.norm(Ro - Ro0) > 1e-6 * np.linalg.norm(Ro)
    assert rel(R - R0, Ro - Ro0) < 1e-8


def test_source_slab_solve(stm):
    """Zero field plus a Gaussian pulse: GPU slab solve vs the oracle's (load enters the solve)."""
    m = meshgen.box_mesh(3, 3, 2, hi=(1.0, 1.0, 0.7), p=2, q=2)
    o = stdg.Oracle(m)
    src = gauss_sources()
    dt = 0.04
    uo = o.end_state(o.slab_solve(np.zeros(o.ne * 6 * 27), 0.08, dt, src=oracle_J(src)))
    s = stm.Slab(m, tol=1e-14, max_it=3000)
    s.set_source_gauss(src)
    s.set_state(np.zeros(s.n_state), t=0.08)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK
    assert rel(s.get_state()[0], uo) < 1e-12


@pytest.mark.parametrize("curved", [False, True])
def test_boundary_data_patch(stm, curved):
    """E = (0,0,x), H = (0,t,0), g = E: the exact solution of Sec. 2 data; slab solve reproduces it."""
    m = meshgen.box_mesh(2, 2, 1, p=2, q=1, perturb=0.3 if curved else 0.0)
    o = stdg.Oracle(m)
    t0, dt = 0.3, 0.2
    Ef = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 0]], 1)
    u0 = o.project(Ef, lambda x: np.stack([0 * x[:, 0], t0 + 0 * x[:, 0], 0 * x[:, 0]], 1))
    u1 = o.project(Ef, lambda x: np.stack([0 * x[:, 0], t0 + dt + 0 * x[:, 0], 0 * x[:, 0]], 1))

    def g(x, t):
        return np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 0]], 1)

    s = stm.Slab(m, tol=1e-14, max_it=2000)
    s.set_boundary(g)
    s.set_state(u0, t=t0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK
    assert np.abs(s.get_state()[0] - u1).max() < 1e-11
    # residual with random U against the oracle's with the same g
    U = meshgen.random_coeffs(m, 16)
    Ro = o.residual(U, t0, dt, g=lambda x, t: np.stack(np.broadcast_arrays(0 * x[..., 0] + 0 * t, 0 * x[..., 0] + 0 * t, x[..., 0] + 0 * t), -1))
    R = np.empty(s.n_test)
    s.residual_apply(U, R, t0, dt)
    assert rel(R, Ro) < 1e-12


def test_curved_full_size_sampled(stm):
    """32^3 curved mesh (perturbation 0.1 h sin sin sin), p = 3, q = 2, Gaussian pulse:
    the launch configuration of a full-size apply, checked on sampled elements."""
    import torch

    m = meshgen.box_mesh(32, p=3, q=2, perturb=0.1, order="morton")
    meshgen.random_materials(m, 21, 22)
    src = [dict(centre=(0.5, 0.5, 0.5), dir=(0.0, 0.0, 1.0), sigma_x=0.05, t0=0.2, sigma_t=0.05, amp=1.0)]
    U = meshgen.random_coeffs(m, 23)
    s = stm.Slab(m)
    s.set_source_gauss(src)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
    dt = (1.0 / 32) / 7
    s.residual_apply(Ud, Rd, 0.18, dt)
    R = Rd.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(24))
    sample = sorted(set([0, m["hex"].shape[0] - 1] + list(rng.integers(0, m["hex"].shape[0], 10))))
    # elements next to the pulse centre carry the source
    cen = np.argmin(np.sum((m["vert"][m["hex"][:, 0]] - 0.49) ** 2, axis=1))
    sample.append(int(cen))
    # the oracle sees the sampled elements and their face neighbours (it finds the faces itself)
    keep = set(sample)
    for e in sample:
        keep |= {int(x) for x in m["nbr"][e] if x >= 0}
    keep = np.array(sorted(keep))
    sub = {k: m[k][keep] for k in ("hex", "p", "q", "eps", "mu")}
    sub.update(vert=m["vert"], geometry=m["geometry"])
    tper = 6 * 3 * 64
    Us = np.concatenate([U[e * tper:(e + 1) * tper] for e in keep])
    loc = {int(e): i for i, e in enumerate(keep)}
    o = stdg.Oracle(sub)
    per = 6 * 2 * 64
    for e in sample:
        Ro = o.element_residual(loc[e], Us, 0.18, dt, src=oracle_J(src))[0].ravel()
        assert rel(R[e * per:(e + 1) * per], Ro) < 1e-12, e


@pytest.mark.parametrize("curved", [False, True])
def test_host_current_source(stm, curved):
    """J(x, t) sampled on the host (stm_set_source): residual vs the oracle's load (J, v),
    on bricks and trilinear hexes; removing it restores the source-free residual."""
    m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.7, 0.9), p=3, q=2, perturb=0.2 if curved else 0.0)
    meshgen.random_materials(m, 31, 32)
    o = stdg.Oracle(m)

    def J(x, t):
        x0, x1, x2 = x[..., 0], x[..., 1], x[..., 2]
        return np.stack(np.broadcast_arrays(np.sin(2 * x0 + t) * x1, np.cos(x2 - t) + 0 * x0, x0 * x1 * x2 * (1 + t)), -1)

    U = meshgen.random_coeffs(m, 33)
    t0, dt = 0.1, 0.07
    s = stm.Slab(m)
    s.set_source(J)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, t0, dt)
    Ro = o.residual(U, t0, dt, src=J)
    assert rel(R, Ro) < 1e-12
    s.set_source(None)
    s.residual_apply(U, R, t0, dt)
    assert rel(R, o.residual(U, t0, dt)) < 1e-12


def test_dof_layout(stm):
    m = meshgen.box_mesh(2, p=2, q=2)
    m["p"] = np.array([1, 2, 3, 1, 2, 3, 1, 2], dtype=np.uint8)
    m["q"] = np.array([1, 2, 3, 1, 2, 3, 1, 2], dtype=np.uint8)
    s = stm.Slab(m)
    tr, te, st = s.dof_layout()
    assert np.array_equal(tr, meshgen.dof_offsets(m, "trial"))
    assert np.array_equal(te, meshgen.dof_offsets(m, "test"))
    assert st[-1] == s.n_state and tr[-1] == s.n_trial and te[-1] == s.n_test


@pytest.mark.parametrize("p", [2, 4])
def test_projection_curved(stm, p):
    """L2 projection of E0, H0 on trilinear hexes (metric mass solved by CG on the device)
    against the oracle's element-wise dense projection."""
    m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.8, 0.6), p=p, q=1, perturb=0.2)
    meshgen.random_materials(m, 41, 42)
    E0 = lambda x: np.stack([np.sin(3 * x[:, 0]) * x[:, 1], np.cos(2 * x[:, 2]) + x[:, 0], x[:, 0] * x[:, 1] * x[:, 2]], 1)
    H0 = lambda x: np.stack([x[:, 2] ** 2, np.sin(x[:, 0] + x[:, 1]), np.exp(-x[:, 1])], 1)
    o = stdg.Oracle(m)
    uo = o.project(E0, H0)
    s = stm.Slab(m)
    s.set_initial(E0, H0, t=0.25)
    ug, t = s.get_state()
    assert t == 0.25
    assert rel(ug, uo) < 1e-12
    assert abs(s.energy() - o.energy(uo)) <= 1e-12 * o.energy(uo)
