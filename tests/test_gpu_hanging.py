"""2:1 hanging faces (corner-refined octree meshes, the hp batch workload):
CUDA path vs the oracle.  The oracle finds the hanging faces geometrically
and integrates the coarse face as four pieces; the CUDA path uses the hang
list and the transfer integrals of the face traces."""
import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def submesh(m, U, elems):
    """The sampled elements and every element that shares a face (or a piece of one)
    with them, as a mesh of its own for the oracle; returns (mesh, U, local ids)."""
    keep = set(elems)
    nbr, hang = m["nbr"], m.get("hang", np.zeros((0, 6), dtype=np.int64))
    for e in elems:
        keep |= {int(x) for x in nbr[e] if x >= 0}
        keep |= {int(x) for x in hang[hang[:, 0] == e, 2]} | {int(x) for x in hang[hang[:, 2] == e, 0]}
    keep = np.array(sorted(keep))
    off = meshgen.dof_offsets(m, "trial")
    sub = {k: m[k][keep] for k in ("hex", "p", "q", "eps", "mu")}
    sub.update(vert=m["vert"], geometry=m["geometry"])
    Us = np.concatenate([U[off[e]:off[e + 1]] for e in keep])
    loc = {int(e): i for i, e in enumerate(keep)}
    return sub, Us, [loc[e] for e in elems]


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


@pytest.mark.parametrize("radii,hp_seed", [([0.8], None), ([0.8], 5), ([0.8, 0.4], 6)])
def test_residual_hanging_fp64(stm, radii, hp_seed):
    m = meshgen.corner_octree_mesh(2, radii, p=2, q=2)
    if hp_seed is None:
        meshgen.random_materials(m, 1, 2)
    else:
        meshgen.random_hp(m, hp_seed, p_range=(1, 4), q_range=(1, 4))
    U = meshgen.random_coeffs(m, 3)
    Ro = stdg.Oracle(m).residual(U, 0.0, 0.03)
    s = stm.Slab(m)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.0, 0.03)
    assert rel(R, Ro) < 1e-12


def test_residual_hanging_fp32(stm):
    m = meshgen.corner_octree_mesh(2, [0.8])
    meshgen.random_hp(m, 7, p_range=(1, 4), q_range=(1, 3))
    U32 = meshgen.random_coeffs(m, 8).astype(np.float32)
    Ro = stdg.Oracle(m).residual(U32.astype(np.float64), 0.0, 0.03)
    s = stm.Slab(m)
    R = np.empty(s.n_test, np.float32)
    s.residual_apply(U32, R, 0.0, 0.03, prec=stm.STM_FP32)
    assert rel(R, Ro) < 2e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_solve_hanging(stm, precision):
    m = meshgen.corner_octree_mesh(2, [0.8])
    meshgen.random_hp(m, 9, p_range=(1, 2), q_range=(1, 3))
    o = stdg.Oracle(m)
    n_state = int(np.sum(6 * (m["p"].astype(np.int64) + 1) ** 3))
    u0 = np.random.Generator(np.random.PCG64(10)).uniform(-1, 1, n_state)
    dt = 0.02
    uo = o.end_state(o.slab_solve(u0, 0.0, dt))
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, tol=1e-14 if precision == "fp64" else 1e-11, max_it=4000)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rel(s.get_state()[0], uo) < (1e-12 if precision == "fp64" else 1e-9)


def test_gauss_source_hanging_hp(stm):
    """Gaussian current pulses on a 2:1 octree mesh with uneven (p, q): the load projected on
    the device per (p, q) class, residual vs the oracle's at 1e-12."""
    m = meshgen.corner_octree_mesh(2, [0.8])
    meshgen.random_hp(m, 17, p_range=(1, 4), q_range=(1, 3))
    srcs = [dict(centre=(0.3, 0.35, 0.4), dir=(0.0, 0.6, 0.8), sigma_x=0.2, t0=0.1, sigma_t=0.06, amp=1.5)]

    def J(x, t):
        sd = srcs[0]
        r2 = np.sum((x - np.asarray(sd["centre"])) ** 2, axis=-1)
        a = sd["amp"] * np.exp(-r2 / (2 * sd["sigma_x"] ** 2)) * np.exp(-(t - sd["t0"]) ** 2 / (2 * sd["sigma_t"] ** 2))
        return a[..., None] * np.asarray(sd["dir"])

    U = meshgen.random_coeffs(m, 18)
    s = stm.Slab(m)
    s.set_source_gauss(srcs)
    R = np.empty(s.n_test)
    s.residual_apply(U, R, 0.04, 0.05)
    assert rel(R, stdg.Oracle(m).residual(U, 0.04, 0.05, src=J)) < 1e-12


def test_hp_batch_full_size_sampled(stm):
    """~200k elements refined 2:1 towards a corner, p ~ U{1..7}, q ~ U{1..4}, eps ~ {1, 2.25, 4}:
    one apply over all (p, q) classes, checked on sampled elements of both sides of 2:1 faces."""
    import torch

    m = meshgen.corner_octree_mesh(50, [0.45, 0.2])
    meshgen.random_hp(m, 1307)
    ne = m["hex"].shape[0]
    assert 196000 <= ne <= 204000
    U = meshgen.random_coeffs(m, 1309)
    s = stm.Slab(m)
    Ud = torch.from_numpy(U).cuda()
    Rd = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
    h = 1.0 / (50 * 4)
    dt = h / 15
    s.residual_apply(Ud, Rd, 0.0, dt)
    R = Rd.cpu().numpy()
    off = meshgen.dof_offsets(m, "test")
    rng = np.random.Generator(np.random.PCG64(11))
    hang = m["hang"]
    sample = set(rng.integers(0, ne, 6).tolist())
    sample |= set(hang[rng.integers(0, hang.shape[0], 4), 0].tolist())  # coarse sides
    sample |= set(hang[rng.integers(0, hang.shape[0], 4), 2].tolist())  # fine sides
    sample |= {0, ne - 1}
    sample = sorted(sample)
    sub, Us, loc = submesh(m, U, sample)
    o = stdg.Oracle(sub)
    for e, le in zip(sample, loc):
        Ro = o.element_residual(le, Us, 0.0, dt)[0].ravel()
        assert rel(R[off[e]:off[e + 1]], Ro) < 1e-12, e


def test_graph_and_autotune(stm):
    """Graph-captured multi-class applies and autotuned block sizes give the same residual,
    and a graph-replayed slab solve matches the oracle."""
    import torch

    m = meshgen.corner_octree_mesh(2, [0.8, 0.4])
    meshgen.random_hp(m, 12, p_range=(1, 5), q_range=(1, 4))
    U = torch.from_numpy(meshgen.random_coeffs(m, 13)).cuda()
    ref = stm.Slab(m, graph=False)
    R0 = torch.empty(ref.n_test, dtype=torch.float64, device="cuda")
    ref.residual_apply(U, R0, 0.0, 0.02)
    s = stm.Slab(m, graph=True)
    R1 = torch.empty_like(R0)
    for _ in range(3):  # first call captures, the others replay
        R1.zero_()
        s.residual_apply(U, R1, 0.0, 0.02)
        torch.cuda.synchronize()
        assert torch.equal(R1, R0)
    tuned = s.autotune(0.02, reps=2)
    assert len(tuned) == len(set(zip(m["p"].tolist(), m["q"].tolist())))
    assert all(b in (64, 128, 256, 512) for _, _, b, _ in tuned)
    s.residual_apply(U, R1, 0.0, 0.02)
    torch.cuda.synchronize()
    assert torch.equal(R1, R0)
    # slab solve with replayed graphs vs the oracle (a smaller hp mesh)
    m = meshgen.corner_octree_mesh(2, [0.8])
    meshgen.random_hp(m, 15, p_range=(1, 2), q_range=(1, 2))
    o = stdg.Oracle(m)
    n_state = int(np.sum(6 * (m["p"].astype(np.int64) + 1) ** 3))
    u0 = np.random.Generator(np.random.PCG64(14)).uniform(-1, 1, n_state)
    uo = o.end_state(o.slab_solve(u0, 0.0, 0.02))
    s2 = stm.Slab(m, graph=True, tol=1e-14, max_it=4000)
    s2.set_state(u0)
    rc, rep = s2.slab_solve(0.02)
    assert rc == stm.STM_OK
    assert rel(s2.get_state()[0], uo) < 1e-12
