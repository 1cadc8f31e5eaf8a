"""Host logic of the seeded input generators (no method arithmetic): mesh
topology, element orders, 2:1 octree structure, per-element degrees and the
coefficient layouts both the oracle and the CUDA path index with."""
import numpy as np
import pytest

from oracle.stdg import face_neighbours
from paper_1307_5310_gb300 import meshgen


@pytest.mark.parametrize("order", ["lex", "morton"])
def test_box_mesh_neighbours_match_vertex_sharing(order):
    """nbr of the generator equals the neighbours found from shared vertex quadruples,
    and face 2d+1 of an element meets face 2d of its neighbour."""
    m = meshgen.box_mesh(3, 4, 2, order=order)
    nb = m["nbr"]
    fv = face_neighbours(m["hex"])
    assert np.array_equal(nb, fv[:, :, 0])
    for e in range(nb.shape[0]):
        for f in range(6):
            if nb[e, f] >= 0:
                assert fv[e, f, 1] == f ^ 1
                assert nb[nb[e, f], f ^ 1] == e


def test_morton_order_is_a_permutation_with_local_neighbours():
    lex, mor = meshgen.box_mesh(8, order="lex"), meshgen.box_mesh(8, order="morton")
    key = lambda m: sorted(map(tuple, np.sort(m["hex"], axis=1)))
    assert key(lex) == key(mor)  # the same cells
    # face neighbours sit closer in memory along the Z-order curve (median id distance)
    dist = lambda m: np.median([abs(e - n) for e in range(512) for n in m["nbr"][e] if n >= 0])
    assert dist(mor) < dist(lex)


def test_perturbed_box_keeps_the_boundary_and_is_curved():
    m = meshgen.box_mesh(3, perturb=0.2)
    assert m["geometry"] == "trilinear"
    v = m["vert"]
    on_bnd = np.any((np.abs(v) < 1e-12) | (np.abs(v - 1) < 1e-12), axis=1)
    flat = meshgen.box_mesh(3)["vert"]
    assert np.allclose(v[on_bnd], flat[on_bnd])
    assert np.abs(v - flat).max() > 1e-3


def test_corner_octree_is_2to1_balanced():
    m = meshgen.corner_octree_mesh(2, [0.8, 0.4])
    ne = m["hex"].shape[0]
    hang = m["hang"]
    assert hang.shape[1] == 6 and hang.shape[0] % 4 == 0
    # every coarse face with a -2 flag has exactly four fine rows covering its quarters
    rows = {}
    for ce, cf, fe, ff, u, v in hang:
        assert m["nbr"][ce, cf] == -2 and m["nbr"][fe, ff] == -2
        assert cf // 2 == ff // 2 and ff == cf ^ 1
        rows.setdefault((ce, cf), set()).add((u, v))
    assert all(q == {(0, 0), (1, 0), (0, 1), (1, 1)} for q in rows.values())
    # fine faces are half the coarse edge length: 2:1, never 4:1
    size = lambda e: np.ptp(m["vert"][m["hex"][e]][:, 0])
    for ce, cf, fe, ff, u, v in hang:
        assert np.isclose(size(ce), 2 * size(fe))
    # conforming neighbours have equal size
    for e in range(ne):
        for f in range(6):
            n = m["nbr"][e, f]
            if n >= 0:
                assert np.isclose(size(e), size(n))


def test_random_degrees_and_nk_are_seeded():
    a, b = meshgen.box_mesh(4), meshgen.box_mesh(4)
    meshgen.random_nk(a, 7)
    meshgen.random_nk(b, 7)
    assert np.array_equal(a["nk"], b["nk"]) and set(a["nk"].tolist()) <= {1, 2, 4}
    meshgen.random_nk(b, 8)
    assert not np.array_equal(a["nk"], b["nk"])
    c = meshgen.corner_octree_mesh(2, [0.8])
    meshgen.random_hp(c, 3, p_range=(1, 3), q_range=(1, 2))
    assert c["p"].min() >= 1 and c["p"].max() <= 3 and c["q"].min() >= 1 and c["q"].max() <= 2


def test_layout_sizes():
    m = meshgen.box_mesh(2, p=2, q=3)
    m["nk"] = np.array([1, 2, 4, 1, 2, 4, 1, 2], dtype=np.uint8)
    tr, te = meshgen.dof_offsets(m, "trial"), meshgen.dof_offsets(m, "test")
    n3 = 27
    assert np.array_equal(np.diff(tr), 6 * (m["nk"].astype(int) * 3 + 1) * n3)
    assert np.array_equal(np.diff(te), 6 * m["nk"].astype(int) * 3 * n3)
    assert meshgen.random_coeffs(m, 1).size == tr[-1]


def test_affine_box_mesh_is_parallelepipeds():
    A = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.2, 1.1]])
    m = meshgen.box_mesh(3, 2, 2, hi=(1.0, 0.8, 0.6), affine=A)
    assert m["geometry"] == "affine"
    X = m["vert"][m["hex"]]                      # [ne, 8, 3]
    DF = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 4] - X[:, 0]], axis=2)  # columns
    for v in range(8):
        b = np.array([v & 1, (v >> 1) & 1, (v >> 2) & 1], dtype=np.float64)
        assert np.allclose(X[:, v], X[:, 0] + DF @ b, atol=1e-14)
    # every element is the image of the same box cell: DF = A diag(h)
    h = np.array([1.0 / 3, 0.4, 0.3])
    assert np.allclose(DF, (A * h)[None], atol=1e-14)
    with pytest.raises(ValueError):
        meshgen.box_mesh(2, affine=-np.eye(3))
