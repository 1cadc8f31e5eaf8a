"""The allocation-free residual entry point against the regular one.

stm_residual_apply_noalloc serves callers that cannot allocate device memory
(for example code inside a CUDA graph capture, or a host whose device memory
all belongs to its own pool): it keeps its scratch in a fixed static device
array and takes every input and output as a device pointer.  This test calls
it through the C ABI twice in a row, on two different meshes and degrees, and
compares each result with stm_residual_apply on the same input, within the
FP64 tolerance of the other GPU tests.  It also checks that a request larger
than the fixed scratch is refused without touching the output.
"""
import numpy as np
import pytest

from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu


def _device_inputs(m):
    import torch

    ne = m["hex"].shape[0]
    v = m["vert"][m["hex"]]                     # [ne, 8, 3]
    h = (v[:, 7, :] - v[:, 0, :]).copy()        # box edge lengths
    return (torch.from_numpy(m["nbr"].astype(np.int32)).cuda(), torch.from_numpy(h).cuda(),
            torch.from_numpy(m["eps"].copy()).cuda(), torch.from_numpy(m["mu"].copy()).cuda(), ne)


def test_noalloc_matches_residual_apply():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm

    for k, (dims, p, q, dt) in enumerate((((3, 3, 2), 3, 2, 0.05), ((4, 2, 3), 2, 3, 0.02))):
        m = meshgen.box_mesh(*dims, hi=(1.0, 0.6, 0.9), p=p, q=q, order="morton")
        meshgen.random_materials(m, 20 + k, 30 + k)
        s = stm.Slab(m)
        U = torch.from_numpy(meshgen.random_coeffs(m, 40 + k)).cuda()
        R_ref = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
        s.residual_apply(U, R_ref, 0.0, dt)
        nbr, h, eps, mu, ne = _device_inputs(m)
        R = torch.full((s.n_test,), float("nan"), dtype=torch.float64, device="cuda")
        rc = stm.residual_apply_noalloc(ne, p, q, dt, nbr, h, eps, mu, U, R)
        assert rc == stm.STM_OK
        torch.cuda.synchronize()
        err = (torch.linalg.norm(R - R_ref) / torch.linalg.norm(R_ref)).item()
        assert err < 1e-12, (k, err)
        s.close()


def test_noalloc_near_limit_back_to_back():
    """Two differently sized calls queued on one stream before a single synchronize, both
    close to the fixed scratch size: 1,000 elements at p=4, q=3 (32.4 MB of 33.5 MB) and
    216 elements at p=7, q=4 (31.9 MB, whose trace pass needs more than 48 KB of shared
    memory per block).  Each result must equal stm_residual_apply's."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm

    cases = []
    for k, (dims, p, q, dt) in enumerate((((10, 10, 10), 4, 3, 0.01), ((6, 6, 6), 7, 4, 0.004))):
        m = meshgen.box_mesh(*dims, hi=(1.0, 0.9, 0.8), p=p, q=q, order="morton")
        meshgen.random_materials(m, 50 + k, 60 + k)
        s = stm.Slab(m)
        U = torch.from_numpy(meshgen.random_coeffs(m, 70 + k)).cuda()
        R_ref = torch.empty(s.n_test, dtype=torch.float64, device="cuda")
        s.residual_apply(U, R_ref, 0.0, dt)
        torch.cuda.synchronize()
        s.close()
        R = torch.full_like(R_ref, float("nan"))
        cases.append((m, p, q, dt, U, R, R_ref) + _device_inputs(m))
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for m, p, q, dt, U, R, R_ref, nbr, h, eps, mu, ne in cases:
            rc = stm.residual_apply_noalloc(ne, p, q, dt, nbr, h, eps, mu, U, R, stream=stream.cuda_stream)
            assert rc == stm.STM_OK
    stream.synchronize()
    for m, p, q, dt, U, R, R_ref, *_ in cases:
        err = (torch.linalg.norm(R - R_ref) / torch.linalg.norm(R_ref)).item()
        assert err < 1e-12, (p, q, err)


def test_noalloc_rejects_oversized_request():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm

    p, q = 7, 4
    per_el = 8 * (6 + 6 * q * 512 + 24 * q * 64)
    ne = (32 * 1024 * 1024) // per_el + 1
    dummy_i = torch.zeros(6, dtype=torch.int32, device="cuda")
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    R = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    rc = stm.residual_apply_noalloc(ne, p, q, 0.1, dummy_i, dummy, dummy, dummy, dummy, R)
    assert rc == stm.STM_EINVAL
    torch.cuda.synchronize()
    assert torch.all(R == 7.0)
