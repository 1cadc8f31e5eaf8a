"""Inexact slab solves with the guaranteed iteration-error bound (Sec. 5.3).

Each slab stops once its share of eta_it (Eq. a_posteriori:iteration) is below
eta_tol / sqrt(N).  Checks:
  * the reported per-slab term equals 4 c_E |R_E|^2_{W'} + 4 c_H |R_H|^2_{W'}
    computed here from the oracle's residual and the closed-form Gram matrix
    of the test basis on bricks (orthonormal Legendre in time and space,
    covariant map: int_{I_n x K} v_a . v_b = dt |K| / h_c^2 delta_ab);
  * the bound holds: the energy-norm distance between the inexact end state
    and the oracle's direct slab solves at t_N is at most eta_it;
  * it is not vacuous (efficiency index eta_it / error below 100) and the
    inexact solve takes fewer GMRES iterations than a tight one.
"""
import math

import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


def _brick_sizes(m):
    v = np.asarray(m["vert"])[np.asarray(m["hex"])]  # [ne, 8, 3]
    return v.max(1) - v.min(1)


def _eta2_closed_form(m, o, R, dt, t_final):
    """4 sum_f c_f |R_f|^2_{W'} with the dual norm from the Gram matrix of the test basis."""
    h = _brick_sizes(m)
    vol = h.prod(1)
    eps = np.asarray(m["eps"], np.float64)
    mu = np.asarray(m["mu"], np.float64)
    cf = [2 * t_final / eps.min() + dt * dt / (2 * t_final * eps.min()),
          2 * t_final / mu.min() + dt * dt / (2 * t_final * mu.min())]
    tot = 0.0
    off = 0
    for e in range(o.ne):
        q, n3 = int(o.q[e]), int((o.p[e] + 1) ** 3)
        r = R[off:off + 6 * q * n3].reshape(2, 3, q * n3)
        off += 6 * q * n3
        for f in range(2):
            for c in range(3):
                gram = dt * vol[e] / h[e, c] ** 2
                tot += 4 * cf[f] * float(r[f, c] @ r[f, c]) / gram
    return tot


def test_eta_term_matches_closed_form(stm):
    """At the initial guess (a loose eta_tol stops before any iteration) the
    reported term equals the dual norm computed from the oracle residual."""
    m = meshgen.box_mesh(2, 3, 2, hi=(0.5, 0.75, 0.5), p=2, q=2)
    meshgen.random_materials(m, 21, 22)
    o = stdg.Oracle(m)
    rng = np.random.Generator(np.random.PCG64(23))
    u0 = rng.uniform(-1, 1, o.ne * 6 * 27)
    dt, t_final = 0.05, 0.4
    # the solver's initial guess is constant in time: modes l_0 = 1 - xi and l_1 = xi both carry u0
    n3, q = 27, 2
    U = o.embed_start(u0).reshape(o.ne, 2, 3, q + 1, n3)
    U[:, :, :, 1, :] = U[:, :, :, 0, :]
    R = o.residual(U.ravel(), 0.0, dt)
    want = _eta2_closed_form(m, o, R, dt, t_final)
    s = stm.Slab(m, eta_tol=1e6, t_final=t_final)
    s.set_state(u0)
    rc, rep = s.slab_solve(dt)
    assert rc == stm.STM_OK, rep
    assert rep["iterations"] == 0
    assert abs(rep["eta2"] - want) <= 1e-10 * want
    ug, _ = s.get_state()
    assert np.array_equal(ug, u0)  # the initial guess is constant in time


def _cavity(x, t=0.0):
    z = np.zeros(x.shape[0])
    return np.stack([z, z, np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])], 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_iteration_error_bound_holds(stm, precision):
    """4^3 PEC cavity, random eps/mu, p = 2, q = 2, 16 slabs: the energy-norm
    iteration error at t_N is below the accumulated eta_it, eta_it <= eta_tol,
    and the bound is within two decades of the true error."""
    m = meshgen.box_mesh(4, p=2, q=2)
    meshgen.random_materials(m, 31, 32)
    o = stdg.Oracle(m)
    dt, N = 0.05, 16
    t_final = N * dt
    u = o.project(_cavity, None)
    A_b = o.assemble(0.0, dt)
    for n in range(N):
        u = o.end_state(o.slab_solve(u, n * dt, dt, A_b=A_b))
    e0 = o.energy(o.project(_cavity, None))
    eta_tol = 1e-3 * math.sqrt(2 * e0)
    prec = stm.STM_FP64 if precision == "fp64" else stm.STM_MIXED
    s = stm.Slab(m, precision=prec, eta_tol=eta_tol, t_final=t_final, max_it=2000)
    s.set_initial(_cavity, None)
    tight = stm.Slab(m, precision=prec, tol=1e-12, max_it=2000)
    tight.set_initial(_cavity, None)
    eta2, it, it_tight = 0.0, 0, 0
    for _ in range(N):
        rc, rep = s.slab_solve(dt)
        assert rc == stm.STM_OK, rep
        eta2 += rep["eta2"]
        it += rep["iterations"]
        rc, rep = tight.slab_solve(dt)
        assert rc == stm.STM_OK, rep
        it_tight += rep["iterations"]
    ug, t = s.get_state()
    assert abs(t - t_final) < 1e-12
    err2 = 2.0 * o.energy(ug - u)  # |eps^1/2 e(t_N)|^2 + |mu^1/2 h(t_N)|^2
    assert err2 <= eta2
    assert eta2 <= eta_tol ** 2 * (1 + 1e-12)
    assert math.sqrt(eta2 / err2) < 100.0
    assert it < it_tight


def test_inexact_rejects_unsupported(stm):
    """Curved meshes (no closed-form dual norm here) and a missing t_N are refused."""
    m = meshgen.box_mesh(3, p=1, q=1, perturb=0.05)
    s = stm.Slab(m, eta_tol=1e-3, t_final=1.0)
    s.set_state(np.zeros(s.n_state))
    with pytest.raises(stm.StmError) as ex:
        s.slab_solve(0.05)
    assert ex.value.code == stm.STM_EUNSUPPORTED
    m = meshgen.box_mesh(2, p=1, q=1)
    s = stm.Slab(m, eta_tol=1e-3, t_final=0.0)
    s.set_state(np.zeros(s.n_state))
    with pytest.raises(stm.StmError) as ex:
        s.slab_solve(0.05)
    assert ex.value.code == stm.STM_EINVAL
