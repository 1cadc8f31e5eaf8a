"""Request server (continuous batching): results match the oracle, are the
same alone and in a concurrent mix, admission respects the HBM budget, and a
failing request leaves the others unaffected."""
import math

import numpy as np
import pytest

from oracle import stdg
from paper_1307_5310_gb300 import meshgen

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_5310_gb300 import stm as s

    return s


SRC = [dict(centre=(0.4, 0.5, 0.6), dir=(0.0, 1.0, 0.0), sigma_x=0.1, t0=0.1, sigma_t=0.05, amp=3.0)]
BOX = [(0.2, 0.2, 0.2, 0.6, 0.7, 0.5, 2.5, 1.5)]


def test_server_matches_oracle(stm):
    srv = stm.Server(workers=2, tol=1e-14)
    t = srv.submit(2, 2, 1, 3, 0.05, kind=0)
    res, state = srv.wait(t, with_state=True)
    srv.close()
    assert res["status"] == 0 and abs(res["t_final"] - 0.15) < 1e-12
    m = meshgen.box_mesh(2, p=2, q=1, order="lex")
    o = stdg.Oracle(m)
    u = o.project(lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], np.sin(math.pi * x[:, 0]) * np.sin(math.pi * x[:, 1])], 1),
                  None)
    A_b = o.assemble(0.0, 0.05)
    for k in range(3):
        u = o.end_state(o.slab_solve(u, k * 0.05, 0.05, A_b=A_b))
    assert rel(state, u) < 1e-12
    assert abs(res["energy"] - o.energy(u)) < 1e-12 * o.energy(u)


def test_server_alone_vs_mix(stm):
    req = dict(n=6, p=3, q=2, n_slabs=4, dt=0.02, kind=1, boxes=BOX, sources=SRC)
    srv = stm.Server(workers=1, tol=1e-10)
    alone, s_alone = srv.wait(srv.submit(**req), with_state=True)
    srv.close()
    assert alone["status"] == 0
    srv = stm.Server(workers=4, tol=1e-10)
    others = [dict(n=8, p=2, q=1, n_slabs=3, dt=0.02, kind=0),
              dict(n=4, p=4, q=3, n_slabs=5, dt=0.01, kind=1, sources=SRC),
              dict(n=10, p=2, q=2, n_slabs=2, dt=0.02, kind=0, boxes=BOX)]
    tickets = [srv.submit(**others[0]), srv.submit(**others[1]), srv.submit(**req), srv.submit(**others[2]),
               srv.submit(**req)]
    outs = [srv.wait(t, with_state=True) for t in tickets]
    st = srv.stats()
    srv.close()
    for res, _ in outs:
        assert res["status"] == 0
    for k in (2, 4):
        res, s_mix = outs[k]
        assert rel(s_mix, s_alone) < 1e-12
        assert res["iterations"] == alone["iterations"]
    assert st["completed"] == 5 and st["failed"] == 0
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]


def test_server_admission_and_failure(stm):
    srv = stm.Server(workers=4, hbm_budget_bytes=100 << 20, tol=1e-9)
    good = [srv.submit(4, 2, 1, 2, 0.02, kind=0) for _ in range(3)]
    bad = srv.submit(4, 9, 1, 2, 0.02)  # p = 9 is out of range
    more = [srv.submit(6, 2, 2, 2, 0.02, kind=1, sources=SRC) for _ in range(2)]
    results = [srv.wait(t)[0] for t in good + more]
    rb = srv.wait(bad)[0]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in results)
    assert rb["status"] < 0
    assert st["completed"] == 5 and st["failed"] == 1
    fp = [r["footprint_bytes"] for r in results]
    assert max(fp) <= st["hbm_budget_bytes"] < 2 * min(fp)  # one at a time
    assert st["peak_admitted_bytes"] <= st["hbm_budget_bytes"]
    assert sum(r["queue_ms"] > 1.0 for r in results) >= 3


def test_server_overlap(stm):
    """With room for all, requests that arrive together run at the same time."""
    srv = stm.Server(workers=4, hbm_budget_bytes=0, tol=1e-9)
    ts = [srv.submit(8, 3, 2, 3, 0.02, kind=0) for _ in range(4)]
    results = [srv.wait(t)[0] for t in ts]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in results)
    assert st["peak_admitted_bytes"] >= 2 * min(r["footprint_bytes"] for r in results)
