"""The serving layer (dot_server_*): continuous batching of many solves.

Every slot of a batch runs the recurrence, schedule and kernels of a DOT_MIXED
dot_create/dot_solve context, and no kernel mixes data of two slots.  So a
request's result must be the same whether it runs alone, in a batch with other
requests of its grid admitted at other times, or as a single context -- here
bit for bit (the mixed path is deterministic).
"""
import time

import numpy as np
import pytest

from gpu_util import ensure_built
from paper_2505_05424_gb300 import workloads as W
from paper_2505_05424_gb300.solver import DotError, DotServer, DotSolver

pytestmark = pytest.mark.gpu

TOL = 1e-6          # the serving stream's tolerance
MAXIT = 100000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def instance(N, T, seed, masked=False):
    """A seeded mixture pair (zeroed on a rectangle mask when masked)."""
    return W.mixture_pair(W.GridSpec(2, T, N), seed, obstacles=masked)


def solve_alone(N, T, seed, masked=False, **srv_kw):
    r0, r1, mask = instance(N, T, seed, masked)
    with DotServer(**srv_kw) as srv:
        rid = srv.submit(2, T, N, r0, r1, mask=mask, tol=TOL, maxit=MAXIT)
        st = srv.wait(rid, 600.0)
        return st, srv.result(rid)


def same(a, b):
    assert a["kkt"]["iterations"] == b["kkt"]["iterations"]
    assert a["objective"] == b["objective"]
    for k in ("eta_dot", "eta_P", "eta_D", "eta_C", "primal_obj", "dual_obj", "sigma"):
        assert a["kkt"][k] == b["kkt"][k], k
    for k in ("rho", "m", "phi"):
        np.testing.assert_array_equal(a[k], b[k])


def test_alone_equals_single_context():
    N, T, seed = 32, 16, 3101
    st, res = solve_alone(N, T, seed)
    assert st == 0 and res["kkt"]["eta_dot"] <= TOL
    r0, r1, _ = instance(N, T, seed)
    s = DotSolver(2, T, N, r0, r1, prec="mixed")
    rc = s.dot_solve(TOL, MAXIT)
    rho, m, phi, obj, kk = s.dot_get()
    s.close()
    assert rc == 0
    assert kk["iterations"] == res["kkt"]["iterations"]
    assert obj == res["objective"]
    np.testing.assert_array_equal(rho, res["rho"])
    np.testing.assert_array_equal(phi, res["phi"])
    np.testing.assert_array_equal(np.concatenate([a.ravel() for a in m]), res["m"])


def test_result_is_the_same_alone_and_in_the_mix():
    # the probe request: 64^2 x 16, masked, seed 3202
    probe = (64, 16, 3202, True)
    st0, alone = solve_alone(*probe)
    assert st0 == 0
    # the mix: requests of the probe's grid and of others, arriving while the
    # probe runs, so they join its batch at other iterations
    with DotServer() as srv:
        ids = []
        others = [(64, 16, 3300 + k, k % 2 == 0) for k in range(5)] + [(32, 16, 3400 + k, False) for k in range(6)]
        for k, (N, T, seed, masked) in enumerate(others[:3]):
            r0, r1, mask = instance(N, T, seed, masked)
            ids.append(srv.submit(2, T, N, r0, r1, mask=mask, tol=TOL, maxit=MAXIT))
        time.sleep(0.05)
        r0, r1, mask = instance(*probe)
        pid = srv.submit(2, probe[1], probe[0], r0, r1, mask=mask, tol=TOL, maxit=MAXIT)
        for N, T, seed, masked in others[3:]:
            time.sleep(0.01)
            r0, r1, mask = instance(N, T, seed, masked)
            ids.append(srv.submit(2, T, N, r0, r1, mask=mask, tol=TOL, maxit=MAXIT))
        assert srv.wait(pid, 600.0) == 0
        mixed = srv.result(pid)
        for rid in ids:
            assert srv.wait(rid, 600.0) == 0           # every request converged
        stats = srv.stats()
    assert stats["peak_running"] >= 2          # the probe shared the device with others
    same(alone, mixed)


def test_admission_waits_for_memory():
    # a budget of one four-slot 32^2 x 16 batch: the 48^2 request waits until that
    # batch has finished and returned its memory
    from paper_2505_05424_gb300.solver import dot_workspace_bytes
    budget = int(4.5 * dot_workspace_bytes(2, 16, 32))
    with DotServer(hbm_budget=budget, max_slots=4, idle_ms=0) as srv:
        ids = []
        for k in range(3):
            r0, r1, _ = instance(32, 16, 3500 + k)
            ids.append(srv.submit(2, 16, 32, r0, r1, tol=TOL, maxit=MAXIT, keep_fields=False))
        r0, r1, _ = instance(48, 16, 3600)
        ids.append(srv.submit(2, 16, 48, r0, r1, tol=TOL, maxit=MAXIT, keep_fields=False))
        for rid in ids:
            assert srv.wait(rid, 600.0) == 0
            res = srv.result(rid)
            assert res["kkt"]["eta_dot"] <= TOL
            assert "phi" not in res
        s = srv.stats()
        assert s["peak_batches"] == 1
        assert s["bytes"] <= budget


def test_request_larger_than_the_budget_is_rejected():
    # a 1 MB budget holds no batch of a 64^2 x 16 grid: DOT_ENOMEM at submit, not a
    # request that waits forever
    with DotServer(hbm_budget=1 << 20) as srv:
        r0, r1, _ = instance(64, 16, 3800)
        with pytest.raises(DotError):
            srv.submit(2, 16, 64, r0, r1, tol=TOL, maxit=10)
        assert srv.stats()["queued"] == 0


def test_non_batchable_grid_and_errors():
    # N = 30 is not a multiple of 4: a batch of one slot on the SIMT passes
    st, res = solve_alone(30, 8, 3700)
    assert st == 0 and res["kkt"]["eta_dot"] <= TOL
    with DotServer() as srv:
        with pytest.raises(DotError):
            srv.submit(2, 8, 16, -np.ones(256), np.ones(256))
        r0, r1, _ = instance(32, 16, 3701)
        rid = srv.submit(2, 16, 32, r0, r1, tol=0.0, maxit=20, keep_fields=False)
        assert srv.wait(rid, 600.0) == 1            # maxit reached: DOT_ENOTCONV
        assert srv.result(rid)["kkt"]["iterations"] == 20
        srv.release(rid)
        with pytest.raises(DotError):
            srv.result(rid)


def test_multilevel_request_matches_context_multilevel():
    """A request served with the multilevel warm start of Sec. 5 takes the path of
    dot_solve_multilevel: its coarse level is served as a request of the coarse grid
    (in that grid's batch) and the prolonged state starts the caller's grid.  Every
    kernel works on one slot's data, so the result is the context's bit for bit."""
    N, T, seed = 64, 16, 3701
    r0, r1, mask = instance(N, T, seed, True)
    with DotServer(multilevel=1, multilevel_min_nodes=0, multilevel_masked=True) as srv:
        rid = srv.submit(2, T, N, r0, r1, mask=mask, tol=TOL, maxit=MAXIT)
        assert srv.wait(rid, 600.0) == 0
        res = srv.result(rid)
    s = DotSolver(2, T, N, r0, r1, mask=mask, prec="mixed")
    rc, its = s.dot_solve_multilevel(1, TOL, MAXIT)
    rho, m, phi, obj, kk = s.dot_get()
    s.close()
    assert rc == 0
    print("multilevel: server", res["kkt"]["iterations"], res["objective"], "context", its, obj)
    assert res["kkt"]["eta_dot"] <= TOL
    assert res["kkt"]["iterations"] == kk["iterations"]
    assert res["objective"] == obj
    np.testing.assert_array_equal(res["rho"], rho)
    np.testing.assert_array_equal(res["phi"], phi)


def test_multilevel_threshold_and_options():
    """Requests below multilevel_min_nodes, and masked requests unless
    multilevel_masked, are served cold; bad options are refused."""
    N, T, seed = 32, 16, 3702
    st_cold, cold = solve_alone(N, T, seed)
    with DotServer(multilevel=1, multilevel_min_nodes=10 ** 9) as srv:
        r0, r1, _ = instance(N, T, seed)
        rid = srv.submit(2, T, N, r0, r1, tol=TOL, maxit=MAXIT)
        assert srv.wait(rid, 600.0) == 0
        res = srv.result(rid)
    same(cold, res)
    st_m, cold_m = solve_alone(N, T, seed + 1, True)
    with DotServer(multilevel=1, multilevel_min_nodes=0) as srv:
        r0, r1, mask = instance(N, T, seed + 1, True)
        rid = srv.submit(2, T, N, r0, r1, mask=mask, tol=TOL, maxit=MAXIT)
        assert srv.wait(rid, 600.0) == 0
        res = srv.result(rid)
    same(cold_m, res)
    with pytest.raises(DotError):
        DotServer(multilevel=9)
