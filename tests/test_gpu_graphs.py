"""dot_solve's CUDA-graph replay of check periods against kernel-by-kernel launches.

With use_graphs = 1 each period of check_every iterations plus the stopping
measures (Algorithm 2 and the checks of Sec. 5.3) is replayed from a captured
graph; the penalty is applied between periods outside the graph and the kernels
read it from device memory.  The launch sequence is the same as without graphs,
so every result must agree bit for bit: iterations, sigma, stopping measures,
objective and the fields.
"""
import numpy as np
import pytest

from gpu_util import ensure_built
from paper_2505_05424_gb300 import workloads as W
from paper_2505_05424_gb300.solver import DotSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def solver(N, T, seed, graphs, masked=False, **opts):
    r0, r1, mask = W.mixture_pair(W.GridSpec(2, T, N), seed, obstacles=masked)
    return DotSolver(2, T, [N, N], r0, r1, mask=mask, prec="mixed", use_graphs=int(graphs), **opts)


def outcome(s):
    rho, m, phi, obj, kk = s.dot_get()
    return {"rho": rho, "m": np.concatenate([a.ravel() for a in m]), "phi": phi, "obj": obj, "kkt": kk}


def same(a, b):
    assert a["kkt"] == b["kkt"]
    assert a["obj"] == b["obj"]
    for k in ("rho", "m", "phi"):
        np.testing.assert_array_equal(a[k], b[k])


def run(calls, graphs, N=32, T=16, seed=4101, masked=False, profile=False, **opts):
    s = solver(N, T, seed, graphs, masked, **opts)
    if profile:
        s.dot_profile(True)
    rcs = [s.dot_solve(tol, maxit) for tol, maxit in calls]
    out = outcome(s)
    out["rcs"] = rcs
    out["launches"] = s.launch_count()
    if profile:
        out["prof"] = s.dot_profile_read()
    s.close()
    return out


def run_both(calls, **kw):
    return run(calls, True, **kw), run(calls, False, **kw)


def test_whole_solve_matches():
    g, d = run_both([(1e-5, 20000)])
    assert g["rcs"] == d["rcs"] == [0]
    same(g, d)
    assert g["launches"] == d["launches"]


def test_remainder_and_chained_calls_match():
    # 37 iterations: three periods and seven iterations without a check; the next
    # call then starts with the residual carried over (its first period runs
    # kernel by kernel), then a masked instance for the obstacle weights
    g, d = run_both([(0.0, 37), (0.0, 25), (1e-4, 400)])
    assert g["rcs"] == d["rcs"]
    same(g, d)
    assert g["launches"] == d["launches"]
    g, d = run_both([(0.0, 53), (1e-5, 3000)], N=48, T=8, seed=4102, masked=True)
    assert g["rcs"] == d["rcs"]
    same(g, d)


def test_odd_check_period_uses_both_parities():
    g, d = run_both([(1e-5, 20000)], seed=4103, check_every=3)
    assert g["rcs"] == d["rcs"] == [0]
    same(g, d)


def test_profiled_solve_matches_graph_replay():
    # a profiled solve launches kernel by kernel (per-kernel events); its results
    # equal those of the unprofiled graph replay
    p = run([(0.0, 60)], True, profile=True)
    g = run([(0.0, 60)], True)
    same(p, g)
    assert p["launches"] == g["launches"]
    launched = {k: v for k, v in p["prof"].items() if v[1] > 0}
    assert launched.get("fused_cone_update", (0.0, 60))[1] == 60
    assert all(ms > 0.0 for ms, _ in launched.values())
