"""Whole solves at the full sizes of the obstacle and 3D workloads, mixed path against
the FP64 path (which runs the oracle's recurrence, lock-step tested in
test_gpu_parity_fp64.py) as the reference, and the mixed path's reported stopping
measures against the oracle's evaluation of the same state (Sec. 5.3).

Reference protocol: the FP64 path from zero to eta_dot <= 1e-7.  On obstacle problems
(omega = 1e-6 on the masked cells, Sec. 5.4) the objective still moves by ~2e-5
relative between eta_dot = 1e-6 and 1e-7, so the mixed solve is continued to 5e-8
(it switches to tau = 1 below 3e-7) before the objectives are compared at 1e-6.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built
from paper_2505_05424_gb300 import workloads as W
from paper_2505_05424_gb300.solver import DotSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def oracle_eta(spec, r0, r1, mask, s):
    """The oracle's stopping measures on the solver's current state (z recomputed as
    Pi_Q(B F q + d - beta/sigma) from the returned q, beta and sigma)."""
    g = O.Grid(spec.D, spec.T, [spec.N] * spec.D)
    prob = O.Problem(g, r0, r1, mask)
    rho, m, phi, obj, kk = s.dot_get()
    q, al, beta, sigma, it = s.dot_get_state()
    z = O.proj_Q(g, O.apply_B(g, prob.omega, O.apply_F(g, q)) + O.fill_d(g) - beta / sigma)
    st = O.State(g, phi.ravel().copy(), z, q, al, beta, sigma)
    oracle_eta.last = (prob, st)
    return g, kk, O.kkt(prob, st), rho, obj


def test_obst128_mixed_against_fp64_reference():
    """2D 128^2 x 32 with rectangle obstacles (the obstacle workload, seed 1003)."""
    spec, r0, r1, mask = W.workload("obst128")
    s = DotSolver(2, spec.T, spec.N, r0, r1, mask=mask, prec="mixed")
    assert s.dot_solve(1e-6, 200000) == 0
    g, kk6, ko6, _, _ = oracle_eta(spec, r0, r1, mask, s)
    assert s.dot_solve(5e-8, 400000) == 0
    g, kk, ko, rho, obj = oracle_eta(spec, r0, r1, mask, s)
    s.close()
    # the reported measures are the oracle's on the same state
    for a, b in ((kk6, ko6), (kk, ko)):
        for name in ("eta_dot", "eta_P", "eta_D", "eta_C"):
            assert abs(a[name] - b[name]) <= 1e-8, name
    ref = DotSolver(2, spec.T, spec.N, r0, r1, mask=mask, prec="fp64")
    assert ref.dot_solve(1e-7, 400000) == 0
    rho_r, _, _, obj_r, kk_r = ref.dot_get()
    ref.close()
    d_rho = np.abs(rho - rho_r).max() / rho_r.max()
    print("obst128 mixed", kk["iterations"], obj, "FP64", kk_r["iterations"], obj_r,
          "rel", abs(obj - obj_r) / obj_r, "max|rho - rho_ref| / max", d_rho)
    assert abs(obj - obj_r) <= 1e-6 * obj_r
    assert d_rho <= 1e-2


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 2e-4)])
def test_mix3d64_two_iterations(prec, tol):
    """3D 64^3 x 32 anisotropic mixtures (the 3D workload, seed 1004): two iterations
    from zero against the oracle, every field (the mixed bound as for the full 2D grid:
    cones at the apex of Q carry FP32 direction rounding)."""
    spec, r0, r1, mask = W.workload("mix3d64")
    g = O.Grid(3, spec.T, [spec.N] * 3)
    prob = O.Problem(g, r0, r1, mask)
    st = O.State.zeros(g)
    for _ in range(2):
        O.iterate(prob, st, tau=1.9)
    s = DotSolver(3, spec.T, spec.N, r0, r1, mask=mask, prec=prec, check_every=0)
    s.dot_solve(0.0, 2)
    q, al, beta, _, it = s.dot_get_state()
    s.close()
    assert it == 2
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    errs = [rel(q, st.q), rel(al, st.alpha), rel(beta, st.beta)]
    print("mix3d64", prec, "q, alpha, beta", errs)
    if prec == "fp64":
        from test_gpu_parity_fp64 import fp64_tol
        tol = fp64_tol(spec.T, [spec.N] * 3)
    assert max(errs) < tol


def test_mix3d64_mixed_whole_solve():
    """The 3D workload solved to eta_dot <= 1e-6 on the mixed path; the oracle's
    stopping measures on the returned state agree with the reported ones, and every
    time slice carries mass 1 up to the dual residual (telescoping of A^*)."""
    spec, r0, r1, mask = W.workload("mix3d64")
    s = DotSolver(3, spec.T, spec.N, r0, r1, mask=mask, prec="mixed")
    assert s.dot_solve(1e-6, 60000) == 0
    g, kk, ko, rho, obj = oracle_eta(spec, r0, r1, mask, s)
    s.close()
    prob, st = oracle_eta.last
    for name in ("eta_dot", "eta_P", "eta_D", "eta_C"):
        assert abs(kk[name] - ko[name]) <= 1e-8, name
    assert kk["eta_dot"] <= 1e-6
    # every slice's mass is 1 up to the l1 norm of the dual residual A^*alpha + c
    area = O.cell_area(g)
    bound = area * np.abs(O.apply_At(g, st.alpha) + prob.c).sum()
    mass = rho.reshape(spec.T, -1).sum(axis=1) * area
    print("mix3d64 mixed", kk["iterations"], obj, "slice masses", mass.min(), mass.max(), "bound", bound)
    assert np.all(np.abs(mass - 1.0) <= bound + 1e-12)
