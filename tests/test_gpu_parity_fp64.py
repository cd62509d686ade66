"""GPU parity of the FP64 path against the oracle (element by element).

The FP64 path computes the same recurrence in the same precision, so iterates
must agree to rounding: the bar is 1e-11 relative to the field's max for one
step from a random state and for lock-step runs of tens of iterations (the
recurrence is contractive, rounding differences do not grow), and identical
stopping iterations and sigma schedules for whole solves.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built, pair, random_state, rel_err
from paper_2505_05424_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


def fp64_tol(T, N):
    """Rounding bound of the FP64 path: the DCT solve amplifies relative rounding by
    the condition number kappa = lambda_max / lambda_min of A^*A on mean-zero fields;
    allow 100 u kappa (u = 1.1e-16), at least TOL."""
    lam = lambda h, M, k: 4.0 / h ** 2 * np.sin(np.pi * k / (2 * M)) ** 2
    M = [T + 1] + list(N)
    h = [1.0 / T] + [1.0 / n for n in N]
    lmax = sum(lam(hh, m, m - 1) for hh, m in zip(h, M))
    lmin = min(lam(hh, m, 1) for hh, m in zip(h, M))
    return max(TOL, 100 * 1.1e-16 * lmax / lmin)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


# grids spanning several 64-wide GEMM tiles with ragged tails, odd sizes, 3D
GRIDS = [(2, 4, [6, 5]), (2, 1, [2, 2]), (2, 69, [70, 3]), (2, 7, [9, 131]), (3, 3, [4, 3, 5]),
         (3, 5, [6, 7, 66])]


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_poisson_parity(D, T, N):
    rng = np.random.default_rng(100 + T)
    g = O.Grid(D, T, N)
    b = rng.standard_normal(g.n_nodes) + 0.5
    r0 = rng.random(int(np.prod(N))) + 0.1
    _, _, gpu = pair(D, T, N, r0, r0, prec="fp64")
    phi = gpu.dot_poisson(b)
    ref = O.poisson(g, b)
    assert rel_err(phi, ref) < TOL
    gpu.close()


@pytest.mark.parametrize("D,T,N", GRIDS)
@pytest.mark.parametrize("masked", [False, True])
def test_one_iteration_from_random_state(D, T, N, masked):
    rng = np.random.default_rng(200 + T + 7 * masked)
    P = int(np.prod(N))
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    mask = (rng.random(P) < 0.2) if masked else None
    g, prob, gpu = pair(D, T, N, r0, r1, mask=mask, prec="fp64", check_every=0)
    q, al, beta = random_state(g, rng)
    sigma = float(rng.uniform(0.5, 3.0))
    st = O.State(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), q.copy(), al.copy(), beta.copy(), sigma)
    O.iterate(prob, st, tau=1.9)
    gpu.dot_set_state(q, al, beta, sigma)
    gpu.dot_solve(tol=0.0, maxit=1)
    q2, al2, b2, s2, it = gpu.dot_get_state()
    _, _, phi, _, _ = gpu.dot_get()
    assert it == 1 and s2 == sigma
    assert rel_err(phi.ravel(), st.phi) < TOL
    assert rel_err(q2, st.q) < TOL
    assert rel_err(al2, st.alpha) < TOL
    assert rel_err(b2, st.beta) < TOL
    # stopping measures of the same iterate
    kg = gpu.dot_kkt()
    ko = O.kkt(prob, st)
    for name in ("eta_P", "eta_D", "eta_C", "eta_P_soc", "eta_D_soc", "primal_obj", "dual_obj"):
        assert abs(kg[name] - ko[name]) <= 1e-10 * max(abs(ko[name]), 1e-30), name
    gpu.close()


@pytest.mark.parametrize("D,T,N,steps", [(2, 8, [12, 10], 60), (3, 4, [5, 6, 4], 30)])
def test_lockstep_with_sigma_rule(D, T, N, steps):
    rng = np.random.default_rng(300 + T)
    P = int(np.prod(N))
    r0 = np.where(rng.random(P) < 0.2, 0.0, rng.random(P))
    r1 = rng.random(P) + 0.01
    g, prob, gpu = pair(D, T, N, r0, r1, prec="fp64", check_every=10)
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=steps, check_every=10)
    gpu.dot_solve(tol=0.0, maxit=steps)
    q2, al2, b2, s2, it = gpu.dot_get_state()
    assert it == steps
    assert s2 == st.sigma          # identical penalty schedule
    assert rel_err(q2, st.q) < 1e-10
    assert rel_err(al2, st.alpha) < 1e-10
    assert rel_err(b2, st.beta) < 1e-10
    gpu.close()


def test_gauss32_full_solve_matches_oracle():
    """2D 32^2 x 16, two Gaussians + floor 1e-3, FP64, stop at KKT 1e-6."""
    from gpu_util import oracle_solution
    spec, r0, r1, mask, g, prob, st, res = oracle_solution("gauss32")
    gpu = pair(spec.D, spec.T, [spec.N] * spec.D, r0, r1, prec="fp64")[2]
    rc = gpu.dot_solve(tol=1e-6, maxit=60000)
    assert rc == 0
    rho, m, phi, obj, kk = gpu.dot_get()
    assert kk["eta_dot"] <= 1e-6
    assert int(kk["iterations"]) == res["iterations"]
    assert abs(obj - O.w2_squared(g, res["primal_obj"])) <= 1e-9 * abs(obj)
    rho_o = O.density_slices(g, st)
    assert np.abs(rho - rho_o).max() <= 1e-9 * rho_o.max()
    # every time slice carries mass 1 up to the l1 norm of the dual residual A^*alpha + c
    # (telescoping of A^*; eta_D <= 1e-6 is an L2 norm weighted by the cell volume)
    area = O.cell_area(g)
    bound = area * np.abs(O.apply_At(g, st.alpha) + prob.c).sum()
    assert np.all(np.abs(rho.reshape(spec.T, -1).sum(axis=1) * area - 1.0) <= bound + 1e-12)
    gpu.close()


def test_obstacle_lockstep():
    spec = W.GridSpec(2, 8, 24)
    r0, r1, mask = W.mixture_pair(spec, 7, obstacles=True)
    g, prob, gpu = pair(2, 8, [24, 24], r0, r1, mask=mask, prec="fp64")
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=40)
    gpu.dot_solve(tol=0.0, maxit=40)
    q2, al2, b2, s2, it = gpu.dot_get_state()
    assert s2 == st.sigma
    assert rel_err(q2, st.q) < 1e-10 and rel_err(al2, st.alpha) < 1e-10 and rel_err(b2, st.beta) < 1e-10
    gpu.close()


def test_edge_cases_single_cell_mass_and_smallest_grid():
    """A single occupied cell (a Dirac-like mass) and the smallest 2 x 2 x 1 grid."""
    rng = np.random.default_rng(400)
    r0 = np.zeros(36); r0[7] = 1.0
    r1 = np.zeros(36); r1[30] = 2.0
    g, prob, gpu = pair(2, 3, [6, 6], r0, r1, prec="fp64")
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=25)
    gpu.dot_solve(tol=0.0, maxit=25)
    q2, al2, b2, _, _ = gpu.dot_get_state()
    assert rel_err(q2, st.q) < 1e-10 and rel_err(b2, st.beta) < 1e-10
    gpu.close()
    g, prob, gpu = pair(2, 1, [2, 2], np.array([1.0, 0, 0, 0]), np.array([0, 0, 0, 1.0]), prec="fp64")
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=20)
    gpu.dot_solve(tol=0.0, maxit=20)
    q2, al2, b2, _, _ = gpu.dot_get_state()
    assert rel_err(q2, st.q) < 1e-10 and rel_err(al2, st.alpha) < 1e-10
    gpu.close()


def test_full_size_mix256_two_iterations():
    """2D 256^2 x 64 Gaussian mixtures (the timed workload's grid): two iterations
    from zero, every field against the oracle."""
    spec, r0, r1, mask = W.workload("mix256")
    g, prob, gpu = pair(2, spec.T, [spec.N] * 2, r0, r1, prec="fp64", check_every=0)
    st = O.State.zeros(g)
    for _ in range(2):
        O.iterate(prob, st, tau=1.9)
    gpu.dot_solve(tol=0.0, maxit=2)
    q2, al2, b2, _, _ = gpu.dot_get_state()
    tol = fp64_tol(spec.T, [spec.N] * 2)
    assert rel_err(q2, st.q) < tol and rel_err(al2, st.alpha) < tol and rel_err(b2, st.beta) < tol
    gpu.close()


@pytest.mark.parametrize("D,T,N", [(2, 3, [8, 1024]), (2, 5, [1024, 6])])
def test_1024_axis(D, T, N):
    """1024-long spatial axes (the scalability case's), first and last: the Poisson solve
    and one iteration from a random state against the oracle."""
    rng = np.random.default_rng(1100 + T)
    g = O.Grid(D, T, N)
    P = int(np.prod(N))
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    _, prob, gpu = pair(D, T, N, r0, r1, prec="fp64", check_every=0)
    tol = fp64_tol(T, N)
    b = rng.standard_normal(g.n_nodes) + 0.5
    assert rel_err(gpu.dot_poisson(b), O.poisson(g, b)) < tol
    q, al, beta = random_state(g, rng)
    st = O.State(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), q.copy(), al.copy(), beta.copy(), 1.3)
    O.iterate(prob, st, tau=1.9)
    gpu.dot_set_state(q, al, beta, 1.3)
    gpu.dot_solve(tol=0.0, maxit=1)
    q2, al2, b2, _, _ = gpu.dot_get_state()
    gpu.close()
    assert rel_err(q2, st.q) < tol and rel_err(al2, st.alpha) < tol and rel_err(b2, st.beta) < tol
