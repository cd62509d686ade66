"""GPU parity of the mixed-precision path against the FP64 oracle.

Tolerances come from the arithmetic.  One step: FP32 unit roundoff u = 6e-8;
each output is the end of at most ~20 roundings with an amplification of at most
~10 (the divisions in the cone projection and the diagonal solve), so a step
agrees to 2e-5 relative to the field's maximum.  The refined Poisson solve
(FP32 solve, exact two-float residual, FP32 correction) is accurate to u^2 times
the conditioning of the DCT pair and of the Laplacian, tested at 1e-9 up to 96
points per axis and scaled with the Laplacian's condition number beyond.  Whole solves: KKT <= 1e-6 and
the objective against the FP64 oracle's continued to eta <= 1e-7.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import ensure_built, pair, random_state, rel_err
from paper_2505_05424_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


# odd sizes (SIMT DCT passes), and axis lengths divisible by 4 (tensor-core DCT
# passes) with row counts that leave ragged 128-row tiles, up to a 300-long axis
# (two 256-column output tiles, the second ragged) and 1024-long axes (four output
# tiles, the axis length of the 1024^2 x 32 scalability case) first and last
GRIDS = [(2, 4, [6, 5]), (2, 1, [2, 2]), (2, 69, [70, 3]), (2, 7, [9, 131]), (3, 3, [4, 3, 5]),
         (3, 5, [6, 7, 66]), (2, 5, [32, 36]), (2, 9, [256, 64]), (2, 16, [32, 32]), (3, 3, [8, 12, 16]),
         (2, 64, [128, 128]), (2, 3, [8, 300]), (2, 3, [8, 1024]), (2, 7, [1024, 12])]


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def centred(v):
    """phi modulo constants.  The FP32 DCT rows are orthogonal to the constant vector
    only up to rounding and A^*A cannot see constants, so the mixed solve leaves an
    O(u_32 |phi|) constant in phi; A removes it and sum(c) = 0, so q, alpha, beta and
    the objective do not depend on it."""
    v = np.asarray(v, dtype=np.float64).ravel()
    return v - v.mean()


# grids whose tcgen05 passes have more work units (128-row tile x column tile) than
# the GPU has SMs, so that each persistent CTA runs several units through its
# stage ring and both TMEM accumulators: 256^2 x 64 (2-4 units per CTA) and
# 512^2 x 8 (a 9-long time axis: about 14 units per CTA)
MANY_UNITS = [(2, 64, [256, 256]), (2, 8, [512, 512]), (2, 2, [1024, 1024])]


@pytest.mark.parametrize("D,T,N", GRIDS + MANY_UNITS)
def test_refined_poisson(D, T, N):
    rng = np.random.default_rng(500 + T)
    g = O.Grid(D, T, N)
    b = f32(rng.standard_normal(g.n_nodes) + 0.5)
    r0 = rng.random(int(np.prod(N))) + 0.1
    _, _, gpu = pair(D, T, N, r0, r0, prec="mixed")
    phi = gpu.dot_poisson(b)
    ref = O.poisson(g, b)
    assert rel_err(centred(phi), ref) < refined_tol(T, N)
    gpu.close()


def refined_tol(T, N):
    """Bound on the refined solve's error relative to max|phi|.  The FP32 solve's
    error scales with the condition number of the Neumann Laplacian on the longest
    axis, (2 n / pi)^2 for n points, and the refinement leaves a multiple of it: 1e-9
    up to 96 points, growing as n^2 beyond (measured 5.0e-10 at 128^2 x 64, 1.05e-9
    at 192^2 x 32, 3.3e-9 at 256^2 x 64, 7.6e-9 at 512^2 x 8)."""
    n = max([T + 1] + list(N))
    return 1e-9 * max(1.0, (n / 96.0) ** 2)


@pytest.mark.parametrize("D,T,N", [(2, 5, [32, 36]), (2, 64, [128, 128]), (3, 3, [8, 12, 16]), (2, 3, [8, 300]),
                                   (2, 3, [8, 1024])] + MANY_UNITS)
def test_poisson_runs_entirely_on_tensor_cores(D, T, N):
    """Every axis fits a tcgen05 tile: each of the two solves of a refined Poisson
    solve is D spatial passes each way plus two time passes, none on the SIMT
    fallback."""
    rng = np.random.default_rng(700 + T)
    r0 = rng.random(int(np.prod(N))) + 0.1
    _, _, gpu = pair(D, T, N, r0, r0, prec="mixed")
    gpu.dot_profile(True)
    gpu.dot_poisson(rng.standard_normal((T + 1) * int(np.prod(N))))
    prof = gpu.dot_profile_read()
    gpu.close()
    assert prof["dct_axis"][1] == 0
    assert prof["dct_tcgen05"][1] == 2 * 2 * D
    assert prof["dct_scale"][1] == 2 * 2


@pytest.mark.parametrize("D,T,N", GRIDS)
@pytest.mark.parametrize("masked", [False, True])
def test_one_iteration_from_random_state(D, T, N, masked):
    rng = np.random.default_rng(600 + T + 7 * masked)
    P = int(np.prod(N))
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    mask = (rng.random(P) < 0.2) if masked else None
    g, prob, gpu = pair(D, T, N, r0, r1, mask=mask, prec="mixed", check_every=0)
    q, al, beta = random_state(g, rng)
    q = f32(q)                      # q is stored in FP32 on the GPU
    sigma = float(rng.uniform(0.5, 3.0))
    st = O.State(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), q.copy(), al.copy(), beta.copy(), sigma)
    O.iterate(prob, st, tau=1.9)
    gpu.dot_set_state(q, al, beta, sigma)
    gpu.dot_solve(tol=0.0, maxit=1)
    q2, al2, b2, _, it = gpu.dot_get_state()
    _, _, phi, _, _ = gpu.dot_get()
    assert it == 1
    tol = step_tol(T, N)
    assert rel_err(centred(phi), st.phi) < tol
    assert rel_err(q2, st.q) < tol
    assert rel_err(al2, st.alpha) < tol
    assert rel_err(b2, st.beta) < tol
    kg, ko = gpu.dot_kkt(), O.kkt(prob, st)
    for name in ("eta_P", "eta_D", "eta_C", "eta_P_soc", "eta_D_soc"):
        assert abs(kg[name] - ko[name]) <= 1e-3 * abs(ko[name]) + 1e-6, name
    assert abs(kg["primal_obj"] - ko["primal_obj"]) <= STEP_TOL * max(abs(ko["primal_obj"]), 1e-12)
    gpu.close()


def step_tol(T, N):
    """STEP_TOL, scaled beyond 256 points per axis with the conditioning of the Neumann
    Laplacian ((2 n / pi)^2 for n points): from a random state the iteration's single
    FP32/3xTF32 solve is a cold solve, and q, alpha, beta inherit its error through
    A phi (measured on 1024-long axes, relative to each field's maximum: phi 2.2e-5,
    alpha 8.6e-5 at 4 x 8 x 1024 nodes; q 9.4e-5 (1.6e-4 masked) at 8 x 1024 x 12;
    phi 2.9e-5, q 1.6e-4, alpha 1.7e-4, beta 1.8e-4 at 3 x 1024^2; bound 3.2e-4)."""
    n = max([T + 1] + list(N))
    return STEP_TOL * max(1.0, (n / 256.0) ** 2)


def test_gauss32_mixed_converges_to_fp64_objective():
    """2D 32^2 x 16 two Gaussians + floor: mixed reaches KKT 1e-6 and its objective is
    within 1e-6 relative of the FP64 oracle's at the same tolerance."""
    from gpu_util import oracle_solution
    spec, r0, r1, mask, g, prob, st, res = oracle_solution("gauss32")
    gpu = pair(2, spec.T, [spec.N] * 2, r0, r1, prec="mixed")[2]
    rc = gpu.dot_solve(tol=1e-6, maxit=40000)
    assert rc == 0
    rho, m, phi, obj, kk = gpu.dot_get()
    assert kk["eta_dot"] <= 1e-6
    ref = O.w2_squared(g, res["primal_obj"])
    rho_o = O.density_slices(g, st)
    print("mixed iters", kk["iterations"], "oracle iters", res["iterations"], "obj", obj, "ref", ref,
          "rel", abs(obj - ref) / abs(ref), "max|rho-rho_o|/max", np.abs(rho - rho_o).max() / rho_o.max())
    assert abs(obj - ref) <= 1e-6 * abs(ref)
    # both iterates stop at eta_dot <= 1e-6; at that tolerance the densities of two
    # runs agree to ~0.5% of their maximum on this grid (FP64 at 1e-6 vs 1e-7 differ
    # by as much), so this is a sanity bound, not a precision claim
    assert np.abs(rho - rho_o).max() <= 1e-2 * rho_o.max()
    gpu.close()


# 3D grids: several 4 x 4 x 32 tiles of the D = 3 face pass with ragged edges on
# every axis, and more than one 16-node time chunk
@pytest.mark.parametrize("D,T,N,masked", [(2, 8, [12, 10], False), (3, 20, [5, 6, 37], False),
                                          (3, 4, [7, 4, 33], True)])
def test_mixed_lockstep_tracks_fp64(D, T, N, masked):
    """Tens of iterations: the mixed iterate stays within the FP32 noise of the oracle's
    (every iteration after the first starts from the residual the previous one left)."""
    rng = np.random.default_rng(700 if D == 2 else 710 + T)
    P = int(np.prod(N))
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    mask = (rng.random(P) < 0.2) if masked else None
    g, prob, gpu = pair(D, T, N, r0, r1, mask=mask, prec="mixed", check_every=10)
    st = O.State.zeros(g)
    O.solve(prob, st, tol=0.0, maxit=50, check_every=10)
    gpu.dot_solve(tol=0.0, maxit=50)
    q2, al2, b2, s2, _ = gpu.dot_get_state()
    assert s2 == st.sigma
    assert rel_err(q2, st.q) < 1e-4 and rel_err(al2, st.alpha) < 1e-4 and rel_err(b2, st.beta) < 1e-4
    gpu.close()


def test_full_size_mix256_two_iterations():
    """2D 256^2 x 64 Gaussian mixtures -- the timed workload's data, grid and launch
    configuration -- two mixed iterations from zero against the oracle, every field.
    The bound is wider than STEP_TOL: the mixtures have exact zeros (pdf < 1e-4 set
    to 0), which put cones at the apex of Q, where the FP32 projection's direction
    carries up to ~1e3 x the unit roundoff relative to the field's maximum; measured
    on GB300: phi 4.6e-6 / 6.0e-5, q 6.8e-5 / 6.4e-5, alpha 3.4e-5 / 2.8e-5,
    beta 4.8e-5 / 3.9e-5 after one / two iterations."""
    spec, r0, r1, mask = W.workload("mix256")
    g, prob, gpu = pair(2, spec.T, [spec.N] * 2, r0, r1, prec="mixed", check_every=0)
    st = O.State.zeros(g)
    for _ in range(2):
        O.iterate(prob, st, tau=1.9)
    gpu.dot_solve(tol=0.0, maxit=2)
    q2, al2, b2, _, it = gpu.dot_get_state()
    _, _, phi, _, _ = gpu.dot_get()
    gpu.close()
    assert it == 2
    tol = 2e-4
    assert rel_err(centred(phi), st.phi) < tol
    assert rel_err(q2, st.q) < tol
    assert rel_err(al2, st.alpha) < tol
    assert rel_err(b2, st.beta) < tol


def test_1024_plane_one_iteration():
    """A full 1024^2 plane (the scalability case's spatial grid) at T = 2: one mixed
    iteration from a random state against the oracle, every field, at step_tol."""
    D, T, N = 2, 2, [1024, 1024]
    rng = np.random.default_rng(1024)
    P = N[0] * N[1]
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    g, prob, gpu = pair(D, T, N, r0, r1, prec="mixed", check_every=0)
    q, al, beta = random_state(g, rng)
    q = f32(q)
    sigma = 1.7
    st = O.State(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), q.copy(), al.copy(), beta.copy(), sigma)
    O.iterate(prob, st, tau=1.9)
    gpu.dot_set_state(q, al, beta, sigma)
    gpu.dot_solve(tol=0.0, maxit=1)
    q2, al2, b2, _, it = gpu.dot_get_state()
    _, _, phi, _, _ = gpu.dot_get()
    gpu.close()
    assert it == 1
    tol = step_tol(T, N)
    errs = [rel_err(centred(phi), st.phi), rel_err(q2, st.q), rel_err(al2, st.alpha), rel_err(b2, st.beta)]
    print("1024^2 x 2 one iteration: phi, q, alpha, beta", errs)
    assert max(errs) < tol


def test_longest_time_axis_one_iteration():
    """T + 1 = 160 time nodes, the most the mixed path accepts: one iteration from a
    random state against the oracle, every field (its tcgen05 time passes run a
    160-long axis: five 32-wide K chunks and a 160-column accumulator)."""
    D, T, N = 2, 159, [8, 12]
    rng = np.random.default_rng(159)
    P = N[0] * N[1]
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    g, prob, gpu = pair(D, T, N, r0, r1, prec="mixed", check_every=0)
    q, al, beta = random_state(g, rng)
    q = f32(q)
    sigma = 1.3
    st = O.State(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), q.copy(), al.copy(), beta.copy(), sigma)
    O.iterate(prob, st, tau=1.9)
    gpu.dot_set_state(q, al, beta, sigma)
    gpu.dot_solve(tol=0.0, maxit=1)
    q2, al2, b2, _, it = gpu.dot_get_state()
    _, _, phi, _, _ = gpu.dot_get()
    gpu.close()
    assert it == 1
    errs = [rel_err(centred(phi), st.phi), rel_err(q2, st.q), rel_err(al2, st.alpha), rel_err(b2, st.beta)]
    print("T + 1 = 160 one iteration: phi, q, alpha, beta", errs)
    assert max(errs) < step_tol(T, N)


def test_time_axis_beyond_the_limit_is_rejected():
    """161 time nodes: the mixed path refuses the grid with DOT_EINVAL before any work."""
    from paper_2505_05424_gb300 import _native as N
    from paper_2505_05424_gb300.solver import DotError, DotSolver
    r = np.ones(64)
    with pytest.raises(DotError) as e:
        DotSolver(2, 160, [8, 8], r, r, prec="mixed")
    assert e.value.code == N.DOT_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_identical_densities_move_nothing(prec):
    """rho_0 = rho_1 (the degenerate problem): both paths solve to eta_dot <= 1e-7 and
    return the static path rho(t) = rho_0, m = 0, W2^2 = 0 up to the tolerance.  The
    oracle on this instance at eta_dot <= 1e-7: rho within 6.6e-4 of rho_0 (relative to
    its maximum), |m| <= 1.9e-5, W2^2 = 4.3e-8 (at 1e-6: 4.8e-3, 1.4e-4, 5.9e-7)."""
    D, T, N = 2, 16, [32, 32]
    rng = np.random.default_rng(1601)
    r = rng.random(1024) + 0.05
    gpu = pair(D, T, N, r, r, prec=prec)[2]
    assert gpu.dot_solve(1e-7, 200000) == 0
    rho, m, phi, obj, kk = gpu.dot_get()
    gpu.close()
    r0 = (r / r.sum() * 1024).reshape(N)          # cell-average density of mass 1 on [0, 1]^2
    dev = np.abs(rho - r0).max() / r0.max()
    mm = max(np.abs(a).max() for a in m) / r0.max()
    print(prec, "iterations", kk["iterations"], "W2^2", obj, "rho dev", dev, "m", mm)
    assert abs(obj) <= 2e-7
    assert dev <= 2e-3
    assert mm <= 1e-4
