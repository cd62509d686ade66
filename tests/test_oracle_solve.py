"""Whole-solve pins for the oracle (Algorithm 2 with the rules of Sec. 5.3).

* brute force: the oracle's fixed point equals the optimum of problem (8) found by an
  independent dense barrier method on 4x4x4 grids (random densities, exact zeros, an
  obstacle mask with omega = 1e-6);
* the stopping measures vanish at that independent optimum (pins og_kkt's formulas);
* mass conservation of every time slice (telescoping of A^*, Sec. 2.2);
* closed-form Wasserstein distances: translated densities (W2^2 = |shift|^2) and
  separable densities (W2^2 = sum of the 1D quantile-formula values), up to
  discretisation error that must shrink under refinement.
"""
import numpy as np
import pytest

import oracle as O
from bruteforce import DenseDOT


def _solve_oracle(g, r0, r1, mask=None, tol=1e-9, maxit=200000):
    prob = O.Problem(g, r0, r1, mask)
    st = O.State.zeros(g)
    res = O.solve(prob, st, tol=tol, maxit=maxit)
    return prob, st, res


CASES = {
    "random": lambda rng: (rng.random(16) + 0.1, rng.random(16) + 0.1, None),
    "zeros": lambda rng: (np.where(rng.random(16) < 0.3, 0.0, rng.random(16)),
                          np.where(rng.random(16) < 0.3, 0.0, rng.random(16)), None),
    "obstacle": lambda rng: (np.r_[rng.random(5) + 0.1, 0.0, 0.0, rng.random(9) + 0.1],
                             np.r_[rng.random(5) + 0.1, 0.0, 0.0, rng.random(9) + 0.1],
                             np.r_[np.zeros(5, bool), True, True, np.zeros(9, bool)]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_bruteforce_4x4x4(case):
    rng = np.random.default_rng({"random": 21, "zeros": 22, "obstacle": 23}[case])
    r0, r1, mask = CASES[case](rng)
    g = O.Grid(2, 4, [4, 4])
    prob, st, res = _solve_oracle(g, r0, r1, mask)
    assert res["eta_dot"] <= 1e-9

    dd = DenseDOT(2, 4, [4, 4])
    c = dd.c(prob.m0, prob.m1)
    np.testing.assert_array_equal(c, prob.c)
    phi_b, q_b, lam = dd.barrier_solve(c, prob.omega)
    obj_b = c @ phi_b
    assert abs(res["primal_obj"] - obj_b) <= 1e-7 * abs(obj_b)
    assert abs(res["dual_obj"] - obj_b) <= 1e-7 * abs(obj_b)
    # densities rho = alpha_0 / h_0 against the barrier multipliers (unique where rho > 0)
    rtol = 1e-7
    rho = O.density_slices(g, st).ravel()
    np.testing.assert_allclose(rho, lam * g.T, atol=rtol * np.abs(rho).max())


@pytest.mark.parametrize("case", sorted(CASES))
def test_kkt_measures_vanish_at_independent_optimum(case):
    rng = np.random.default_rng({"random": 31, "zeros": 32, "obstacle": 33}[case])
    r0, r1, mask = CASES[case](rng)
    g = O.Grid(2, 4, [4, 4])
    prob = O.Problem(g, r0, r1, mask)
    dd = DenseDOT(2, 4, [4, 4])
    phi_b, q_b, lam = dd.barrier_solve(prob.c, prob.omega)
    st = O.State.zeros(g)
    st.phi = phi_b.copy()
    st.q = np.concatenate(q_b)
    st.alpha = np.concatenate(dd.alpha_from(lam, q_b, prob.omega))
    kk = O.kkt(prob, st)
    assert kk["eta_P"] <= 1e-13
    assert kk["eta_D"] <= 1e-8
    assert kk["eta_C"] <= 1e-8
    assert kk["gap"] <= 1e-8
    # a perturbed point must not pass: guards against measures that are identically small
    st.alpha[: g.n_cones] *= 1.01
    assert O.kkt(prob, st)["eta_D"] > 1e-6


def test_mass_conservation_every_slice():
    g = O.Grid(2, 8, [8, 8])
    rng = np.random.default_rng(41)
    r0, r1 = rng.random(64) + 0.05, rng.random(64) + 0.05
    prob = O.Problem(g, r0, r1)
    st = O.State.zeros(g)
    for maxit in (7, 150):
        O.solve(prob, st, tol=0.0, maxit=maxit, check_every=0)
        resid = O.apply_At(g, st.alpha) + prob.c
        area = O.cell_area(g)
        bound = area * np.abs(resid).sum()
        mass = O.density_slices(g, st).reshape(g.T, -1).sum(axis=1) * area
        assert np.all(np.abs(mass - 1.0) <= bound + 1e-12)


def _w2_1d(f0, f1, n=200001):
    """Textbook 1D W2^2 = int_0^1 |F0^{-1}(u) - F1^{-1}(u)|^2 du for cell-mass densities on [0,1]."""
    def qf(f):
        m = f / f.sum()
        edges = np.linspace(0, 1, len(f) + 1)
        cdf = np.concatenate([[0.0], np.cumsum(m)])
        u = (np.arange(n) + 0.5) / n
        return np.interp(u, cdf, edges)     # piecewise-constant density -> piecewise-linear CDF
    return np.mean((qf(f0) - qf(f1)) ** 2)


def test_translated_gaussians_w2():
    """W2^2 between a density and its translate is |shift|^2 (closed form), up to discretisation."""
    from paper_2505_05424_gb300.workloads import gaussian_pair
    vals = []
    for N, T in ((12, 6), (20, 8)):
        r0, r1 = gaussian_pair(N, 2, mu0=(0.4, 0.45), mu1=(0.6, 0.55), sig=0.07, floor=0.0)
        g = O.Grid(2, T, [N, N])
        prob, st, res = _solve_oracle(g, r0, r1, tol=1e-6, maxit=20000)
        vals.append(O.w2_squared(g, res["primal_obj"]))
    exact = 0.2 ** 2 + 0.1 ** 2
    err = [abs(v - exact) / exact for v in vals]
    assert err[-1] < 0.06
    assert err[1] < err[0]


def test_separable_densities_w2():
    """(f0(x)+e)(g0(y)+e) -> (f1(x)+e)(g1(y)+e): W2^2 = W2^2(f0,f1) + W2^2(g0,g1) in the continuum."""
    from paper_2505_05424_gb300.workloads import product_pair
    errs = []
    for N, T in ((10, 5), (20, 8)):
        r0, r1, (f0, g0, f1, g1) = product_pair(N)
        g = O.Grid(2, T, [N, N])
        prob, st, res = _solve_oracle(g, r0, r1, tol=1e-6, maxit=20000)
        exact = _w2_1d(f0, f1) + _w2_1d(g0, g1)
        errs.append(abs(O.w2_squared(g, res["primal_obj"]) - exact) / exact)
    assert errs[-1] < 0.04
    assert errs[1] < errs[0]


@pytest.mark.parametrize("masked", [False, True])
def test_feasibility_at_convergence(masked):
    """At eta_dot <= 1e-7 the iterate is feasible up to the tolerance: the density
    rho = alpha_0 / h_0 is nonnegative (complementarity part of eta_C), z lies in Q
    exactly (it is a projection, eq. (app-proj)), B F q + d lies within the primal
    residual of Q (q in P, eq. (socobservation)), and beta lies in Q = Q^* (the dual
    cone of the SOCP).  Measured: rho >= -9e-10, z 2e-16, B F q + d 7e-7 and beta
    1.6e-9 outside their cones."""
    g = O.Grid(2, 8, [10, 12])
    rng = np.random.default_rng(91 + masked)
    P = 120
    r0, r1 = rng.random(P) + 0.05, rng.random(P) + 0.05
    r0[rng.random(P) < 0.15] = 0.0          # exact zeros, as in the mixture workloads
    mask = (rng.random(P) < 0.1) if masked else None
    prob = O.Problem(g, r0, r1, mask)
    st = O.State.zeros(g)
    res = O.solve(prob, st, tol=1e-7, maxit=400000)
    assert res["eta_dot"] <= 1e-7
    K = g.K

    def outside(a):   # largest ||a_bar|| - a_0 over the cones (<= 0 inside Q)
        a = a.reshape(K, -1)
        return float(np.max(np.linalg.norm(a[1:], axis=0) - a[0]))

    rho = O.density_slices(g, st)
    assert rho.min() >= -1e-6 * rho.max()
    assert outside(st.z) <= 1e-13
    y = O.apply_B(g, prob.omega, O.apply_F(g, st.q)) + O.fill_d(g)
    assert outside(y) <= 2e-6
    assert outside(st.beta) <= 1e-7


def test_identical_densities_static_solution():
    """rho_0 = rho_1: nothing moves.  The optimum is the static path rho(t) = rho_0,
    m = 0 with W2^2 = 0 (the Benamou-Brenier cost vanishes only for m = 0).  Measured
    at eta_dot <= 1e-8: W2^2 = -1.6e-9, rho within 7.7e-6 of rho_0, |m| <= 1.1e-6."""
    g = O.Grid(2, 8, [12, 10])
    rng = np.random.default_rng(5)
    r = rng.random(120) + 0.05
    prob = O.Problem(g, r, r)
    st = O.State.zeros(g)
    res = O.solve(prob, st, tol=1e-8, maxit=400000)
    assert res["eta_dot"] <= 1e-8
    assert abs(O.w2_squared(g, res["primal_obj"])) <= 1e-7
    r0 = (r / r.sum() / O.cell_area(g)).reshape(g.N)
    rho = O.density_slices(g, st)
    assert np.abs(rho - r0).max() <= 1e-4 * r0.max()
    assert max(np.abs(a).max() for a in O.momentum(g, st)) <= 1e-4 * r0.max()
