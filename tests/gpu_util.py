"""Helpers shared by the GPU parity tests: build the library once, pair a GPU
solver with the oracle on identical seeded inputs, and convert layouts."""
import numpy as np

import oracle as O
from paper_2505_05424_gb300 import _native as N
from paper_2505_05424_gb300.solver import DotSolver


def ensure_built():
    N.build()
    return N.load()


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


def pair(D, T, N_, r0, r1, mask=None, prec="fp64", **opts):
    g = O.Grid(D, T, N_)
    prob = O.Problem(g, r0, r1, mask)
    gpu = DotSolver(D, T, N_, r0, r1, mask=mask, prec=prec, **opts)
    return g, prob, gpu


def random_state(g, rng, scale=1.0):
    """A random iterate (q, alpha, beta) in the oracle's natural layout."""
    q = rng.standard_normal(g.n_q) * scale
    al = rng.standard_normal(g.n_q) * scale * 0.1
    beta = rng.standard_normal(g.K * g.n_cones) * scale
    return q, al, beta


_ORACLE_CACHE = {}


def oracle_solution(name, tol=1e-6, maxit=60000):
    """Oracle solve of a named workload from zero (cached for the test session)."""
    key = (name, tol)
    if key not in _ORACLE_CACHE:
        from paper_2505_05424_gb300 import workloads as W
        spec, r0, r1, mask = W.workload(name)
        g = O.Grid(spec.D, spec.T, [spec.N] * spec.D)
        prob = O.Problem(g, r0, r1, mask)
        st = O.State.zeros(g)
        res = O.solve(prob, st, tol=tol, maxit=maxit)
        _ORACLE_CACHE[key] = (spec, r0, r1, mask, g, prob, st, res)
    return _ORACLE_CACHE[key]


_MIX_CACHE = {}


def oracle_mixture(T, N, seed, masked=False, tol=1e-7, tau=1.9, maxit=400000):
    """Oracle solve from zero of a seeded 2D Gaussian-mixture instance on an N^2 x T grid
    (optionally with rectangle obstacles), cached for the test session.
    Returns (r0, r1, mask, g, prob, st, res)."""
    key = (T, N, seed, masked, tol, tau)
    if key not in _MIX_CACHE:
        from paper_2505_05424_gb300 import workloads as W
        r0, r1, mask = W.mixture_pair(W.GridSpec(2, T, N), seed, obstacles=masked)
        g = O.Grid(2, T, [N, N])
        prob = O.Problem(g, r0, r1, mask)
        st = O.State.zeros(g)
        res = O.solve(prob, st, tol=tol, maxit=maxit, tau=tau)
        assert res["eta_dot"] <= tol
        _MIX_CACHE[key] = (r0, r1, mask, g, prob, st, res)
    return _MIX_CACHE[key]
