"""Pins for the oracle's cone projection (eq. (app-proj)) and Poisson solve (Sec. 4).

Projection: the three closed-form cases, the Moreau decomposition for the
self-dual second-order cone, idempotence and the variational inequality
against random cone points.  Poisson: the DCT-II matrix against scipy's
orthonormal DCT-II (a library special case), the closed-form eigenvalues of the
Neumann Laplacian A^*A, and the residual A^*A phi = b - mean(b) with phi mean-zero.
"""
import numpy as np
import pytest
import scipy.fft

import oracle as O


def in_cone(z, tol=1e-12):
    return z[0] >= np.linalg.norm(z[1:]) - tol * (1 + np.abs(z).max())


@pytest.mark.parametrize("n", [10, 14, 6])
def test_projection_cases(n):
    rng = np.random.default_rng(10)
    # case 1: inside the cone -> unchanged
    y = rng.standard_normal(n)
    y[0] = np.linalg.norm(y[1:]) + 0.5
    np.testing.assert_array_equal(O.proj_soc(y), y)
    # case 2: inside the polar cone -> 0
    y[0] = -np.linalg.norm(y[1:]) - 0.5
    np.testing.assert_array_equal(O.proj_soc(y), 0.0)
    # case 3: boundary point 1/2 (y0 + |ybar|)(1, ybar/|ybar|)
    y[0] = 0.3 * np.linalg.norm(y[1:])
    z = O.proj_soc(y)
    nb = np.linalg.norm(y[1:])
    assert np.isclose(z[0], 0.5 * (y[0] + nb), rtol=1e-14)
    assert np.isclose(z[0], np.linalg.norm(z[1:]), rtol=1e-13)


@pytest.mark.parametrize("n", [10, 14])
def test_projection_moreau_and_optimality(n):
    rng = np.random.default_rng(11)
    for _ in range(500):
        y = rng.standard_normal(n) * rng.uniform(0.01, 10)
        p, m = O.proj_soc(y), O.proj_soc(-y)
        np.testing.assert_allclose(p - m, y, atol=1e-12 * np.abs(y).max())   # y = P_K(y) + P_{K°}(y)
        assert abs(p @ m) <= 1e-12 * (1 + np.abs(y).max() ** 2)
        assert in_cone(p)
        np.testing.assert_allclose(O.proj_soc(p), p, atol=1e-13 * (1 + np.abs(p).max()))
        # <y - P(y), w - P(y)> <= 0 for every w in K
        for _k in range(5):
            w = rng.standard_normal(n)
            w[0] = np.linalg.norm(w[1:]) + abs(rng.standard_normal())
            assert (y - p) @ (w - p) <= 1e-10 * (1 + np.abs(y).max() * np.abs(w).max())


def test_projection_beats_random_cone_points():
    """Brute force: no sampled cone point is closer to y than P(y)."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        y = rng.standard_normal(10)
        p = O.proj_soc(y)
        d0 = np.linalg.norm(y - p)
        W = rng.standard_normal((20000, 10))
        W[:, 0] = np.linalg.norm(W[:, 1:], axis=1) * (1 + rng.exponential(0.1, 20000))
        W *= rng.exponential(1.0, (20000, 1))
        assert d0 <= np.linalg.norm(W - y, axis=1).min() + 1e-12


@pytest.mark.parametrize("D,T,N", [(1, 5, [7]), (2, 4, [6, 5]), (3, 3, [4, 3, 5])])
def test_dct_matches_scipy(D, T, N):
    g = O.Grid(D, T, N)
    x = np.random.default_rng(13).standard_normal(g.node_shape)
    for axis in range(D + 1):
        ref = scipy.fft.dct(x, type=2, norm="ortho", axis=axis)
        np.testing.assert_allclose(O.dct_axis(g, axis, x).reshape(g.node_shape), ref, atol=1e-13)
        back = O.dct_axis(g, axis, ref, inverse=True).reshape(g.node_shape)
        np.testing.assert_allclose(back, x, atol=1e-13)
    np.testing.assert_allclose(O.dct_matrix(9) @ O.dct_matrix(9).T, np.eye(9), atol=1e-14)


@pytest.mark.parametrize("D,T,N", [(1, 5, [7]), (2, 4, [6, 5]), (2, 8, [8, 8]), (3, 3, [4, 3, 5])])
def test_poisson_eigenvectors(D, T, N):
    """A DCT basis vector cos(pi k (n + 1/2) / M) per axis is an eigenvector of A^*A with
    eigenvalue sum_d (4/h_d^2) sin^2(pi k_d / (2 M_d)) -- the textbook Neumann spectrum."""
    g = O.Grid(D, T, N)
    rng = np.random.default_rng(14)
    for _ in range(5):
        k = [int(rng.integers(0, m)) for m in g.node_shape]
        if all(v == 0 for v in k):
            k[0] = 1
        grids = np.meshgrid(*[np.arange(m) for m in g.node_shape], indexing="ij")
        v = np.ones(g.node_shape)
        lam = 0.0
        for a, m in enumerate(g.node_shape):
            v = v * np.cos(np.pi * k[a] * (grids[a] + 0.5) / m)
            lam += 4.0 / g.h[a] ** 2 * np.sin(np.pi * k[a] / (2 * m)) ** 2
        np.testing.assert_allclose(O.apply_At(g, O.apply_A(g, v)), lam * v.ravel(), atol=1e-9 * lam)
        np.testing.assert_allclose(O.poisson(g, v), v.ravel() / lam, atol=1e-12 / lam * 10)


@pytest.mark.parametrize("D,T,N", [(2, 4, [6, 5]), (2, 16, [32, 32]), (3, 3, [4, 3, 5])])
def test_poisson_residual_and_zero_mode(D, T, N):
    g = O.Grid(D, T, N)
    b = np.random.default_rng(15).standard_normal(g.n_nodes) + 3.0   # non-zero mean on purpose
    phi = O.poisson(g, b)
    assert abs(phi.mean()) < 1e-13 * np.abs(phi).max()
    r = O.apply_At(g, O.apply_A(g, phi)) - (b - b.mean())
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
