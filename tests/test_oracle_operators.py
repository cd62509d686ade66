"""Pins for the oracle's linear operators (Sec. 2.2, Sec. 3.2-3.3).

Each check is a fact the paper or plain mathematics fixes: the kernel of A
(eq. (kerA)), exactness on linear functions, the telescoping of A^* behind mass
conservation, the identity L_T L_X^* = 1/4 sum F^d_v (eq. (f1vf2v)), the
diagonal of F^*B^*BF (Proposition 3.2), and the cone equivalence
(eq. (socobservation)) including the weighted set P_omega (Sec. 5.4).
"""
import numpy as np
import pytest

import oracle as O

GRIDS = [(1, 3, [5]), (2, 4, [4, 4]), (2, 3, [5, 3]), (3, 2, [3, 4, 2])]


def node_coords(g):
    axes = [np.arange(g.T + 1) / g.T] + [(np.arange(n) + 0.5) / n for n in g.N]
    return np.meshgrid(*axes, indexing="ij")


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_kernel_of_A_is_constants(D, T, N):
    g = O.Grid(D, T, N)
    q = O.apply_A(g, np.full(g.n_nodes, 3.7))
    assert np.max(np.abs(q)) == 0.0
    # and nothing else: A^*A has a one-dimensional kernel (rank n_nodes - 1)
    M = np.stack([O.apply_A(g, e) for e in np.eye(g.n_nodes)], axis=1)
    assert np.linalg.matrix_rank(M) == g.n_nodes - 1


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_A_exact_on_linear_functions(D, T, N):
    g = O.Grid(D, T, N)
    X = node_coords(g)
    coef = [1.5, -0.25, 2.0, 0.75][: D + 1]
    phi = sum(c * x for c, x in zip(coef, X))
    blocks = g.split_q(O.apply_A(g, phi))
    for f, blk in enumerate(blocks):
        np.testing.assert_allclose(blk, coef[f], rtol=0, atol=1e-12)


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_At_telescopes_over_space(D, T, N):
    """sum over space of (A^*a)(t, .) = (sum a_0(t-1, .) - sum a_0(t, .)) / h_0, a_0 := 0 outside."""
    g = O.Grid(D, T, N)
    a = np.random.default_rng(1).standard_normal(g.n_q)
    out = O.apply_At(g, a).reshape(g.node_shape)
    a0 = g.split_q(a)[0]
    s0 = a0.reshape(T, -1).sum(axis=1)
    prev = np.concatenate([[0.0], s0])
    cur = np.concatenate([s0, [0.0]])
    np.testing.assert_allclose(out.reshape(T + 1, -1).sum(axis=1), (prev - cur) * T, atol=1e-10)


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_adjoint_pairs(D, T, N):
    g = O.Grid(D, T, N)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(g.n_nodes), rng.standard_normal(g.n_q)
    assert np.isclose(O.apply_A(g, x) @ y, x @ O.apply_At(g, y), rtol=1e-12)
    for fam in range(D + 1):
        v = rng.standard_normal(g.face_sizes[fam])
        assert np.isclose(O.apply_L(g, fam, x) @ v, x @ O.apply_Lt(g, fam, v), rtol=1e-12)
    u = rng.standard_normal((g.K - 1) * g.n_cones)
    assert np.isclose(O.apply_F(g, y) @ u, y @ O.apply_Ft(g, u), rtol=1e-12)
    w = rng.uniform(0.1, 2.0, g.n_cones)
    z = rng.standard_normal(g.K * g.n_cones)
    assert np.isclose(O.apply_B(g, w, u) @ z, u @ O.apply_Bt(g, w, z), rtol=1e-12)


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_L_exact_on_linear_functions(D, T, N):
    """An average of two neighbours of a linear function is its value at the midpoint."""
    g = O.Grid(D, T, N)
    X = node_coords(g)
    coef = [0.5, 1.0, -2.0, 3.0][: D + 1]
    phi = 0.3 + sum(c * x for c, x in zip(coef, X))
    for fam in range(D + 1):
        out = O.apply_L(g, fam, phi).reshape(g.face_shape(fam))
        shifted = [x.copy() for x in X]
        sl = [slice(None)] * (D + 1)
        sl[fam] = slice(0, -1)
        mid = 0.3
        for a in range(D + 1):
            xa = X[a][tuple(sl)]
            if a == fam:
                xa = xa + 0.5 * g.h[a]
            mid = mid + coef[a] * xa
        np.testing.assert_allclose(out, mid, atol=1e-12)


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_identity_LT_LXstar_equals_quarter_sum_F(D, T, N):
    """eq. (f1vf2v): L_T L_X^*(q_1; ...; q_D) = 1/4 sum_d sum_v F^d_v q_d."""
    g = O.Grid(D, T, N)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(g.n_q)
    qb = g.split_q(q)
    lhs_nodes = sum(O.apply_Lt(g, d, qb[d].ravel()) for d in range(1, D + 1))
    lhs = O.apply_L(g, 0, lhs_nodes)
    Fq = O.apply_F(g, q).reshape(g.K - 1, g.n_cones)
    rhs = 0.25 * Fq[1:].sum(axis=0)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    np.testing.assert_array_equal(Fq[0], qb[0].ravel())   # F_0 is the identity


@pytest.mark.parametrize("D,T,N", GRIDS)
def test_FBBF_is_diagonal_with_paper_values(D, T, N):
    """Proposition 3.2 / eq. (FFF): F^*B^*BF = diag(2 on q_0; 1 at i_0 in {0, n_0}, 2 inside on q_d)."""
    g = O.Grid(D, T, N)
    w = np.ones(g.n_cones)
    cols = []
    for e in np.eye(g.n_q):
        cols.append(O.apply_Ft(g, O.apply_Bt(g, w, O.apply_B(g, w, O.apply_F(g, e)))))
    M = np.stack(cols, axis=1)
    assert np.max(np.abs(M - np.diag(np.diag(M)))) == 0.0
    dg = g.split_q(np.diag(M).copy())
    # exact up to the rounding of sqrt(1/2)^2
    np.testing.assert_allclose(dg[0], 2.0, rtol=1e-15)
    for d in range(1, D + 1):
        expect = np.full(g.face_shape(d), 2.0)
        expect[0] = 1.0
        expect[-1] = 1.0
        np.testing.assert_allclose(dg[d], expect, rtol=1e-15)


@pytest.mark.parametrize("D,T,N", GRIDS)
@pytest.mark.parametrize("weighted", [False, True])
def test_cone_membership_equals_P(D, T, N, weighted):
    """eq. (socobservation): B F q + d in Q  <=>  q_0 + 1/2 omega L_T L_X^*(|qbar|^2) <= 0."""
    g = O.Grid(D, T, N)
    rng = np.random.default_rng(4)
    w = rng.choice([1.0, 1e-6, 0.3], size=g.n_cones) if weighted else np.ones(g.n_cones)
    for trial in range(20):
        q = rng.standard_normal(g.n_q) * 0.5
        qb = g.split_q(q)
        sq = sum(O.apply_Lt(g, d, qb[d].ravel() ** 2) for d in range(1, D + 1))
        f = qb[0].ravel() + 0.5 * w * O.apply_L(g, 0, sq)
        y = (O.apply_B(g, w, O.apply_F(g, q)) + O.fill_d(g)).reshape(g.K, g.n_cones)
        in_cone = y[0] - np.linalg.norm(y[1:], axis=0)
        # same sign up to rounding; the two sides differ by a positive factor
        # ((1-x0)^2 - (1+x0)^2 - ... = -4 f), so compare signs away from 0
        sel = np.abs(f) > 1e-9
        assert np.all((in_cone[sel] >= 0) == (f[sel] <= 0))


def test_c_vector_densities():
    """eq. (defc): rho_0 on the first time slice, minus rho_1 on the last, as cell-average
    densities (mass / cell area); zero in between."""
    g = O.Grid(2, 3, [4, 5])
    rng = np.random.default_rng(5)
    m0, m1 = rng.random(20), rng.random(20)
    c = O.fill_c(g, m0, m1).reshape(g.node_shape)
    np.testing.assert_allclose(c[0].ravel(), m0 * 20, rtol=1e-15)
    np.testing.assert_allclose(c[-1].ravel(), -m1 * 20, rtol=1e-15)
    assert np.all(c[1:-1] == 0)
