"""CPU checks of dot_prolong_state, the interpolation of the multilevel strategy
(Sec. 5): piecewise-linear interpolation reproduces affine fields between the
coarse samples, fine samples that coincide with coarse ones keep their values,
space faces keep zero flux at the walls, alpha and beta scale like h_0, and a
grid onto itself is the identity."""
import numpy as np
import pytest

from paper_2505_05424_gb300 import _native as N
from paper_2505_05424_gb300.solver import DotError, dot_prolong_state


@pytest.fixture(scope="module", autouse=True)
def lib():
    N.build()
    return N.load()


def fam_shapes(D, T, Ns):
    shapes = [(T,) + tuple(Ns)]
    for d in range(D):
        s = [T + 1] + list(Ns)
        s[1 + d] -= 1
        shapes.append(tuple(s))
    return shapes


def split(v, shapes):
    out, off = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(v[off:off + n].reshape(s))
        off += n
    return out


def centres(n):
    return (np.arange(n) + 0.5) / n


def test_affine_time_faces_reproduced_inside_the_coarse_hull():
    D, Tc, Nc, Tf, Nf = 2, 4, [6, 5], 8, [12, 10]
    a, b, c, d = 0.3, -1.2, 0.7, 2.1
    tc, xc, yc = centres(Tc), centres(Nc[0]), centres(Nc[1])
    q0c = a + b * tc[:, None, None] + c * xc[None, :, None] + d * yc[None, None, :]
    shc = fam_shapes(D, Tc, Nc)
    nq = sum(int(np.prod(s)) for s in shc)
    q = np.zeros(nq)
    q[:q0c.size] = q0c.ravel()
    K = 4 * D + 2
    beta = np.concatenate([q0c.ravel() * (k + 1) for k in range(K)])
    qf, af, bf = dot_prolong_state(D, Tc, Nc, Tf, Nf, q, q, beta)
    q0f = split(qf, fam_shapes(D, Tf, Nf))[0]
    tf, xf, yf = centres(Tf), centres(Nf[0]), centres(Nf[1])
    exact = a + b * tf[:, None, None] + c * xf[None, :, None] + d * yf[None, None, :]
    inside = ((tf >= tc[0]) & (tf <= tc[-1]))[:, None, None] & ((xf >= xc[0]) & (xf <= xc[-1]))[None, :, None] \
        & ((yf >= yc[0]) & (yf <= yc[-1]))[None, None, :]
    np.testing.assert_allclose(q0f[inside], exact[inside], rtol=0, atol=1e-13)
    # alpha and beta: the same interpolant times T_coarse / T_fine
    a0f = split(af, fam_shapes(D, Tf, Nf))[0]
    np.testing.assert_allclose(a0f, 0.5 * q0f, rtol=0, atol=1e-15)
    bfs = bf.reshape(K, -1)
    for k in range(K):
        np.testing.assert_allclose(bfs[k], 0.5 * (k + 1) * q0f.ravel(), rtol=1e-15, atol=1e-14)
    # before the first coarse time centre the interpolant is constant in time
    sp = ((xf >= xc[0]) & (xf <= xc[-1]))[:, None] & ((yf >= yc[0]) & (yf <= yc[-1]))[None, :]
    at_first = a + b * tc[0] + c * xf[:, None] + d * yf[None, :]
    assert tf[0] < tc[0]
    np.testing.assert_allclose(q0f[0][sp], at_first[sp], rtol=0, atol=1e-13)


def test_space_faces_keep_coarse_values_and_zero_walls():
    D, Tc, Nc, Tf, Nf = 2, 3, [4, 6], 6, [8, 12]
    shc, shf = fam_shapes(D, Tc, Nc), fam_shapes(D, Tf, Nf)
    rng = np.random.default_rng(11)
    nq = sum(int(np.prod(s)) for s in shc)
    q = rng.standard_normal(nq)
    qf, _, _ = dot_prolong_state(D, Tc, Nc, Tf, Nf, q, q, np.zeros(10 * Tc * 24))
    qc1, qf1 = split(q, shc)[1], split(qf, shf)[1]      # x-faces: [T+1][N1-1][N2]
    # fine time node 2k is coarse node k; fine face 2j+1 (position (j+1)/Nc) is coarse face j
    yc, yf = centres(Nc[1]), centres(Nf[1])
    for k in range(Tc + 1):
        for j in range(Nc[0] - 1):
            row = qf1[2 * k, 2 * j + 1]
            # along y (cell centres) the fine row interpolates the coarse row linearly
            np.testing.assert_allclose(row, np.interp(yf, yc, qc1[k, j]), rtol=0, atol=1e-13)
    # fine faces next to a wall: halfway between the wall's zero and the first coarse face
    for k in range(Tc + 1):
        np.testing.assert_allclose(qf1[2 * k, 0], 0.5 * np.interp(yf, yc, qc1[k, 0]), rtol=0, atol=1e-13)
        np.testing.assert_allclose(qf1[2 * k, -1], 0.5 * np.interp(yf, yc, qc1[k, -1]), rtol=0, atol=1e-13)
    # odd fine time nodes average their two coarse neighbours
    np.testing.assert_allclose(qf1[1], 0.5 * (qf1[0] + qf1[2]), rtol=0, atol=1e-13)


def test_same_grid_is_identity_and_bad_grids_are_rejected():
    D, T, Ns = 3, 2, [3, 4, 2]
    rng = np.random.default_rng(5)
    nq = sum(int(np.prod(s)) for s in fam_shapes(D, T, Ns))
    nb = (4 * D + 2) * T * int(np.prod(Ns))
    q, al, be = rng.standard_normal(nq), rng.standard_normal(nq), rng.standard_normal(nb)
    qf, af, bf = dot_prolong_state(D, T, Ns, T, Ns, q, al, be)
    np.testing.assert_array_equal(qf, q)
    np.testing.assert_array_equal(af, al)
    np.testing.assert_array_equal(bf, be)
    with pytest.raises(DotError):
        dot_prolong_state(2, 4, [8, 8], 2, [8, 8], np.zeros(1000), np.zeros(1000), np.zeros(10000))
