"""Pins for the oracle's stopping and penalty-rule measures (Sec. 5.3).

og_kkt returns eta_P, eta_D, eta_C (the KKT system of problem (8)) and eta_P^soc,
eta_D^soc (the KKT system of the SOCP (opt-dualsoc)), which decide every change of
sigma.  Each measure is checked here against a value fixed by the definitions alone:

* a "consistent" state built with independent dense operators (tests/bruteforce.py:
  A from eq. (Amap), F from eq. (operatorF)/(fdetails) by matching cone and face
  positions, B from eq. (bdd) with the weight sqrt(omega/2) of P_omega, Sec. 5.4):
  q = A phi, z = B F q + d, beta solving A^* F^* B^* beta = c and alpha = -F^* B^* beta.
  There every residual the measures contain vanishes, so eta_P, eta_D, eta_P^soc and
  eta_D^soc must be zero up to rounding;
* single-entry perturbations of that state, for which the numerator of each measure
  is known in closed form (one entry of size delta times the volume weight of the
  discrete L2 norm, sqrt(h_0 h_1 h_2), times the weight the perturbed entry carries in
  B, F or A).  A wrong weight, a missing omega, a dropped component of B or B^*, or a
  wrong boundary rule of F changes the value;
* eta_C at the independent optimum of problem (8) (barrier method), perturbed in
  q_0 (the complementarity part, including the max(0, .) of its definition) and in
  alpha_d (the g_d part).
"""
import numpy as np
import pytest

import oracle as O
from bruteforce import DenseDOT, DenseSOC
from test_oracle_solve import CASES

GRIDS = [(4, [4, 4]), (3, [5, 4])]


def _l2(g, v):
    """Discrete L2 norm: every entry carries one space-time cell volume (Sec. 5.3)."""
    return np.sqrt(g.vol * np.sum(np.asarray(v) ** 2))


class Consistent:
    """A state at which z = B F q + d, q = A phi and A^* alpha + c = 0 = alpha + F^* B^* beta."""

    def __init__(self, T, N, seed):
        rng = np.random.default_rng(seed)
        self.g = g = O.Grid(2, T, N)
        self.dd = dd = DenseDOT(2, T, N)
        self.ds = ds = DenseSOC(2, T, N)
        assert ds.n0 == g.n_cones and ds.nq == g.n_q
        P = N[0] * N[1]
        m0, m1 = rng.random(P) + 0.1, rng.random(P) + 0.1
        self.prob = O.Problem(g, m0, m1)
        # omega: arbitrary positive weights per cone, two of them the obstacle value
        om = rng.uniform(0.2, 1.0, g.n_cones)
        om[[3, 17]] = 1e-6
        self.prob.omega = om
        A = np.vstack(dd.A)
        F, B, d = ds.F, ds.B(om), ds.d()
        self.A, self.F, self.B, self.dv = A, F, B, d
        phi = rng.standard_normal(g.n_nodes)
        phi -= phi.mean()
        q = A @ phi
        z = B @ (F @ q) + d
        M = A.T @ F.T @ B.T
        beta = np.linalg.lstsq(M, self.prob.c, rcond=None)[0]
        # plus an arbitrary element of ker M: beta is not unique
        r = rng.standard_normal(M.shape[1])
        beta += r - np.linalg.pinv(M, rcond=1e-10) @ (M @ r)
        assert np.abs(M @ beta - self.prob.c).max() <= 1e-9 * np.abs(self.prob.c).max()
        alpha = -F.T @ (B.T @ beta)
        st = O.State.zeros(g)
        st.phi, st.q, st.z, st.alpha, st.beta = phi, q, z, alpha, beta
        self.st = st

    def FtBt(self, beta):
        return self.F.T @ (self.B.T @ beta)


@pytest.fixture(params=GRIDS, ids=["4x4x4", "3x5x4"])
def cons(request):
    T, N = request.param
    return Consistent(T, N, seed=7 + T)


def test_measures_vanish_at_consistent_state(cons):
    kk = O.kkt(cons.prob, cons.st)
    assert kk["eta_P"] <= 1e-14
    assert kk["eta_D"] <= 1e-12
    assert kk["eta_P_soc"] <= 1e-14
    assert kk["eta_D_soc"] <= 1e-12


def test_eta_P_soc_z_perturbation(cons):
    """z_j += delta in one cone: the second term of eta_P^soc is sqrt(V) delta / (1 + ||d||)
    with ||d|| = sqrt(V 2 n_0); eta_P, eta_D, eta_D^soc do not see z."""
    g, st = cons.g, cons.st
    V, n0, delta = g.vol, g.n_cones, 3e-3
    for j, c in ((0, 5), (4, 9), (g.K - 1, 0)):
        s = st.copy()
        s.z[j * n0 + c] += delta
        kk = O.kkt(cons.prob, s)
        want = np.sqrt(V) * delta / (1.0 + np.sqrt(V * 2 * n0))
        assert kk["eta_P_soc"] == pytest.approx(want, rel=1e-10)
        assert kk["eta_P"] <= 1e-14 and kk["eta_D_soc"] <= 1e-12


def test_eta_P_soc_q0_perturbation(cons):
    """q_0 += delta in one cone: B F moves components 0 and K-1 of that cone by -delta and
    +delta, so the SOC term is sqrt(2V) delta / (1 + ||d||); eta_P is sqrt(V) delta over its
    own denominator."""
    g, st = cons.g, cons.st
    V, n0, delta = g.vol, g.n_cones, 2e-3
    c = 11
    s = st.copy()
    s.q[c] += delta
    kk = O.kkt(cons.prob, s)
    Aphi = cons.A @ st.phi
    etaP = np.sqrt(V) * delta / (1.0 + _l2(g, Aphi) + _l2(g, s.q))
    soc = np.sqrt(2 * V) * delta / (1.0 + np.sqrt(V * 2 * n0))
    assert kk["eta_P"] == pytest.approx(etaP, rel=1e-10)
    assert kk["eta_P_soc"] == pytest.approx(max(etaP, soc), rel=1e-10)
    assert soc > etaP


def test_eta_P_soc_space_face_perturbation(cons):
    """q_d += delta on one space face: F copies it into one slot of every cone that reads
    the face (found here from positions alone), B scales it by sqrt(omega_c / 2), so the
    SOC numerator is delta sqrt(V sum_c omega_c / 2)."""
    g, st, ds = cons.g, cons.st, cons.ds
    V, n0, delta = g.vol, g.n_cones, 2e-3
    om = cons.prob.omega
    checked = 0
    for (fam, pos), col in ds.face_index.items():
        if fam == 0 or col % 7:
            continue
        cones = ds.cones_reading_face(fam, pos)
        s = st.copy()
        s.q[col] += delta
        kk = O.kkt(cons.prob, s)
        soc = delta * np.sqrt(V * sum(om[c] / 2.0 for c in cones)) / (1.0 + np.sqrt(V * 2 * n0))
        etaP = np.sqrt(V) * delta / (1.0 + _l2(g, cons.A @ st.phi) + _l2(g, s.q))
        assert kk["eta_P_soc"] == pytest.approx(max(etaP, soc), rel=1e-10), (fam, pos, cones)
        checked += 1
    assert checked >= 10


def test_eta_P_phi_perturbation(cons):
    """phi += delta at one interior node: A puts +-delta/h_f on each of its faces (two per
    axis), so eta_P = delta sqrt(V sum_f 1/h_f^2) / (1 + ||A phi|| + ||q||), while z = B F q + d
    still holds: eta_P^soc takes eta_P through its max."""
    g, st = cons.g, cons.st
    V, delta = g.vol, 1e-3
    node = (1, 1, 2)
    k = int(np.ravel_multi_index(node, g.node_shape))
    s = st.copy()
    s.phi[k] += delta
    kk = O.kkt(cons.prob, s)
    inv_h2 = 2 * (g.T ** 2 + g.N[0] ** 2 + g.N[1] ** 2)
    etaP = delta * np.sqrt(V * inv_h2) / (1.0 + _l2(g, cons.A @ s.phi) + _l2(g, st.q))
    assert kk["eta_P"] == pytest.approx(etaP, rel=1e-10)
    assert kk["eta_P_soc"] == pytest.approx(etaP, rel=1e-10)


def test_eta_D_soc_beta_perturbations(cons):
    """beta += delta in one slot: B^* F^* maps components 0 and K-1 to q_0 with opposite
    signs, component j = 1 + 4(d-1) + (v-1) to the face F^d_v reads with weight
    sqrt(omega/2), and nothing where F^d_v is zero at the wall."""
    g, st, ds = cons.g, cons.st, cons.ds
    V, n0, K, delta = g.vol, g.n_cones, g.K, 4e-3
    om = cons.prob.omega

    def eta_dsoc(beta):
        s = st.copy()
        s.beta = beta
        return O.kkt(cons.prob, s)["eta_D_soc"]

    def denom(beta):
        return 1.0 + _l2(g, cons.FtBt(beta)) + _l2(g, st.alpha)

    # components 0 and K-1 together cancel in B^*
    c = 6
    b = st.beta.copy()
    b[c] += delta
    b[(K - 1) * n0 + c] += delta
    assert eta_dsoc(b) <= 1e-12
    # component 0 alone
    b = st.beta.copy()
    b[c] += delta
    assert eta_dsoc(b) == pytest.approx(np.sqrt(V) * delta / denom(b), rel=1e-10)
    # components 1..4D: present or absent source face, by position
    hits = misses = 0
    for c in (0, 5, n0 - 1):
        for j in range(1, K - 1):
            d, v = 1 + (j - 1) // 4, (j - 1) % 4
            dt, dx = ((-0.5, -0.5), (-0.5, 0.5), (0.5, -0.5), (0.5, 0.5))[v]
            src = list(ds.cone_pos[c])
            src[0] += dt
            src[d] += dx
            b = st.beta.copy()
            b[j * n0 + c] += delta
            if (d, tuple(src)) in ds.face_index:
                want = np.sqrt(V) * np.sqrt(om[c] / 2.0) * delta / denom(b)
                assert eta_dsoc(b) == pytest.approx(want, rel=1e-10), (c, j)
                hits += 1
            else:
                assert eta_dsoc(b) <= 1e-12, (c, j)
                misses += 1
    assert hits and misses


def test_eta_D_and_D_soc_alpha_perturbation(cons):
    """alpha_0 += delta in one cone: A^* puts +-delta/h_0 on the two nodes of that time
    face (eta_D = sqrt(2V) delta T / (1 + ||c||)); the SOC term is sqrt(V) delta over
    1 + ||F^* B^* beta|| + ||alpha||."""
    g, st = cons.g, cons.st
    V, delta = g.vol, 1e-3
    s = st.copy()
    s.alpha[13] += delta
    kk = O.kkt(cons.prob, s)
    etaD = np.sqrt(2 * V) * delta * g.T / (1.0 + _l2(g, cons.prob.c))
    dsoc = np.sqrt(V) * delta / (1.0 + _l2(g, cons.FtBt(st.beta)) + _l2(g, s.alpha))
    assert kk["eta_D"] == pytest.approx(etaD, rel=1e-9)
    assert kk["eta_D_soc"] == pytest.approx(max(etaD, dsoc), rel=1e-9)
    # and a space face: A^* puts +-delta/h_d on the two nodes of the face
    s = st.copy()
    col = g.n_cones + 8
    s.alpha[col] += delta
    kk = O.kkt(cons.prob, s)
    etaD = np.sqrt(2 * V) * delta * g.N[0] / (1.0 + _l2(g, cons.prob.c))
    assert kk["eta_D"] == pytest.approx(etaD, rel=1e-9)


def test_eta_dot_is_max_of_three(cons):
    s = cons.st.copy()
    s.q[2] += 1e-3
    s.alpha[40] -= 2e-3
    kk = O.kkt(cons.prob, s)
    assert kk["eta_dot"] == max(kk["eta_P"], kk["eta_D"], kk["eta_C"])


# ---- eta_C at the independent optimum of problem (8) -----------------------

def _optimum(case):
    rng = np.random.default_rng({"random": 51, "zeros": 52, "obstacle": 53}[case])
    r0, r1, mask = CASES[case](rng)
    g = O.Grid(2, 4, [4, 4])
    prob = O.Problem(g, r0, r1, mask)
    dd = DenseDOT(2, 4, [4, 4])
    phi_b, q_b, lam = dd.barrier_solve(prob.c, prob.omega)
    st = O.State.zeros(g)
    st.phi = phi_b.copy()
    st.q = np.concatenate(q_b)
    st.alpha = np.concatenate(dd.alpha_from(lam, q_b, prob.omega))
    f, _ = dd.f(phi_b, prob.omega)
    return g, prob, st, dd, f


@pytest.mark.parametrize("case", ["random", "obstacle"])
def test_eta_C_complementarity_part(case):
    """At the optimum with rho > 0 every constraint is active (f = 0).  q_0 += delta at one
    cone raises f there by delta (q_0 enters only its own f), and with alpha_0 + f > 0 the
    residual alpha_0 - max(0, f + alpha_0) is -delta there: eta_C = sqrt(V) delta /
    (1 + ||alpha_0|| + ||f||), ||f|| = sqrt(V) delta."""
    g, prob, st, dd, f = _optimum(case)
    V, delta = g.vol, 1e-2
    a0 = st.alpha[: g.n_cones]
    c = int(np.argmax(a0))
    assert a0[c] > 0.1
    assert O.kkt(prob, st)["eta_C"] <= 1e-8
    s = st.copy()
    s.q[c] += delta
    kk = O.kkt(prob, s)
    want = np.sqrt(V) * delta / (1.0 + _l2(g, a0) + np.sqrt(V) * delta)
    assert kk["eta_C"] == pytest.approx(want, rel=1e-5)


def test_eta_C_max_zero_branch():
    """A cone with alpha_0 = 0 (no mass) and f < 0 has alpha_0 - max(0, f + alpha_0) = 0:
    eta_C stays at the optimum's level however negative f is, where the same formula
    without max(0, .) would give |f|.  Raising f to delta > 0 makes that entry -delta.
    The momenta are reset to g(alpha_0, q_bar) (dense, eq. of Sec. 5.3) so that the g_d
    part of eta_C stays zero."""
    g, prob, st, dd, f = _optimum("random")
    V = g.vol
    c = 9
    a0 = st.alpha[: g.n_cones].copy()
    a0[c] = 0.0
    qbar = dd.f(st.phi, prob.omega)[1]
    s0 = st.copy()
    s0.alpha = np.concatenate(dd.alpha_from(a0, qbar, prob.omega))
    s = s0.copy()
    s.q[c] -= 0.5                     # f_c = -0.5
    assert O.kkt(prob, s)["eta_C"] <= 1e-8
    delta = 1e-2
    s = s0.copy()
    s.q[c] += delta - f[c]            # f_c = delta
    fn = f.copy()
    fn[c] = delta
    want = np.sqrt(V) * delta / (1.0 + _l2(g, a0) + _l2(g, fn))
    assert O.kkt(prob, s)["eta_C"] == pytest.approx(want, rel=1e-5)


@pytest.mark.parametrize("case", ["random", "obstacle"])
def test_eta_C_momentum_part(case):
    """alpha_d += delta on one space face: the residual alpha_bar - g(alpha_0, q_bar) is delta
    there, so eta_C = sqrt(V) delta / (1 + ||alpha_bar|| + ||g||), g unchanged by alpha_d."""
    g, prob, st, dd, f = _optimum(case)
    V, delta = g.vol, 1e-2
    col = g.n_cones + 17
    s = st.copy()
    s.alpha[col] += delta
    kk = O.kkt(prob, s)
    gq = np.concatenate(dd.alpha_from(st.alpha[: g.n_cones], dd.f(st.phi, prob.omega)[1], prob.omega)[1:])
    want = np.sqrt(V) * delta / (1.0 + _l2(g, s.alpha[g.n_cones:]) + _l2(g, gq))
    assert kk["eta_C"] == pytest.approx(want, rel=1e-5)
