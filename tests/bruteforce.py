"""Independent dense reference for tiny grids: problem (8) by a log-barrier Newton method.

Written from the problem statement alone (eq. (Amap), (ltlx), (defc), (defp) and the
weighted set P_omega of Sec. 5.4) with explicit dense matrices; it shares nothing with
the oracle.  Used by the tests to pin the oracle's fixed point.
"""
import numpy as np


class DenseDOT:
    """Dense matrices of the discretisation for D spatial axes, N cells each, T intervals."""

    def __init__(self, D, T, N):
        self.D, self.T, self.N = D, T, list(N)
        self.node_shape = (T + 1,) + tuple(N)
        self.nn = int(np.prod(self.node_shape))
        idx = np.arange(self.nn).reshape(self.node_shape)
        h = [1.0 / T] + [1.0 / n for n in N]
        self.h = h
        self.A, self.L = [], []          # A_f and L_f (f = 0: time faces), dense rows
        for f in range(D + 1):
            lo = np.take(idx, np.arange(self.node_shape[f] - 1), axis=f).ravel()
            hi = np.take(idx, np.arange(1, self.node_shape[f]), axis=f).ravel()
            A = np.zeros((lo.size, self.nn))
            L = np.zeros((lo.size, self.nn))
            A[np.arange(lo.size), hi] += 1.0 / h[f]
            A[np.arange(lo.size), lo] -= 1.0 / h[f]
            L[np.arange(lo.size), hi] += 0.5
            L[np.arange(lo.size), lo] += 0.5
            self.A.append(A)
            self.L.append(L)
        # M_d = L_T L_X^{d*}: time-face x d-face
        self.M = [self.L[0] @ self.L[d].T for d in range(1, D + 1)]
        self.ncone = self.A[0].shape[0]

    def c(self, m0, m1):
        """eq. (defc) with the data as cell-average densities (mass / cell area)."""
        area = float(np.prod([1.0 / n for n in self.N]))
        c = np.zeros(self.node_shape)
        c[0] = np.asarray(m0).reshape(self.N) / area
        c[-1] = -np.asarray(m1).reshape(self.N) / area
        return c.ravel()

    def f(self, phi, omega):
        """Constraint values q_0 + 1/2 omega L_T L_X^*(|q_d|^2) per cone, with q = A phi."""
        q = [A @ phi for A in self.A]
        return q[0] + 0.5 * omega * sum(M @ (qd * qd) for M, qd in zip(self.M, q[1:])), q

    def barrier_solve(self, c, omega, gap=1e-10, mu=8.0, zeta=1.0):
        """min <c, phi> s.t. f(phi) <= 0 by the barrier method, phi restricted to mean zero.

        Start: the paper's strictly feasible phi*(i_0) = -h_0 (i_0 + 1) zeta (Prop. 3.1)."""
        T = self.T
        phi = (-(np.arange(T + 1) + 1.0) / T * zeta)[:, None] * np.ones((1, self.nn // (T + 1)))
        phi = phi.ravel()
        phi -= phi.mean()
        # orthonormal basis of the mean-zero subspace
        Q = np.linalg.qr(np.eye(self.nn) - 1.0 / self.nn, mode="reduced")[0][:, : self.nn - 1]
        m = self.ncone
        t = 1.0
        while True:
            for _newton in range(200):
                fv, q = self.f(phi, omega)
                s = -fv
                # gradient rows of f_i: A_0 + omega_i sum_d diag(M_d q_d) ... (chain rule)
                Jf = self.A[0].copy()
                for M, Ad, qd in zip(self.M, self.A[1:], q[1:]):
                    Jf += omega[:, None] * (M * qd[None, :]) @ Ad
                grad = t * c + Jf.T @ (1.0 / s)
                H = Jf.T @ (Jf / (s * s)[:, None])
                for M, Ad in zip(self.M, self.A[1:]):
                    wrow = (omega / s) @ M            # sum_i (omega_i / s_i) M_d[i, :]
                    H += Ad.T @ (wrow[:, None] * Ad)
                gr, Hr = Q.T @ grad, Q.T @ H @ Q
                dx = -np.linalg.solve(Hr, gr)
                dec = -gr @ dx
                if dec / 2 < 1e-14:
                    break
                step = Q @ dx
                a = 1.0
                obj0 = t * c @ phi - np.log(s).sum()
                while True:
                    cand = phi + a * step
                    fc, _ = self.f(cand, omega)
                    if np.all(fc < 0) and t * c @ cand - np.log(-fc).sum() <= obj0 - 0.25 * a * dec:
                        break
                    a *= 0.5
                    if a < 1e-14:
                        break
                phi = cand
            if m / t < gap:
                break
            t *= mu
        fv, q = self.f(phi, omega)
        # Multipliers Lambda_0 (= alpha_0) from the stationarity condition of (8),
        # c + sum_i Lambda_i grad f_i(phi) = 0, in the least-squares sense at the
        # barrier's phi.  The central-path estimate 1/(t(-f_i)) loses digits at large
        # t (cancellation in f), the least-squares one does not.
        Jf = self.A[0].copy()
        for M, Ad, qd in zip(self.M, self.A[1:], q[1:]):
            Jf += omega[:, None] * (M * qd[None, :]) @ Ad
        lam = np.linalg.lstsq(Jf.T, -c, rcond=None)[0]
        return phi, q, lam

    def alpha_from(self, lam, q, omega):
        """alpha = (Lambda_0; (L_X^d L_T^*(omega Lambda_0)) o q_d) -- stationarity of (8)."""
        return [lam] + [(M.T @ (omega * lam)) * qd for M, qd in zip(self.M, q[1:])]


class DenseSOC:
    """Dense F (eq. (operatorF), (fdetails)), B (eq. (bdd), weighted by sqrt(omega/2) as for
    P_omega in Sec. 5.4) and d for the SOCP reformulation (opt-dualsoc).

    Written from the definitions by placing every cone and face at its space-time
    position (index units: node (t, x), time face (t + 1/2, x), space face of axis d at
    x_d + 1/2) and matching positions, so no index arithmetic is shared with the oracle.
    F^d_v of the cone at (t + 1/2, x) is q_d at (t, x_d - 1/2), (t, x_d + 1/2),
    (t + 1, x_d - 1/2), (t + 1, x_d + 1/2) for v = 1..4, and 0 where no such face exists.
    Layouts follow the oracle's interface: q = (q_0; q_1; ..; q_D) with each block in
    C order, cone vectors block-major (component, cone)."""

    def __init__(self, D, T, N):
        self.D, self.T, self.N = D, T, list(N)
        self.K = 4 * D + 2
        cone_shape = (T,) + tuple(N)
        self.cone_pos = [(t + 0.5,) + tuple(float(v) for v in x)
                         for t, *x in np.ndindex(*cone_shape)]
        self.n0 = len(self.cone_pos)
        # faces: family 0 are the cones' own time faces; family d has N_d - 1 faces along d
        self.face_index = {}                   # (family, position) -> column of q
        col = 0
        for t, *x in np.ndindex(*cone_shape):
            self.face_index[(0, (t + 0.5,) + tuple(float(v) for v in x))] = col
            col += 1
        for d in range(1, D + 1):
            shape = [T + 1] + list(N)
            shape[d] -= 1
            for idx in np.ndindex(*shape):
                pos = [float(v) for v in idx]
                pos[d] += 0.5
                self.face_index[(d, tuple(pos))] = col
                col += 1
        self.nq = col
        self.F = np.zeros(((self.K - 1) * self.n0, self.nq))
        for c, pos in enumerate(self.cone_pos):
            self.F[c, self.face_index[(0, pos)]] = 1.0
            for d in range(1, D + 1):
                for v, (dt, dx) in enumerate(((-0.5, -0.5), (-0.5, 0.5), (0.5, -0.5), (0.5, 0.5))):
                    src = list(pos)
                    src[0] += dt
                    src[d] += dx
                    j = self.face_index.get((d, tuple(src)))
                    if j is not None:
                        self.F[(1 + 4 * (d - 1) + v) * self.n0 + c, j] = 1.0

    def B(self, omega):
        """x = (x_0; x_1..x_4D) per cone -> (-x_0; s x_1; ..; s x_4D; x_0), s = sqrt(omega/2)."""
        n0, K = self.n0, self.K
        s = np.sqrt(np.asarray(omega, dtype=float) / 2.0)
        B = np.zeros((K * n0, (K - 1) * n0))
        for c in range(n0):
            B[c, c] = -1.0
            for j in range(1, K - 1):
                B[j * n0 + c, j * n0 + c] = s[c]
            B[(K - 1) * n0 + c, c] = 1.0
        return B

    def d(self):
        v = np.zeros(self.K * self.n0)
        v[: self.n0] = 1.0
        v[(self.K - 1) * self.n0:] = 1.0
        return v

    def cones_reading_face(self, d, face_pos):
        """Cones whose F^d_v reads the space face at face_pos (explicit geometry: cone
        times t - 1/2 and t + 1/2 of the face's time node t, cells x_d -+ 1/2 along d)."""
        out = []
        for dt in (-0.5, 0.5):
            for dx in (-0.5, 0.5):
                p = list(face_pos)
                p[0] += dt
                p[d] += dx
                p = tuple(p)
                if 0 < p[0] < self.T and all(0 <= p[a] <= self.N[a - 1] - 1 for a in range(1, self.D + 1)):
                    out.append(self.cone_pos.index(p))
        return out
