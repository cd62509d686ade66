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
