"""Test infrastructure: the FP64 CPU oracle for the inexact proximal ALM.

A plain, slow restatement of Algorithm 2 (Sec. 4) for the SOCP reformulation
(Sec. 3) of the staggered-grid dynamic OT problem (Sec. 2.2, eq. (8)), written in
C (``palm_oracle.c``) and called through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package; the product path never does, and this package imports nothing from it.

Layout (every array C-order, float64):
  nodes   [T+1, N_1, ..., N_D]
  q/alpha concatenation of G^s_0 [T, N_1..N_D] and G^s_d [T+1, .., N_d - 1, ..]
  beta/z  [K, T, N_1..N_D] with K = 4D + 2

Parity notes: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, library special cases or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "palm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpalm_oracle.so")

KKT_NAMES = ("eta_dot", "eta_P", "eta_D", "eta_C", "eta_P_soc", "eta_D_soc",
             "primal_obj", "dual_obj", "gap")
NUM_KKT = len(KKT_NAMES)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("T", ctypes.c_int), ("N", ctypes.c_int * 3)]


class _Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("sigma", ctypes.c_double)]


_lib = None
_P = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        G = ctypes.POINTER(_Grid)
        for name in ("og_num_nodes", "og_num_cones", "og_num_q"):
            getattr(lib, name).restype = ctypes.c_long
            getattr(lib, name).argtypes = [G]
        lib.og_num_faces.restype = ctypes.c_long
        lib.og_num_faces.argtypes = [G, ctypes.c_int]
        lib.og_cone_dim.restype = ctypes.c_int
        lib.og_cone_dim.argtypes = [G]
        for name in ("og_apply_A", "og_apply_At", "og_apply_F", "og_apply_Ft", "og_poisson",
                     "og_proj_Q"):
            getattr(lib, name).argtypes = [G, _P, _P]
        lib.og_apply_L.argtypes = [G, ctypes.c_int, _P, _P]
        lib.og_apply_Lt.argtypes = [G, ctypes.c_int, _P, _P]
        lib.og_apply_B.argtypes = [G, _P, _P, _P]
        lib.og_apply_Bt.argtypes = [G, _P, _P, _P]
        lib.og_fill_d.argtypes = [G, _P]
        lib.og_fill_c.argtypes = [G, _P, _P, _P]
        lib.og_proj_soc.argtypes = [ctypes.c_int, _P, _P]
        lib.og_dct_matrix.argtypes = [ctypes.c_int, _P]
        lib.og_dct_axis.argtypes = [G, ctypes.c_int, ctypes.c_int, _P, _P]
        lib.og_iterate.argtypes = [G, ctypes.POINTER(_Params), _P, _P, _P, _P, _P, _P, _P]
        lib.og_kkt.argtypes = [G, _P, _P, _P, _P, _P, _P, _P, _P]
        lib.og_solve.restype = ctypes.c_long
        lib.og_solve.argtypes = [G, ctypes.c_double, _P, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_double, ctypes.c_long, _P, _P, _P, _P,
                                 _P, _P, _P, _P, _P, ctypes.c_long,
                                 ctypes.POINTER(ctypes.c_long)]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """D spatial axes with N_d cells each (h_d = 1/N_d), T time intervals (h_0 = 1/T)."""

    def __init__(self, D: int, T: int, N):
        N = [int(N)] * D if np.isscalar(N) else [int(n) for n in N]
        assert 1 <= D <= 3 and len(N) == D and T >= 1 and all(n >= 2 for n in N)
        self.D, self.T, self.N = D, T, tuple(N)
        self._c = _Grid(D, T, (ctypes.c_int * 3)(*(N + [1] * (3 - D))))
        lib = _load()
        r = ctypes.byref(self._c)
        self.n_nodes = lib.og_num_nodes(r)
        self.n_cones = lib.og_num_cones(r)
        self.n_q = lib.og_num_q(r)
        self.K = lib.og_cone_dim(r)
        self.face_sizes = [lib.og_num_faces(r, f) for f in range(D + 1)]

    @property
    def ref(self):
        return ctypes.byref(self._c)

    @property
    def node_shape(self):
        return (self.T + 1,) + self.N

    def face_shape(self, fam: int):
        if fam == 0:
            return (self.T,) + self.N
        s = [self.T + 1] + list(self.N)
        s[fam] -= 1
        return tuple(s)

    @property
    def h(self):
        return (1.0 / self.T,) + tuple(1.0 / n for n in self.N)

    @property
    def vol(self) -> float:
        return float(np.prod(self.h))

    def split_q(self, q: np.ndarray):
        """Split a concatenated q-like vector into its D+1 shaped blocks (views)."""
        out, off = [], 0
        for f in range(self.D + 1):
            n = self.face_sizes[f]
            out.append(q[off:off + n].reshape(self.face_shape(f)))
            off += n
        return out


# ---- operators (thin wrappers) -------------------------------------------

def apply_A(g: Grid, phi):
    phi = _f64(phi).ravel()
    q = np.zeros(g.n_q)
    _load().og_apply_A(g.ref, _ptr(phi), _ptr(q))
    return q


def apply_At(g: Grid, q):
    q = _f64(q).ravel()
    out = np.zeros(g.n_nodes)
    _load().og_apply_At(g.ref, _ptr(q), _ptr(out))
    return out


def apply_L(g: Grid, fam: int, y):
    y = _f64(y).ravel()
    out = np.zeros(g.face_sizes[fam])
    _load().og_apply_L(g.ref, fam, _ptr(y), _ptr(out))
    return out


def apply_Lt(g: Grid, fam: int, v):
    v = _f64(v).ravel()
    out = np.zeros(g.n_nodes)
    _load().og_apply_Lt(g.ref, fam, _ptr(v), _ptr(out))
    return out


def apply_F(g: Grid, q):
    q = _f64(q).ravel()
    out = np.zeros((g.K - 1) * g.n_cones)
    _load().og_apply_F(g.ref, _ptr(q), _ptr(out))
    return out


def apply_Ft(g: Grid, u):
    u = _f64(u).ravel()
    out = np.zeros(g.n_q)
    _load().og_apply_Ft(g.ref, _ptr(u), _ptr(out))
    return out


def apply_B(g: Grid, omega, x):
    omega, x = _f64(omega).ravel(), _f64(x).ravel()
    out = np.zeros(g.K * g.n_cones)
    _load().og_apply_B(g.ref, _ptr(omega), _ptr(x), _ptr(out))
    return out


def apply_Bt(g: Grid, omega, u):
    omega, u = _f64(omega).ravel(), _f64(u).ravel()
    out = np.zeros((g.K - 1) * g.n_cones)
    _load().og_apply_Bt(g.ref, _ptr(omega), _ptr(u), _ptr(out))
    return out


def fill_d(g: Grid):
    out = np.zeros(g.K * g.n_cones)
    _load().og_fill_d(g.ref, _ptr(out))
    return out


def fill_c(g: Grid, m0, m1):
    """c of eq. (defc) from cell masses, as cell-average densities (see og_fill_c)."""
    m0, m1 = _f64(m0).ravel(), _f64(m1).ravel()
    out = np.zeros(g.n_nodes)
    _load().og_fill_c(g.ref, _ptr(m0), _ptr(m1), _ptr(out))
    return out


def proj_soc(y):
    y = _f64(y).ravel()
    z = np.zeros_like(y)
    _load().og_proj_soc(len(y), _ptr(y), _ptr(z))
    return z


def proj_Q(g: Grid, Y):
    Y = _f64(Y).ravel()
    Z = np.zeros_like(Y)
    _load().og_proj_Q(g.ref, _ptr(Y), _ptr(Z))
    return Z


def dct_matrix(M: int):
    C = np.zeros((M, M))
    _load().og_dct_matrix(M, _ptr(C))
    return C


def dct_axis(g: Grid, axis: int, x, inverse: bool = False):
    x = _f64(x).ravel()
    out = np.zeros_like(x)
    _load().og_dct_axis(g.ref, axis, int(inverse), _ptr(x), _ptr(out))
    return out


def poisson(g: Grid, b):
    b = _f64(b).ravel()
    phi = np.zeros(g.n_nodes)
    _load().og_poisson(g.ref, _ptr(b), _ptr(phi))
    return phi


# ---- problem set-up and the solve loop -----------------------------------

def masses(rho) -> np.ndarray:
    """Cell masses from a non-negative density sample: rho / sum(rho) (eq. (defc))."""
    rho = _f64(rho)
    s = rho.sum()
    if not np.isfinite(s) or s <= 0 or np.any(rho < 0):
        raise ValueError("density must be non-negative with positive finite mass")
    return rho / s


def omega_from_mask(g: Grid, mask, weight: float = 1e-6) -> np.ndarray:
    """omega on G^s_0: `weight` on obstacle cells, 1 elsewhere, constant in time (Sec. 5.4)."""
    if mask is None:
        return np.ones(g.n_cones)
    m = np.asarray(mask, dtype=bool).reshape(g.N)
    w = np.where(m, weight, 1.0)
    return np.broadcast_to(w, (g.T,) + g.N).ravel().copy()


@dataclass
class State:
    """Iterate (phi, z, q, alpha, beta) of Algorithm 2 plus the penalty sigma."""
    g: Grid
    phi: np.ndarray
    z: np.ndarray
    q: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    sigma: float = 1.0
    k: int = 0
    history: list = field(default_factory=list)

    @classmethod
    def zeros(cls, g: Grid, sigma: float = 1.0) -> "State":
        """The initial point q = alpha = beta = 0 (0 lies in Q), sigma_0 = sigma."""
        return cls(g, np.zeros(g.n_nodes), np.zeros(g.K * g.n_cones), np.zeros(g.n_q),
                   np.zeros(g.n_q), np.zeros(g.K * g.n_cones), float(sigma))

    def copy(self) -> "State":
        return State(self.g, self.phi.copy(), self.z.copy(), self.q.copy(), self.alpha.copy(),
                     self.beta.copy(), self.sigma, self.k, list(self.history))


class Problem:
    """Discrete (weighted) DOT problem data: c (eq. (defc)) and omega (Sec. 5.4)."""

    def __init__(self, g: Grid, rho0, rho1, mask=None, obstacle_weight: float = 1e-6):
        self.g = g
        m0 = masses(np.asarray(rho0).reshape(g.N))
        m1 = masses(np.asarray(rho1).reshape(g.N))
        self.m0, self.m1 = m0, m1
        self.c = fill_c(g, m0, m1)
        self.omega = omega_from_mask(g, mask, obstacle_weight)


def iterate(prob: Problem, st: State, tau: float = 1.9):
    """One iteration of Algorithm 2 in place."""
    p = _Params(tau, st.sigma)
    _load().og_iterate(prob.g.ref, ctypes.byref(p), _ptr(prob.c), _ptr(prob.omega), _ptr(st.phi),
                       _ptr(st.z), _ptr(st.q), _ptr(st.alpha), _ptr(st.beta))
    st.k += 1


def kkt(prob: Problem, st: State) -> dict:
    out = np.zeros(NUM_KKT)
    _load().og_kkt(prob.g.ref, _ptr(prob.c), _ptr(prob.omega), _ptr(st.phi), _ptr(st.z),
                   _ptr(st.q), _ptr(st.alpha), _ptr(st.beta), _ptr(out))
    return dict(zip(KKT_NAMES, out.tolist()))


def solve(prob: Problem, st: State, tol: float = 1e-6, maxit: int = 100000, tau: float = 1.9,
          s_sigma: float = 1.25, s_r: float = 2.0, check_every: int = 10) -> dict:
    """Algorithm 2 with the sigma rule and eta_dot stopping test of Sec. 5.3, in place.

    Returns the final KKT dict plus 'iterations'; st.history gets one row per check:
    (iteration, sigma used, eta_dot, eta_P, ...)."""
    sig = ctypes.c_double(st.sigma)
    kk = np.zeros(NUM_KKT)
    cap = maxit // check_every + 1 if check_every > 0 else 1
    hist = np.zeros(cap * (NUM_KKT + 2))
    hl = ctypes.c_long(0)
    it = _load().og_solve(prob.g.ref, tau, ctypes.byref(sig), s_sigma, s_r, check_every, tol,
                          maxit, _ptr(prob.c), _ptr(prob.omega), _ptr(st.phi), _ptr(st.z),
                          _ptr(st.q), _ptr(st.alpha), _ptr(st.beta), _ptr(kk), _ptr(hist), cap,
                          ctypes.byref(hl))
    st.sigma = sig.value
    st.k += int(it)
    rows = hist[: hl.value * (NUM_KKT + 2)].reshape(hl.value, NUM_KKT + 2)
    st.history.extend(rows.tolist())
    res = dict(zip(KKT_NAMES, kk.tolist()))
    res["iterations"] = int(it)
    return res


def density_slices(g: Grid, st: State) -> np.ndarray:
    """rho on G^s_0 as a density (mass per unit area) per time slice: alpha_0 / h_0
    (Proposition 3.3; c carries densities, see og_fill_c).  Each slice integrates
    to sum(rho) * cell_area = 1."""
    return st.alpha[: g.n_cones].reshape((g.T,) + g.N) * g.T


def cell_area(g: Grid) -> float:
    """|X_i| = h_1 ... h_D, the spatial cell volume."""
    return float(np.prod([1.0 / n for n in g.N]))


def w2_squared(g: Grid, primal_obj: float) -> float:
    """Squared W2 of the discrete problem from <c, phi>: -2 |X_i| <c, phi>."""
    return -2.0 * cell_area(g) * primal_obj


def momentum(g: Grid, st: State):
    """m_d on G^s_d as alpha_d / h_0 (Proposition 3.3)."""
    return [a * g.T for a in g.split_q(st.alpha)[1:]]
