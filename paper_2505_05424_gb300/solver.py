"""Python binding of the C ABI in include/dot.h (argument marshalling only).

Every step of the solve runs in the CUDA library; PyTorch supplies the device
workspace (one uint8 tensor of dot_workspace_bytes) and the stream.  There is no
CPU path: constructing a solver without a CUDA device or without the built
library raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N


class DotError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dot error {code}: {msg}")
        self.code = code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(D: int, T: int, N_) -> N.DotGrid:
    Ns = [int(N_)] * D if np.isscalar(N_) else [int(n) for n in N_]
    return N.DotGrid(int(D), int(T), (ctypes.c_int * 3)(*(Ns + [1] * (3 - len(Ns)))))


def default_options(prec: str = "mixed", **kw) -> N.DotOptions:
    lib = N.load()
    o = N.DotOptions()
    lib.dot_default_options(ctypes.byref(o))
    o.prec = {"fp64": N.DOT_FP64, "mixed": N.DOT_MIXED}[prec]
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def dot_workspace_bytes(D: int, T: int, N_, prec: str = "mixed") -> int:
    g = make_grid(D, T, N_)
    return int(N.load().dot_workspace_bytes(ctypes.byref(g), {"fp64": N.DOT_FP64, "mixed": N.DOT_MIXED}[prec]))


class DotSolver:
    """One DOT solve on the current CUDA device: dot_create on construction.

    Shapes: rho0/rho1/mask (N,)*D; phi (T+1, N..); rho (T, N..); m a list of D arrays."""

    def __init__(self, D: int, T: int, N_, rho0, rho1, mask=None, prec: str = "mixed", device=None,
                 stream=None, **options):
        import torch  # device memory and streams only
        if not torch.cuda.is_available():
            raise RuntimeError("DotSolver needs a CUDA device (no CPU fallback)")
        self.lib = N.load()
        self.D, self.T = int(D), int(T)
        self.N = tuple([int(N_)] * D if np.isscalar(N_) else [int(n) for n in N_])
        self.grid = make_grid(D, T, self.N)
        self.opt = default_options(prec, **options)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        nbytes = int(self.lib.dot_workspace_bytes(ctypes.byref(self.grid), self.opt.prec))
        if nbytes == 0:
            raise DotError(N.DOT_EINVAL, "invalid grid")
        with torch.cuda.device(dev):
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            self.stream = torch.cuda.current_stream(dev) if stream is None else stream
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        r0, r1 = _f64(rho0).reshape(-1), _f64(rho1).reshape(-1)
        P = int(np.prod(self.N))
        if r0.size != P or r1.size != P:
            raise DotError(N.DOT_EINVAL, f"densities must have {P} entries")
        m = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
            if m.size != P:
                raise DotError(N.DOT_EINVAL, "mask size mismatch")
        ctx = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = self.lib.dot_create(ctypes.byref(self.grid), _dp(r0), _dp(r1),
                                     None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     ctypes.byref(self.opt), ctypes.c_void_p(aligned), ctypes.c_size_t(nbytes),
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if rc != N.DOT_OK:
            raise DotError(rc, self.lib.dot_last_error(None).decode())
        self.ctx = ctx
        self.workspace_bytes = nbytes

    # -- helpers -------------------------------------------------------------
    def _check(self, rc: int, allow=(N.DOT_OK,)):
        if rc not in allow:
            raise DotError(rc, self.lib.dot_last_error(self.ctx).decode())
        return rc

    @property
    def n_nodes(self):
        return (self.T + 1) * int(np.prod(self.N))

    @property
    def n_cones(self):
        return self.T * int(np.prod(self.N))

    def face_shape(self, fam: int):
        if fam == 0:
            return (self.T,) + self.N
        s = [self.T + 1] + list(self.N)
        s[fam] -= 1
        return tuple(s)

    @property
    def n_q(self):
        return sum(int(np.prod(self.face_shape(f))) for f in range(self.D + 1))

    @property
    def K(self):
        return 4 * self.D + 2

    # -- C ABI mirrors ---------------------------------------------------------
    def dot_solve(self, tol: float = 1e-6, maxit: int = 100000) -> int:
        return self._check(self.lib.dot_solve(self.ctx, float(tol), int(maxit)), (N.DOT_OK, N.DOT_ENOTCONV))

    def dot_kkt(self) -> dict:
        out = np.zeros(N.DOT_KKT_LEN)
        self._check(self.lib.dot_kkt(self.ctx, _dp(out)))
        return dict(zip(N.KKT_NAMES, out.tolist()))

    def dot_get(self):
        """(rho [T,N..], m [D arrays], phi [T+1,N..], objective, kkt dict)."""
        rho = np.zeros(self.face_shape(0))
        nm = sum(int(np.prod(self.face_shape(f))) for f in range(1, self.D + 1))
        m = np.zeros(nm)
        phi = np.zeros((self.T + 1,) + self.N)
        obj = ctypes.c_double(0.0)
        kk = np.zeros(N.DOT_KKT_LEN)
        self._check(self.lib.dot_get(self.ctx, _dp(rho), _dp(m), _dp(phi), ctypes.byref(obj), _dp(kk)))
        ms, off = [], 0
        for f in range(1, self.D + 1):
            n = int(np.prod(self.face_shape(f)))
            ms.append(m[off:off + n].reshape(self.face_shape(f)))
            off += n
        return rho, ms, phi, obj.value, dict(zip(N.KKT_NAMES, kk.tolist()))

    def dot_get_state(self):
        q, al = np.zeros(self.n_q), np.zeros(self.n_q)
        beta = np.zeros(self.K * self.n_cones)
        sig = ctypes.c_double(0.0)
        it = ctypes.c_long(0)
        self._check(self.lib.dot_get_state(self.ctx, _dp(q), _dp(al), _dp(beta), ctypes.byref(sig),
                                           ctypes.byref(it)))
        return q, al, beta, sig.value, it.value

    def dot_set_state(self, q, alpha, beta, sigma: float, iters: int = 0):
        q, al, b = _f64(q).ravel(), _f64(alpha).ravel(), _f64(beta).ravel()
        if q.size != self.n_q or al.size != self.n_q or b.size != self.K * self.n_cones:
            raise DotError(N.DOT_EINVAL, "state size mismatch")
        self._check(self.lib.dot_set_state(self.ctx, _dp(q), _dp(al), _dp(b), float(sigma), int(iters)))

    def dot_poisson(self, b):
        b = _f64(b).ravel()
        if b.size != self.n_nodes:
            raise DotError(N.DOT_EINVAL, "b size mismatch")
        phi = np.zeros(self.n_nodes)
        self._check(self.lib.dot_poisson(self.ctx, _dp(b), _dp(phi)))
        return phi

    def dot_solve_multilevel(self, levels: int, tol: float = 1e-6, maxit: int = 100000, coarse_tol: float = 0.0):
        """(status, iterations per level, finest first) of dot_solve_multilevel;
        coarse_tol <= 0 selects the paper's per-level tolerance."""
        it = (ctypes.c_long * (int(levels) + 1))()
        rc = self.lib.dot_solve_multilevel(self.ctx, int(levels), float(tol), float(coarse_tol), int(maxit), it)
        if rc not in (N.DOT_OK, N.DOT_ENOTCONV):
            raise DotError(rc, self.lib.dot_multilevel_last_error().decode())
        return rc, [int(v) for v in it]

    def dot_profile(self, enable: bool = True):
        self._check(self.lib.dot_profile(self.ctx, int(bool(enable))))

    def dot_profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since dot_profile(True)."""
        n = 16
        ms = np.zeros(n)
        cnt = (ctypes.c_long * n)()
        k = self.lib.dot_profile_read(self.ctx, _dp(ms), cnt, n)
        return {self.lib.dot_kernel_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}

    def launch_count(self) -> int:
        return int(self.lib.dot_launch_count(self.ctx))

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.dot_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dot_poisson_f32_noalloc(D: int, T: int, N_, b, phi, stream=None) -> None:
    """Binding of dot_poisson_f32_noalloc (see include/dot.h): b is a CUDA float32
    tensor of (T+1) * prod(N) entries, phi a CUDA float32 tensor of twice that many
    (hi, lo pairs).  Raises DotError on a non-zero status."""
    lib = N.load()
    g = make_grid(D, T, N_)
    s = 0 if stream is None else stream.cuda_stream
    rc = lib.dot_poisson_f32_noalloc(ctypes.byref(g), ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(s))
    if rc != N.DOT_OK:
        raise DotError(rc, lib.dot_noalloc_last_error().decode())


class DotServer:
    """Binding of the dot_server_* functions (see include/dot.h): many DOT solves
    of mixed grids advanced together on the current CUDA device.

    submit() returns a request id; wait() blocks until it finished; result()
    returns (objective, kkt dict, times (submit, admit, done) in seconds since the
    server started, and rho/m/phi when the request kept its fields).  The keyword
    arguments are the fields of dot_server_options (multilevel > 0: the multilevel
    warm start for requests of at least multilevel_min_nodes nodes, obstacle
    requests only with multilevel_masked); **options are those of dot_options."""

    STATS = ("queued", "running", "finished", "batches", "bytes", "graph_launches", "kernel_launches",
             "peak_running", "peak_batches")

    def __init__(self, hbm_budget: int = 0, max_slots: int = 64, target_nodes: int = 4194304,
                 use_graphs: bool = True, idle_ms: int = 200, multilevel: int = 0,
                 multilevel_min_nodes: int = 1000000, multilevel_coarse_tol: float = 0.0,
                 multilevel_masked: bool = False, **options):
        import torch  # the device only
        if not torch.cuda.is_available():
            raise RuntimeError("DotServer needs a CUDA device (no CPU fallback)")
        torch.cuda.init()
        self.lib = N.load()
        self.opt = default_options("mixed", **options)
        so = N.DotServerOptions()
        self.lib.dot_server_default_options(ctypes.byref(so))
        so.hbm_budget = int(hbm_budget)
        so.max_slots = int(max_slots)
        so.target_nodes = int(target_nodes)
        so.use_graphs = int(bool(use_graphs))
        so.idle_ms = int(idle_ms)
        so.multilevel = int(multilevel)
        so.multilevel_min_nodes = int(multilevel_min_nodes)
        so.multilevel_coarse_tol = float(multilevel_coarse_tol)
        so.multilevel_masked = int(bool(multilevel_masked))
        srv = ctypes.c_void_p()
        rc = self.lib.dot_server_create(ctypes.byref(self.opt), ctypes.byref(so), ctypes.byref(srv))
        if rc != N.DOT_OK:
            raise DotError(rc, self.lib.dot_server_last_error(None).decode())
        self.srv = srv
        self._shapes = {}

    def _check(self, rc: int, allow=(N.DOT_OK,)):
        if rc not in allow:
            raise DotError(rc, self.lib.dot_server_last_error(self.srv).decode())
        return rc

    def submit(self, D: int, T: int, N_, rho0, rho1, mask=None, tol: float = 1e-6, maxit: int = 100000,
               keep_fields: bool = True) -> int:
        Ns = tuple([int(N_)] * D if np.isscalar(N_) else [int(n) for n in N_])
        g = make_grid(D, T, Ns)
        r0, r1 = _f64(rho0).reshape(-1), _f64(rho1).reshape(-1)
        P = int(np.prod(Ns))
        if r0.size != P or r1.size != P:
            raise DotError(N.DOT_EINVAL, f"densities must have {P} entries")
        m = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
            if m.size != P:
                raise DotError(N.DOT_EINVAL, "mask size mismatch")
        rid = ctypes.c_longlong(0)
        self._check(self.lib.dot_server_submit(
            self.srv, ctypes.byref(g), _dp(r0), _dp(r1),
            None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            float(tol), int(maxit), int(bool(keep_fields)), ctypes.byref(rid)))
        self._shapes[rid.value] = (int(D), int(T), Ns, bool(keep_fields))
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0):
        """The solve status (as dot_solve returns it), or None on timeout."""
        st = ctypes.c_int(0)
        rc = self.lib.dot_server_wait(self.srv, int(rid), float(timeout), ctypes.byref(st))
        if rc == N.DOT_ETIMEOUT:
            return None
        self._check(rc)
        return st.value

    def result(self, rid: int) -> dict:
        if rid not in self._shapes:
            raise DotError(N.DOT_EINVAL, f"unknown request id {rid}")
        D, T, Ns, keep = self._shapes[rid]
        obj = ctypes.c_double(0.0)
        kk = np.zeros(N.DOT_KKT_LEN)
        times = np.zeros(3)
        out = {}
        if keep:
            rho = np.zeros((T,) + Ns)
            nm = sum((T + 1) * int(np.prod(Ns)) // Ns[d] * (Ns[d] - 1) for d in range(D))
            m = np.zeros(nm)
            phi = np.zeros((T + 1,) + Ns)
            self._check(self.lib.dot_server_result(self.srv, int(rid), _dp(rho), _dp(m), _dp(phi),
                                                   ctypes.byref(obj), _dp(kk), _dp(times)))
            out.update(rho=rho, m=m, phi=phi)
        else:
            self._check(self.lib.dot_server_result(self.srv, int(rid), None, None, None, ctypes.byref(obj),
                                                   _dp(kk), _dp(times)))
        out.update(objective=obj.value, kkt=dict(zip(N.KKT_NAMES, kk.tolist())), times=tuple(times.tolist()))
        return out

    def release(self, rid: int):
        self._check(self.lib.dot_server_release(self.srv, int(rid)))
        self._shapes.pop(rid, None)

    def stats(self) -> dict:
        out = np.zeros(len(self.STATS))
        k = self.lib.dot_server_stats(self.srv, _dp(out), len(self.STATS))
        return dict(zip(self.STATS[:k], out[:k].tolist()))

    def close(self):
        if getattr(self, "srv", None) is not None and self.srv.value:
            self.lib.dot_server_destroy(self.srv)
            self.srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dot_prolong_state(D: int, Tc: int, Nc, Tf: int, Nf, q, alpha, beta):
    """Binding of dot_prolong_state (host only): the coarse state (q, alpha, beta in
    the layouts of dot_get_state) interpolated onto the fine grid."""
    lib = N.load()
    gc, gf = make_grid(D, Tc, Nc), make_grid(D, Tf, Nf)
    Ns = [int(Nf)] * D if np.isscalar(Nf) else [int(n) for n in Nf]
    Pf = int(np.prod(Ns))
    nq = Tf * Pf + sum((Tf + 1) * (Pf // Ns[d]) * (Ns[d] - 1) for d in range(D))
    nb = (4 * D + 2) * Tf * Pf
    qf, af, bf = np.zeros(nq), np.zeros(nq), np.zeros(nb)
    q, alpha, beta = _f64(q).ravel(), _f64(alpha).ravel(), _f64(beta).ravel()
    rc = lib.dot_prolong_state(ctypes.byref(gc), ctypes.byref(gf), _dp(q), _dp(alpha), _dp(beta), _dp(qf),
                               _dp(af), _dp(bf))
    if rc != N.DOT_OK:
        raise DotError(rc, lib.dot_multilevel_last_error().decode())
    return qf, af, bf
