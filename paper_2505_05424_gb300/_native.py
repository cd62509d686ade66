"""Build and load the CUDA library (libdot_gb300.so) and declare its C ABI for ctypes.

The library is compiled in-tree for sm_103a only.  There is no fallback: when the
library or a CUDA device is missing every solver call raises.
"""
from __future__ import annotations

import ctypes
import glob
import os
import shutil
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_BUILD, "libdot_gb300.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdot_gb300.so")


def _sources():
    return sorted(glob.glob(os.path.join(_CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(_CSRC, "*.cuh")) + [os.path.join(_INCLUDE, "dot.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ in parallel and link libdot_gb300.so."""
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(p) <= t for p in _deps()):
            return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in _sources():
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-I", _INCLUDE, "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + cuda_lib]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class DotGrid(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("T", ctypes.c_int), ("N", ctypes.c_int * 3)]


class DotOptions(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tau", ctypes.c_double), ("sigma0", ctypes.c_double),
                ("s_sigma", ctypes.c_double), ("s_r", ctypes.c_double), ("check_every", ctypes.c_int),
                ("obstacle_weight", ctypes.c_double), ("max_seconds", ctypes.c_double), ("use_graphs", ctypes.c_int),
                ("tau_switch_below", ctypes.c_double)]


class DotServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("target_nodes", ctypes.c_long),
                ("use_graphs", ctypes.c_int), ("idle_ms", ctypes.c_int), ("multilevel", ctypes.c_int),
                ("multilevel_min_nodes", ctypes.c_longlong), ("multilevel_coarse_tol", ctypes.c_double),
                ("multilevel_masked", ctypes.c_int)]


DOT_OK, DOT_EINVAL, DOT_ENOMEM, DOT_ECUDA, DOT_EDIVERGED, DOT_ETIMEOUT, DOT_ENOTCONV = 0, -1, -2, -3, -4, -5, 1
DOT_FP64, DOT_MIXED = 0, 1
KKT_NAMES = ("eta_dot", "eta_P", "eta_D", "eta_C", "eta_P_soc", "eta_D_soc", "primal_obj", "dual_obj",
             "gap", "iterations", "sigma")
DOT_KKT_LEN = len(KKT_NAMES)

# Every symbol include/dot.h declares.
EXPORTS = ("dot_default_options", "dot_workspace_bytes", "dot_create", "dot_solve", "dot_get", "dot_kkt",
           "dot_get_state", "dot_set_state", "dot_poisson", "dot_destroy", "dot_last_error", "dot_version",
           "dot_launch_count", "dot_profile", "dot_profile_read", "dot_kernel_name", "dot_poisson_f32_noalloc",
           "dot_noalloc_last_error", "dot_server_default_options", "dot_server_create", "dot_server_submit",
           "dot_server_wait", "dot_server_result", "dot_server_release", "dot_server_stats",
           "dot_server_destroy", "dot_server_last_error", "dot_solve_multilevel", "dot_prolong_state",
           "dot_multilevel_last_error", "dot_selftest_pipeline_timeout")

_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libdot_gb300.so (building it first if allowed) and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError("libdot_gb300.so is not built (run __graft_entry__.build())")
            build()
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        vp = ctypes.c_void_p
        lib.dot_default_options.argtypes = [P(DotOptions)]
        lib.dot_default_options.restype = None
        lib.dot_workspace_bytes.argtypes = [P(DotGrid), ctypes.c_int]
        lib.dot_workspace_bytes.restype = ctypes.c_size_t
        lib.dot_create.argtypes = [P(DotGrid), dp, dp, P(ctypes.c_uint8), P(DotOptions), vp, ctypes.c_size_t, vp,
                                   P(vp)]
        lib.dot_create.restype = ctypes.c_int
        lib.dot_solve.argtypes = [vp, ctypes.c_double, ctypes.c_long]
        lib.dot_solve.restype = ctypes.c_int
        lib.dot_get.argtypes = [vp, dp, dp, dp, dp, dp]
        lib.dot_get.restype = ctypes.c_int
        lib.dot_kkt.argtypes = [vp, dp]
        lib.dot_kkt.restype = ctypes.c_int
        lib.dot_get_state.argtypes = [vp, dp, dp, dp, dp, P(ctypes.c_long)]
        lib.dot_get_state.restype = ctypes.c_int
        lib.dot_set_state.argtypes = [vp, dp, dp, dp, ctypes.c_double, ctypes.c_long]
        lib.dot_set_state.restype = ctypes.c_int
        lib.dot_poisson.argtypes = [vp, dp, dp]
        lib.dot_poisson.restype = ctypes.c_int
        lib.dot_destroy.argtypes = [vp]
        lib.dot_destroy.restype = None
        lib.dot_last_error.argtypes = [vp]
        lib.dot_last_error.restype = ctypes.c_char_p
        lib.dot_version.argtypes = []
        lib.dot_version.restype = ctypes.c_char_p
        lib.dot_launch_count.argtypes = [vp]
        lib.dot_launch_count.restype = ctypes.c_long
        lib.dot_profile.argtypes = [vp, ctypes.c_int]
        lib.dot_profile.restype = ctypes.c_int
        lib.dot_profile_read.argtypes = [vp, dp, P(ctypes.c_long), ctypes.c_int]
        lib.dot_profile_read.restype = ctypes.c_int
        lib.dot_kernel_name.argtypes = [ctypes.c_int]
        lib.dot_kernel_name.restype = ctypes.c_char_p
        lib.dot_poisson_f32_noalloc.argtypes = [P(DotGrid), vp, vp, vp]
        lib.dot_poisson_f32_noalloc.restype = ctypes.c_int
        lib.dot_noalloc_last_error.argtypes = []
        lib.dot_noalloc_last_error.restype = ctypes.c_char_p
        lib.dot_server_default_options.argtypes = [P(DotServerOptions)]
        lib.dot_server_default_options.restype = None
        lib.dot_server_create.argtypes = [P(DotOptions), P(DotServerOptions), P(vp)]
        lib.dot_server_create.restype = ctypes.c_int
        lib.dot_server_submit.argtypes = [vp, P(DotGrid), dp, dp, P(ctypes.c_uint8), ctypes.c_double, ctypes.c_long,
                                          ctypes.c_int, P(ctypes.c_longlong)]
        lib.dot_server_submit.restype = ctypes.c_int
        lib.dot_server_wait.argtypes = [vp, ctypes.c_longlong, ctypes.c_double, P(ctypes.c_int)]
        lib.dot_server_wait.restype = ctypes.c_int
        lib.dot_server_result.argtypes = [vp, ctypes.c_longlong, dp, dp, dp, dp, dp, dp]
        lib.dot_server_result.restype = ctypes.c_int
        lib.dot_server_release.argtypes = [vp, ctypes.c_longlong]
        lib.dot_server_release.restype = ctypes.c_int
        lib.dot_server_stats.argtypes = [vp, dp, ctypes.c_int]
        lib.dot_server_stats.restype = ctypes.c_int
        lib.dot_server_destroy.argtypes = [vp]
        lib.dot_server_destroy.restype = None
        lib.dot_server_last_error.argtypes = [vp]
        lib.dot_server_last_error.restype = ctypes.c_char_p
        lib.dot_solve_multilevel.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                             P(ctypes.c_long)]
        lib.dot_solve_multilevel.restype = ctypes.c_int
        lib.dot_prolong_state.argtypes = [P(DotGrid), P(DotGrid), dp, dp, dp, dp, dp, dp]
        lib.dot_prolong_state.restype = ctypes.c_int
        lib.dot_multilevel_last_error.argtypes = []
        lib.dot_multilevel_last_error.restype = ctypes.c_char_p
        lib.dot_selftest_pipeline_timeout.argtypes = [ctypes.c_int, dp, P(ctypes.c_int)]
        lib.dot_selftest_pipeline_timeout.restype = ctypes.c_int
        _lib = lib
        return lib
